// lbm_internal.cuh -- device-side types, lattice tables and helpers shared by
// the kernels and the runtime of the GB300 coupled LBM / rigid-body step.
//
// Data layout in HBM (one handle):
//   pop[2]     populations, SoA [19][C] of the storage type, ping-pong by step
//              parity; stored as deviations delta_a = f_a - w_a (FP16 scaled)
//   flags[2]   uint8 per cell and flag epoch (bits below), ping-pong by parity
//   bid[2]     uint8 body id of solid cells per epoch (0xFF: none)
//   bodies[2]  BodyState per body (FP64), ping-pong: state n and n-1 / n+1
//   links      per (body, z-plane) segments of fluid->solid links
// C = nx * ny * nz, cell index c = (z * ny + y) * nx + x.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

constexpr int Q = 19;

// D3Q19 velocity set (Qian, d'Humieres, Lallemand), in the order of lbm.h,
// as constexpr functions so that unrolled loops fold them to immediates.
__host__ __device__ constexpr int ex(int a) {
    switch (a) {
    case 1: case 7: case 9: case 11: case 13: return 1;
    case 2: case 8: case 10: case 12: case 14: return -1;
    default: return 0;
    }
}
__host__ __device__ constexpr int ey(int a) {
    switch (a) {
    case 3: case 7: case 10: case 15: case 17: return 1;
    case 4: case 8: case 9: case 16: case 18: return -1;
    default: return 0;
    }
}
__host__ __device__ constexpr int ez(int a) {
    switch (a) {
    case 5: case 11: case 14: case 15: case 18: return 1;
    case 6: case 12: case 13: case 16: case 17: return -1;
    default: return 0;
    }
}
// opposite direction: pairs (1,2), (3,4), ... are each other's reverse
__host__ __device__ constexpr int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
// weights 1/3 (rest), 1/18 (axes), 1/36 (diagonals)
__host__ __device__ constexpr double wgt(int a) { return a == 0 ? 1.0 / 3.0 : (a < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

// flag bits of one cell in epoch n
constexpr uint8_t F_SOLID = 1;      // solid at n
constexpr uint8_t F_SOLID_PREV = 2; // solid at n-1 (uncovered if F_SOLID is clear)
constexpr uint8_t F_NEAR = 4;       // some neighbour x - e_b was solid at n-1
constexpr uint8_t F_WALL = 8;       // some neighbour lies beyond a no-slip wall
constexpr uint8_t NO_BODY = 0xFF;

// device status word bits
constexpr int ST_OVERLAP = 1, ST_OUTSIDE = 2, ST_NAN = 4, ST_UNSTABLE = 8, ST_LINKS = 16, ST_TIMEOUT = 32;

// cells added around a body's extent in the remap region (the cube of
// half-width E + REMAP_MARGIN around floor(X)).  The remap of step n
// rewrites the buffer that holds epoch n-2, so the cube must hold every
// cell solid in epochs n-3 .. n and the neighbours of those solid in n-3
// and n-1.  A solid cell lies within reach = r + l/2 of its epoch's centre
// on each axis, the centre moves at most MAX_STEP = 0.5 per step and axis,
// so these cells lie within reach + 1.5 + 1 of X_n: at most
// floor(X) + ceil(reach) + 3 = floor(X) + E + 2 above and less below.  One
// cell more is kept as a spare.
constexpr int REMAP_MARGIN = 3;
constexpr double MAX_STEP = 0.5;
constexpr int FORCE_BLOCKS = 8;     // blocks per body in the momentum-exchange sum
constexpr int LBM_MAX_BODIES_DEV = 254;

struct BodyProps {
    int shape;          // 0 sphere, 1 capsule
    int E;              // ceil(r + l/2) + 1: half-width of the box that holds every solid cell
    float r2f, hf, marginf;     // r^2, l / 2 and the FP32 inside test's margin, in FP32
    double r, l, m, volume;
    double reach;       // r + l / 2
    double inertia[3];      // body-frame principal moments of inertia
    double inv_m, inv_inertia[3];
    int drive_first, drive_count;   // this body's drive terms, in term order
    int spring_first, spring_count; // this body's springs, in spring order (per-body list)
};

struct BodyState {      // 13 doubles, the layout of lbm_get_bodies
    double X[3], q[4], V[3], W[3];
};

struct Spring {
    int i, j;
    double k, rest, gamma;
};

struct DriveTerm {
    int body;
    double amp, freq, phase, t_off;
    double omega, t_on;     // 2 pi freq and phase / omega
    double axis[3];         // body-frame direction (default the body x axis)
};

struct Link {
    uint32_t cell;
    uint32_t dir;
};

// One body state in the forms the cell kernels use: integers and FP32, so
// that no per-cell path needs the (slow) FP64 pipe.  The rigid-body step
// writes the record of the state it produces; prep_kernel checks each
// slot's stamp against the state in use and remakes it when they differ.
struct BodyGeom {
    int origin[3];          // corner of the body's remap cube, floor(X) - (E + REMAP_MARGIN), wrapped into [0, n) on periodic axes
    int ci[3];              // centre wrapped into the domain: its cell ...
    float cf[3];            // ... and its position within that cell
    float ax[3];            // body x axis (a capsule's axis)
    float v[3], w[3];       // velocity and angular velocity
    float r2, h, margin;    // r^2, l / 2 and the margin of the FP32 inside test
    int shape;
    int side;               // edge of the remap cube, 2 (E + REMAP_MARGIN) + 1
    int ncand;              // state n: bodies whose grown box meets this body's remap cube (cand list; the batched remap's)
    int box[6];             // per axis: lower corner (wrapped) and width of [floor(X - reach), floor(X + reach)]
    int ebox[6];            // the same grown by STATIC_REACH cells
    double cfd[3];          // the position within the cell in FP64
};

// momentum-exchange sums of 32/16-bit storage: FP32 link terms rounded to
// multiples of 2^-FIX_BITS and added as 64-bit integers (exact, so the sum
// does not depend on the order in which blocks add their parts).  With
// |term| < 2^9 (the force kernel's bound) a sum of 2^13 terms stays in range.
constexpr int FIX_BITS = 40;

struct Domain {
    int nx, ny, nz;
    int px, py, pz;     // periodic flags
    long long C;
    double inx, iny, inz;   // 1 / n per axis
};

__host__ __device__ inline int wrap_axis(int i, int n) {
    // i in [-n, 2n)
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// periodic minimum image d - n k with k the integer nearest to d / n
// (a multiply and a floor: FP64 division is slow on this part)
__device__ inline double min_image(double d, int n, double inv_n, int periodic) {
    return periodic ? d - n * floor(d * inv_n + 0.5) : d;
}

__device__ inline void quat_to_matrix(const double q[4], double R[3][3]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

// offset of lattice point p from the body centre (periodic minimum image)
__device__ inline void offset_from(const Domain &d, const BodyState &b, double px, double py,
                                   double pz, double o[3]) {
    o[0] = min_image(px - b.X[0], d.nx, d.inx, d.px);
    o[1] = min_image(py - b.X[1], d.ny, d.iny, d.py);
    o[2] = min_image(pz - b.X[2], d.nz, d.inz, d.pz);
}

// velocity of the body surface at lattice point p: V + Omega x (p - X)
__device__ inline void surface_velocity(const Domain &d, const BodyState &b, double px, double py,
                                        double pz, double u[3]) {
    double o[3];
    offset_from(d, b, px, py, pz, o);
    u[0] = b.V[0] + (b.W[1] * o[2] - b.W[2] * o[1]);
    u[1] = b.V[1] + (b.W[2] * o[0] - b.W[0] * o[2]);
    u[2] = b.V[2] + (b.W[0] * o[1] - b.W[1] * o[0]);
}

// Recording of a forward run for the reverse sweep: when `on`, the rigid-body
// step t writes the state t + 1 and the hydrodynamic load of step t.
struct TapeCtl {
    double *state;      // [cap + 2][nb][13]: index t - t0 + 1 holds the state of step t
    double *force;      // [cap][nb][6]: index t - t0 holds force and torque of step t
    long long t0;       // first recorded step
    int cap;            // steps the buffers hold
    int on;
};

// kernel launch parameters of one step
struct StepPtrs {
    const void *src;        // populations of step n-1
    void *dst;              // populations of step n
    const uint8_t *flags_prev, *bid_prev;   // epoch n-1
    uint8_t *flags_cur, *bid_cur;           // epoch n
    const BodyState *body_prev;             // state n-1
    const BodyState *body_cur;              // state n
    BodyState *body_next;                   // state n+1
    // overlapped steps: the tiles of step n near a body, which the bulk
    // kernel leaves to the near kernel (null: the bulk kernel does every cell)
    const unsigned *far_skip;
    const long long *tstep;                 // step index n (the BF16 rounding bits' counter)
    int parity;
};

// Overlapped steps.  The bulk kernel of step n needs only the populations of
// step n-1 where no body is near: outside the remap cubes flags are static
// in every epoch.  The tiles of TILE_X cells of an x-row that meet the remap
// cube of any body at state n-1 grown by one cell (which holds the cube at
// state n: a body moves at most half a cell a step) are near tiles; the bulk
// kernel skips them and the near kernel does them after the remap.  So the
// far part of step n's bulk runs beside the force and rigid-body step of
// step n-1 and the remap of step n.  An option (LBM_OPT_OVERLAP), not the
// default: the bulk kernel needs nearly every SM's memory parallelism to
// hold HBM at its peak, so short kernels that share the SMs with it slow it
// by about as much as their own time (measured on the 33.5 M-cell capsule
// swarm: 0.889 ms a step overlapped against 0.872 ms serial).
constexpr int TILE_X = 64;

struct Device {
    Domain dom;
    int precision;          // LBM_PREC_*
    int vec;                // cells per thread of the bulk stream-collide kernel
    int minb;               // its minimum resident blocks per SM (0: the default variant)
    int nb, ns, nd;
    double tau, omega, g[3];
    float omega_f, guo_f, g_f[3];   // omega, 1 - omega / 2 and g rounded to FP32 once (the FP32 collision's)
    float om1_f, ow_f[3], gw_f[3];  // 1 - omega; omega w and (1 - omega / 2) w per weight class (rest, axis, diagonal)
    int forced;
    int avg_force;          // the rigid-body step uses the mean load of steps n and n-1
    float f16_scale, f16_inv_scale;
    const BodyProps *props;
    const Spring *springs;
    const DriveTerm *drives;
    const int *spring_list; // per-body spring indices (BodyProps::spring_first/count)
    double *fh;             // [nb][6] force, torque of the last step
    double *fpart;          // [nb][FORCE_BLOCKS][6] per-block partial sums of the force kernel (FP64 storage)
    long long *fx;          // [nb][6] 32/16-bit storage: fixed-point sums of the variable link terms
    int *fi;                // [nb][6] 32/16-bit storage: integer sums of the constant link terms
    BodyGeom *geom;         // [2][nb]: slot p holds the geometry of the state in body buffer p (parity)
    BodyState *gstamp;      // [2][nb]: the state each slot was made from (prep_kernel remakes on mismatch)
    long long blist_cap;
    uint8_t *cand;          // [nb][nb]: body b's remap candidates in body order (BodyGeom::ncand of them)
    float *rho_near;        // [C] 32/16-bit storage: rho - 1 of each cell the boundary kernel collided this step
    uint32_t *blist;        // cells the remap found fluid with F_NEAR or F_SOLID_PREV (the boundary kernel's)
    int *bcount;            // entries in blist (a cell in two bodies' cubes may appear twice)
    double *drive_f;        // [nd][3] drive forces of the current step (integrator scratch)
    double *spring_f;       // [ns][3] spring forces on body i of each spring (integrator scratch)
    unsigned *blocks_done;  // bodies whose rigid-body step finished in the current step
    unsigned *body_done;    // [nb] force blocks of each body finished in the current step
    Link *links;            // [nb][link_side][seg_cap]
    int *seg_count;         // [nb][link_side]
    int link_side, seg_cap, remap_side;
    int *status;
    int *changed;           // [2]: some cell changed solidity or body in epoch parity p
    long long *t_dev;       // step counter seen by the drive
    double *hist;           // [hist_cap][nb][13] or null
    int hist_cap;
    TapeCtl *tape;          // recording switch of the reverse sweep, or null
    int expire_waits;       // checks of the timeout path: the row-staged kernel's first wait cannot succeed
    double *avg_u;          // [3][C] running sum of the velocity while an average is taken, or null
    long long *avg_n;       // steps added to avg_u
    // overlapped steps, by step parity: near-tile marks [tiles] (non-zero:
    // near), near-tile lists [near_cap] and their lengths [2], the step index
    int overlap;
    unsigned *near_mask[2];
    int *near_list[2];
    int *near_count;
    int near_cap;
    long long *tstep;       // [2]
    // launch the remap, bulk and force kernels with programmatic dependent
    // launch (pdl_enter, launch_kernel); the step graphs set it for the
    // remap and force kernels when LBM_DEBUG_NO_PDL is 0
    int pdl;
};

// Programmatic dependent launch, device side: wait until the grids this one
// depends on have completed with their writes visible (at once in a launch
// without such a dependency), then let the next grid of the stream start
// launching if it was launched with the attribute, so that its blocks are
// resident when this grid ends (the bulk kernel, launched without it, lets
// the force kernel in early).  A kernel launched with the attribute calls it
// before touching global memory.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Host side: launch `k`, with programmatic stream serialization when `pdl`
// (then `k` must begin with pdl_enter).  In a captured graph the edge from
// the kernel before it becomes a programmatic one.
template <typename... P, typename... A>
inline void launch_kernel(bool pdl, void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          A &&...args) {
    if (!pdl) {
        k<<<grid, block, smem, s>>>(static_cast<A &&>(args)...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1] = {};
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, static_cast<A &&>(args)...);
}

// ---- batched launches over the members of an ensemble ------------------------
//
// Each per-step kernel is a body run by a block at block coordinates within
// one lattice's grid: the launch's own (a single lattice), or, in a batched
// launch over several lattices (members), the block's place in its member's
// grid.  A batched launch flattens the members' grids into one 1-D grid:
// member m owns the blocks [first[m], first[m + 1]).  Its block looks up its
// member, copies the member's record and step pointers into shared memory
// and runs the same body, so one launch does the work of one launch per
// member, with no wait between blocks.
struct Blk {
    int x, y, z;        // block index within the lattice's grid
    int gx, gy, gz;     // that grid's dimensions
};

__device__ __forceinline__ Blk launch_blk() {
    return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x, (int)gridDim.y, (int)gridDim.z};
}

struct Batch {
    const Device *dv;       // [members] member records
    const StepPtrs *sp;     // [2][members] step pointers by step parity
    const int *first;       // [members + 1] first flattened block of each member (this kernel's grids)
    const int *grid;        // [members][3] each member's grid (this kernel's)
    const unsigned short *member;   // [blocks] the member of each flattened block
    int members;
    int parity;             // step parity of this launch
};


// the member record, step pointers and block coordinates of this block of a
// batched launch, in shared memory (every thread of the block calls this)
__device__ inline void batch_member(const Batch &bt, Device &sdv, StepPtrs &ssp, Blk &sbk) {
    __shared__ int s_m;
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
        const int blk = (int)blockIdx.x;
        const int m = bt.member[blk];       // first[m] <= blk < first[m + 1]
        s_m = m;
        const int l = blk - bt.first[m];
        const int gx = bt.grid[3 * m], gy = bt.grid[3 * m + 1], gz = bt.grid[3 * m + 2];
        sbk = Blk{l % gx, (l / gx) % gy, l / (gx * gy), gx, gy, gz};
    }
    __syncthreads();
    const int m = s_m;
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    static_assert(sizeof(Device) % 4 == 0 && sizeof(StepPtrs) % 4 == 0, "records are copied as words");
    const int *src = reinterpret_cast<const int *>(bt.dv + m);
    int *dst = reinterpret_cast<int *>(&sdv);
    for (int i = tid; i < (int)(sizeof(Device) / 4); i += nt) dst[i] = __ldg(src + i);
    const int *ssrc = reinterpret_cast<const int *>(bt.sp + bt.parity * bt.members + m);
    int *sdst = reinterpret_cast<int *>(&ssp);
    for (int i = tid; i < (int)(sizeof(StepPtrs) / 4); i += nt) sdst[i] = __ldg(ssrc + i);
    __syncthreads();
}

// the per-step kernels a batched step launches, in step order
enum BatchKernel { BK_PREP, BK_REMAP, BK_BOUNDARY, BK_WALLS, BK_LINKS, BK_LOADS, BK_BULK, BK_FORCE, BK_COUNT };

// the start of a batched kernel: sdv, ssp and sbk are this block's member
// record, step pointers and block coordinates
#define LBM_BATCH_MEMBER(bt)          \
    __shared__ Device sdv;            \
    __shared__ StepPtrs ssp;          \
    __shared__ Blk sbk;               \
    batch_member((bt), sdv, ssp, sbk)

// pointers of one reverse step n of the cell part (adjoint.cu)
struct AdjPtrs {
    const void *G;                  // post-collision populations of step n (storage type)
    const uint8_t *flags_cur;       // flags of epoch n
    const uint8_t *bid_cur;         // body ids of epoch n
    const uint8_t *bid_prev;        // body ids of epoch n-1 (the body an uncovered cell left)
    const uint8_t *flags_next;      // flags of epoch n+1
    const void *ain;                // [19][C] adjoint of the pre-collision populations of step n+1
    const void *rin;                // [C] density adjoint of the cells uncovered at step n+1
    void *aout;                     // [19][C] adjoint of the pre-collision populations of step n
    void *rout;                     // [C] density adjoint of the cells uncovered at step n
    const BodyState *body;          // state n
    const double *fadj;             // [nb][6] adjoint of force and torque of step n
    double *part;                   // [nb][part_stride][9] per-block body sums (X, V, W)
    int part_stride;
};

// pointers of the reversed rigid-body step n (adjoint.cu)
// Terms of the reversed rigid-body step n that depend only on the state S^n
// and the load of step n (adj_terms_kernel makes them for all steps of a
// segment at once, so that the reverse sweep's serial chain holds only the
// adjoint's own arithmetic).
struct AdjBodyTerms {
    double R[9];                    // R(q^n), row-major
    double F[3];                    // total force of step n
    double beta[3];                 // R^T T
    double W1[3];                   // Omega after the update
    double q1[4];                   // the renormalised quaternion
    double inv_nn;                  // 1 / |q before renormalisation|
};
struct AdjDriveTerms {
    double f, sn, cs;               // a sin(omega t - phase) (0 outside the window), its sine and cosine
    double aw[3];                   // R(q^n) axis: the term's world direction
};
struct AdjSpringTerms {
    double dir[3];                  // (X_i - X_j) / |X_i - X_j| (0 at zero length)
    double len;                     // |X_i - X_j|
    double ratio;                   // (len - rest) / len (0 at zero length)
    double dv[3];                   // V_i - V_j
};

struct AdjBody {
    const BodyState *state;         // state n
    const double *fh;               // [nb][6] hydrodynamic force and torque of step n
    const AdjBodyTerms *tb;         // [nb] state-only terms of step n
    const AdjDriveTerms *td;        // [nd]
    const AdjSpringTerms *ts;       // [ns]
    double *sa_next;                // [nb][13] adjoint of state n+1 (completed in place)
    double *sa_cur;                 // [nb][13] adjoint of state n (written)
    double *fadj;                   // [nb][6] adjoint of the hydrodynamic load (written)
    const double *part;             // cell sums of reverse step n+1
    int part_stride, part_count;
    double *grad_drive, *grad_spring, *grad_body;   // [nd][2], [ns][3], [nb][5] (added to)
    long long t;                    // step n
};

// ---- launch wrappers (kernels.cu / stream_collide.cu / adjoint.cu) ---------
void launch_init_flags(const Device &dv, uint8_t *flags0, uint8_t *flags1, uint8_t *bid0,
                       uint8_t *bid1, cudaStream_t s);
// the remap of a step, after the body preparation (geometry records remade
// where a state was set from outside, the boundary list emptied) unless
// `prep` is false: steps whose states the rigid-body step made skip it
void launch_remap(const Device &dv, const StepPtrs &sp, int init_mode, cudaStream_t s, bool prep = true);
void launch_prep(const Device &dv, const StepPtrs &sp, cudaStream_t s);
void launch_stream_collide(const Device &dv, const StepPtrs &sp, cudaStream_t s);
void launch_boundary_fix(const Device &dv, const StepPtrs &sp, cudaStream_t s);
bool needs_boundary_fix(const Device &dv);
bool valid_vector_width(const Device &dv, int v);
bool valid_variant(const Device &dv, int v, int minb);
int list_variants(const Device &dv, int *vec, int *minb, int max);
int default_vector_width(const Device &dv);
void prepare_bulk_variants();           // host: shared-memory opt-in of the staged variants (once)
void launch_links(const Device &dv, const StepPtrs &sp, cudaStream_t s);
void launch_force(const Device &dv, const StepPtrs &sp, cudaStream_t s);
void launch_integrate(const Device &dv, const StepPtrs &sp, int with_fluid, cudaStream_t s);
void launch_tick(const Device &dv, const StepPtrs &sp, cudaStream_t s);
// the near tiles of the step of parity q from the body states `states`
// (their remap cubes grown by one cell), and that step's index,
// t_dev + step_offset
void launch_near_tiles(const Device &dv, const BodyState *states, int q, int step_offset, cudaStream_t s);
void launch_near_bulk(const Device &dv, const StepPtrs &sp, cudaStream_t s);
long long near_tile_count(const Device &dv);     // tiles of the lattice (host)
int near_tile_cap(const Device &dv, int emax);   // most near tiles a step can have (host)
void launch_export(const Device &dv, const void *pop, const uint8_t *flags, const uint8_t *bid,
                   int what, int mask_solid, void *out, int dtype, cudaStream_t s);
void launch_import_pop(const Device &dv, void *pop, const double *in, cudaStream_t s);
void launch_average(const Device &dv, const StepPtrs &sp, cudaStream_t s);

// batched launches (ensembles): the grid g[3] of kernel k of lattice dv (all
// zero when it does not run), and one launch of k over `blocks` flattened
// blocks of the members of bt (all of storage `precision`); for BK_BULK,
// `variant` indexes the batched bulk shapes (batch_bulk_shape)
void batch_grid_small(const Device &dv, int k, int g[3]);                     // kernels.cu
void launch_batch_small(int k, const Batch &bt, unsigned blocks, int precision, cudaStream_t s);
void batch_grid_cells(const Device &dv, int k, int variant, int g[3]);        // stream_collide.cu
void launch_batch_cells(int k, int variant, const Batch &bt, unsigned blocks, int precision, cudaStream_t s);
// batched bulk shape i of a precision: its cells per thread, or 0 past the list
int batch_bulk_shape(int precision, int i);
int adjoint_part_stride(const Device &dv);
void launch_adj_integrate(const Device &dv, const AdjBody &ab, cudaStream_t s);
// the state-only terms of steps t0 .. t0 + L - 1 from the tape's states
// (state t0 + j at states + j nb) and loads (fh + 6 j nb)
void launch_adj_terms(const Device &dv, const BodyState *states, const double *fh, long long t0, int L,
                      AdjBodyTerms *tb, AdjDriveTerms *td, AdjSpringTerms *ts, cudaStream_t s);
void launch_adj_bulk(const Device &dv, const AdjPtrs &ap, bool first, cudaStream_t s);
void launch_adj_boundary(const Device &dv, const AdjPtrs &ap, bool first, cudaStream_t s);
void launch_adj_reduce(const Device &dv, const double *part, int stride, int count, double *sa, cudaStream_t s);

}  // namespace lbm
