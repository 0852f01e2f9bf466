// kernels.cu -- the per-body kernels of one coupled step and the field
// export / import kernels:
//   prep       per-body geometry records (remade only for states set from
//              outside), remap candidate lists for the batched remap; a
//              single lattice runs it only after the host wrote a state
//   remap      map the bodies onto the lattice (Sec. 2.3), epoch flags, the
//              boundary kernel's cell list
//   links      per-body list of fluid->solid links (ballot + block scan)
//   loads      drive terms (Eq. FB1-FB3) and spring forces (Eq. osci_i,
//              osci_j) of the step
//   force      momentum-exchange force and torque (Eq. hydroF): FP64 with a
//              fixed-order reduction for FP64 storage, exact integer and
//              fixed-point sums for 32/16-bit storage (deterministic both);
//              the last block of each body runs its rigid-body time step
//              (Algorithm 1) in FP64 on one warp
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

__device__ inline bool cell_inside(const Domain &d, const BodyProps &p, const BodyState &b, int x,
                                   int y, int z) {
    double o[3];
    offset_from(d, b, x, y, z, o);
    if (p.shape == 0) return o[0] * o[0] + o[1] * o[1] + o[2] * o[2] <= p.r * p.r;
    double R[3][3];
    quat_to_matrix(b.q, R);
    const double a0 = R[0][0], a1 = R[1][0], a2 = R[2][0];
    double s = o[0] * a0 + o[1] * a1 + o[2] * a2;
    const double h = 0.5 * p.l;
    s = s > h ? h : (s < -h ? -h : s);
    const double e0 = o[0] - s * a0, e1 = o[1] - s * a1, e2 = o[2] - s * a2;
    return e0 * e0 + e1 * e1 + e2 * e2 <= p.r * p.r;
}

// The inside test in FP32: the minimum-image offset as an integer difference
// of cells (wrapped by compares) minus the centre's offset within its cell,
// then the distance in FP32 from that small, nearly exact offset.  Its
// error in the squared distance stays below about 1e-5 max(r^2, 1) (offsets
// exact to an FP32 ulp of the few-cell offset, an axis rounded once, a few
// roundings of the sums), growing like 1.3e-7 l r for long thin capsules;
// outside the margin max(1e-3 max(r^2, 1), 2e-6 l max(r, 1)) of r^2 it
// returns 1 (inside) or 0 (outside), within it -1 and the FP64 test
// decides: the map is the FP64 map bit for bit.
__device__ inline int inside_screen(const Domain &d, const BodyGeom *__restrict__ g, int x, int y, int z) {
    const int n3[3] = {d.nx, d.ny, d.nz}, per[3] = {d.px, d.py, d.pz}, q3[3] = {x, y, z};
    float o[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        int io = q3[i] - g->ci[i];
        if (per[i]) io = 2 * io > n3[i] ? io - n3[i] : (2 * io < -n3[i] ? io + n3[i] : io);
        o[i] = (float)io - g->cf[i];
    }
    const float o0 = o[0], o1 = o[1], o2 = o[2];
    float d2;
    if (g->shape == 0) {
        d2 = o0 * o0 + o1 * o1 + o2 * o2;
    } else {
        const float h = g->h;
        float sp = o0 * g->ax[0] + o1 * g->ax[1] + o2 * g->ax[2];
        sp = sp > h ? h : (sp < -h ? -h : sp);
        const float e0 = o0 - sp * g->ax[0], e1 = o1 - sp * g->ax[1], e2 = o2 - sp * g->ax[2];
        d2 = e0 * e0 + e1 * e1 + e2 * e2;
    }
    const float r2 = g->r2, margin = g->margin;
    return d2 < r2 - margin ? 1 : (d2 > r2 + margin ? 0 : -1);
}

__device__ inline uint8_t wall_bit(const Domain &d, int x, int y, int z) {
    const bool w = (!d.px && (x == 0 || x == d.nx - 1)) || (!d.py && (y == 0 || y == d.ny - 1)) ||
                   (!d.pz && (z == 0 || z == d.nz - 1));
    return w ? F_WALL : 0;
}

__global__ void init_flags_kernel(const Domain d, uint8_t *f0, uint8_t *f1, uint8_t *b0, uint8_t *b1) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.C) return;
    const int x = (int)(c % d.nx);
    const int y = (int)((c / d.nx) % d.ny);
    const int z = (int)(c / ((long long)d.nx * d.ny));
    const uint8_t w = wall_bit(d, x, y, z);
    f0[c] = w;
    f1[c] = w;
    b0[c] = NO_BODY;
    b1[c] = NO_BODY;
}

// A cell farther than this from a body's bounding box [floor(X - reach),
// floor(X + reach)] can hold no flag of that body in epochs n-2 .. n: solid
// cells of epoch n-3 lie within 1.5 cells of the current extent, NEAR adds a
// neighbour's 1.42 cells, and the floor of the upper bound loses up to one.
constexpr int STATIC_REACH = 4;

// Axis a of a body's geometry record from that axis' centre coordinate,
// velocity, angular velocity and the body x axis' component.  Every FP64
// rounding is explicit, so a record made here and one made by the
// rigid-body step's warp agree bit for bit.
__device__ inline void geom_axis(const Domain &d, const BodyProps &p, int a, double Xa, double Va, double Wa,
                                 double axa, BodyGeom &g) {
    const int n = a == 0 ? d.nx : (a == 1 ? d.ny : d.nz);
    const int per = a == 0 ? d.px : (a == 1 ? d.py : d.pz);
    const double inv = a == 0 ? d.inx : (a == 1 ? d.iny : d.inz);
    const int half = p.E + REMAP_MARGIN;
    const double c = per ? __fma_rn(-(double)n, floor(__dmul_rn(Xa, inv)), Xa) : Xa;
    const double fc = floor(c);
    int o = (int)fc - half;
    if (per) o = ((o % n) + n) % n;
    g.origin[a] = o;
    g.ci[a] = (int)fc;
    g.cfd[a] = __dsub_rn(c, fc);
    g.cf[a] = (float)g.cfd[a];
    g.v[a] = (float)Va;
    g.w[a] = (float)Wa;
    g.ax[a] = (float)axa;
    int lo = (int)floor(__dsub_rn(Xa, p.reach)), hi = (int)floor(__dadd_rn(Xa, p.reach));
    int width = hi - lo + 1;
    int elo = lo - STATIC_REACH, ewidth = width + 2 * STATIC_REACH;
    if (per) {
        lo %= n;
        if (lo < 0) lo += n;
        if (width > n) width = n;
        elo %= n;
        if (elo < 0) elo += n;
        if (ewidth > n) ewidth = n;
    }
    g.box[a] = lo;
    g.box[3 + a] = width;
    g.ebox[a] = elo;
    g.ebox[3 + a] = ewidth;
}

__device__ inline void geom_scalars(const BodyProps &p, BodyGeom &g) {
    g.r2 = p.r2f;
    g.h = p.hf;
    g.margin = p.marginf;
    g.shape = p.shape;
    g.side = 2 * (p.E + REMAP_MARGIN) + 1;
}

// a body may not cross a wall: its extent along axis a (with the x axis'
// component axa of a capsule) beyond the wall planes
__device__ inline bool outside_walls(const Domain &d, const BodyProps &p, int a, double Xa, double axa) {
    const int per = a == 0 ? d.px : (a == 1 ? d.py : d.pz);
    if (per) return false;
    const int n = a == 0 ? d.nx : (a == 1 ? d.ny : d.nz);
    const double ext = p.r + (p.shape == 1 ? 0.5 * p.l * fabs(axa) : 0.0);
    return Xa - ext < -0.5 || Xa + ext > n - 0.5;
}

// the whole record of state s, one thread (prep_kernel's fallback)
__device__ void make_geom(const Domain &d, const BodyProps &p, const BodyState &s, BodyGeom &g, int *status) {
    const double w = s.q[0], qx = s.q[1], qy = s.q[2], qz = s.q[3];
    const double axv[3] = {__dsub_rn(1.0, __dmul_rn(2.0, __fma_rn(qy, qy, __dmul_rn(qz, qz)))),
                           __dmul_rn(2.0, __fma_rn(qx, qy, __dmul_rn(w, qz))),
                           __dmul_rn(2.0, __fma_rn(qx, qz, -__dmul_rn(w, qy)))};
    bool out = false;
    for (int a = 0; a < 3; ++a) {
        geom_axis(d, p, a, s.X[a], s.V[a], s.W[a], axv[a], g);
        out = out || outside_walls(d, p, a, s.X[a], axv[a]);
    }
    geom_scalars(p, g);
    if (out) atomicOr(status, ST_OUTSIDE);
}

__device__ inline bool same_state(const BodyState &a, const BodyState &b) {
    const long long *x = reinterpret_cast<const long long *>(&a), *y = reinterpret_cast<const long long *>(&b);
    bool eq = true;
#pragma unroll
    for (int i = 0; i < 13; ++i) eq = eq && x[i] == y[i];
    return eq;
}

// Drive terms (Eq. FB1-FB3) and spring forces (Eq. osci_i, osci_j) of step
// n into scratch: they depend on state n only.  Thread `rank` of `count`
// takes drive terms rank, rank + count, ... and springs likewise.
__device__ void body_loads(const Device &dv, const StepPtrs &sp, int drive_rank, int spring_rank, int count) {
    const double t = (double)*dv.t_dev;
    for (int k = drive_rank; k < dv.nd; k += count) {
        const DriveTerm dt = dv.drives[k];
        double f = 0.0;
        if (!(t < dt.t_on || t >= dt.t_off)) f = dt.amp * sin(dt.omega * t - dt.phase);
        double R[3][3];                                 // the drive acts along R(q) axis
        quat_to_matrix(sp.body_cur[dt.body].q, R);
        for (int i = 0; i < 3; ++i)
            dv.drive_f[3 * k + i] = f * (R[i][0] * dt.axis[0] + R[i][1] * dt.axis[1] + R[i][2] * dt.axis[2]);
    }
    for (int k = spring_rank; k < dv.ns; k += count) {
        const Spring sp_ = dv.springs[k];
        const BodyState si = sp.body_cur[sp_.i], sj = sp.body_cur[sp_.j];
        const double dd[3] = {si.X[0] - sj.X[0], si.X[1] - sj.X[1], si.X[2] - sj.X[2]};
        const double len = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        const double inv_len = len > 0 ? 1.0 / len : 0.0;
        for (int i = 0; i < 3; ++i)
            dv.spring_f[3 * k + i] = -sp_.k * (len - sp_.rest) * (dd[i] * inv_len) - sp_.gamma * (si.V[i] - sj.V[i]);
    }
}

// the drive and spring loads of step n, two warps on two SM sub-partitions
// (an FP64 warp instruction occupies its sub-partition's FP64 pipe for the
// same time however many lanes it carries)
__device__ __forceinline__ void loads_body(const Device &dv, const StepPtrs &sp) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) body_loads(dv, sp, lane, dv.ns, 32);
    else body_loads(dv, sp, dv.nd, lane, 32);
}

__global__ void __launch_bounds__(64) loads_kernel(const Device dv, const StepPtrs sp) { loads_body(dv, sp); }

__global__ void __launch_bounds__(64) loads_batch(const Batch bt) {
    LBM_BATCH_MEMBER(bt);
    loads_body(sdv, ssp);
}

// does the cell span [b0, b0 + bw) meet the span [e0, e0 + ew) on an axis of
// n cells?  (On a periodic axis b0 and e0 are wrapped into [0, n).)
__device__ inline bool spans_meet(int b0, int bw, int e0, int ew, int n, int periodic) {
    if (!periodic) return b0 < e0 + ew && e0 < b0 + bw;
    if (bw >= n || ew >= n) return true;
    int o = b0 - e0;                // the start of [b0, ..) seen from e0, in [0, n)
    if (o < 0) o += n;
    return o < ew || o + bw > n;
}

// Body preparation, one block: the geometry records of states n and n-1
// (slots by body buffer: remade only when the slot's stamp differs from the
// state, i.e. when no rigid-body step produced that state), each body's
// remap candidates for the batched remap (the bodies, in order, whose grown
// box meets its remap cube; a warp a body, ballots over the candidates; a
// single lattice's remap finds its own), and the start of the boundary
// kernel's list.  A single lattice's steps whose states the rigid-body step
// made (and whose list the previous step's last block emptied) skip it.
constexpr int PREP_THREADS = 256;

__device__ __forceinline__ void prep_body(const Device &dv, const StepPtrs &sp) {
    const Domain d = dv.dom;
    const int n3[3] = {d.nx, d.ny, d.nz}, per[3] = {d.px, d.py, d.pz};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BodyGeom *cur = dv.geom + sp.parity * dv.nb, *prev = dv.geom + (sp.parity ^ 1) * dv.nb;
    BodyState *scur = dv.gstamp + sp.parity * dv.nb, *sprev = dv.gstamp + (sp.parity ^ 1) * dv.nb;
    if (threadIdx.x == 0) *dv.bcount = 0;           // the remap refills the boundary kernel's list
    if (warp < 2) {
        BodyGeom *g = warp == 0 ? cur : prev;
        BodyState *st = warp == 0 ? scur : sprev;
        const BodyState *state = warp == 0 ? sp.body_cur : sp.body_prev;
        for (int k = lane; k < dv.nb; k += 32) {
            const BodyState sb = state[k];
            if (same_state(sb, st[k])) continue;
            make_geom(d, dv.props[k], sb, g[k], dv.status);
            st[k] = sb;
        }
    }
    __syncthreads();
    __shared__ int s_box[LBM_MAX_BODIES_DEV][8];        // ebox (6), then origin packed per axis below
    __shared__ int s_org[LBM_MAX_BODIES_DEV][4];
    for (int k = threadIdx.x; k < dv.nb; k += blockDim.x) {
        for (int i = 0; i < 6; ++i) s_box[k][i] = cur[k].ebox[i];
        for (int i = 0; i < 3; ++i) s_org[k][i] = cur[k].origin[i];
        s_org[k][3] = cur[k].side;
    }
    __syncthreads();
    for (int b = warp; b < dv.nb; b += PREP_THREADS / 32) {
        int cnt = 0;
        for (int k0 = 0; k0 < dv.nb; k0 += 32) {
            const int k = k0 + lane;
            bool meets = k < dv.nb;
            for (int a = 0; a < 3 && meets; ++a)
                meets = spans_meet(s_org[b][a], s_org[b][3], s_box[k][a], s_box[k][3 + a], n3[a], per[a]);
            const unsigned bal = __ballot_sync(0xffffffffu, meets);
            if (meets) dv.cand[b * dv.nb + cnt + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)k;
            cnt += __popc(bal);
        }
        if (lane == 0) cur[b].ncand = cnt;
    }
}

__global__ void __launch_bounds__(PREP_THREADS) prep_kernel(const Device dv, const StepPtrs sp) { prep_body(dv, sp); }

__global__ void __launch_bounds__(PREP_THREADS) prep_batch(const Batch bt) {
    LBM_BATCH_MEMBER(bt);
    prep_body(sdv, ssp);
}


// a coordinate of the cube, o + l with o in [0, n) and l < side, wrapped
// into [0, n) on a periodic axis (one compare unless the cube exceeds the axis)
__device__ inline int wrap_up(int v, int n) { return v < n ? v : (v - n < n ? v - n : v % n); }

// Remap: block row blockIdx.y = body b; the cube of side 2 (E_b +
// REMAP_MARGIN) + 1 around floor(X_b) at state n is taken as one run of
// side^3 cells in (z, y, x) order, REMAP_CELLS consecutive cells a block and
// REMAP_R a thread (i and i + REMAP_THREADS: their flag loads are issued
// together, so a block's latency chain covers both).  No thread idles on a
// cube narrower than a warp, and the grid of the 24-capsule swarm (side 23)
// fits in one wave of resident blocks.  Every covered cell gets its epoch-n
// flags from the geometry of all bodies and the epoch-(n-1) buffer;
// overlapping cubes write identical values.  A cell tests only body b's
// candidates, in body order (integer boxes, the FP32 screen, and the FP64
// inside test only within the screen's margin).  Fluid cells flagged F_NEAR
// or F_SOLID_PREV are appended to the boundary kernel's list.
constexpr int REMAP_THREADS = 256;
constexpr int REMAP_R = 2;
constexpr int REMAP_CELLS = REMAP_THREADS * REMAP_R;    // cube cells a block covers
constexpr int REMAP_STAGED = 8;
constexpr int REMAP_LIST_BUF = REMAP_CELLS;             // a block lists at most all of its cells

// blocks a body of remap-cube side `side` takes
inline int remap_blocks(int side) {
    const long long cells = (long long)side * side * side;
    return (int)((cells + REMAP_CELLS - 1) / REMAP_CELLS);
}
static_assert(sizeof(BodyGeom) % sizeof(int) == 0, "geometry records are copied as ints");

template <bool SELF_CAND>
__device__ __forceinline__ void remap_body(const Device &dv, const StepPtrs &sp, const Blk &bk, int init_mode) {
    const Domain d = dv.dom;
    const int b = bk.y;
    const BodyGeom *__restrict__ geo = dv.geom + sp.parity * dv.nb;    // state n
    // body b's candidates, the first REMAP_STAGED of them with their
    // records in shared memory
    __shared__ BodyGeom cg[REMAP_STAGED];
    __shared__ int cid[LBM_MAX_BODIES_DEV];
    __shared__ int s_ncand;
    const int n3[3] = {d.nx, d.ny, d.nz}, per[3] = {d.px, d.py, d.pz};
    const int side = geo[b].side;
    const int side2 = side * side, cells = side2 * side;
    const int i0 = bk.x * REMAP_CELLS;
    if (i0 >= cells) return;                  // the grid covers the largest body's cube
    // this block's share of the boundary kernel's list, gathered in shared
    // memory and appended with one atomic at the end
    __shared__ uint32_t lbuf[REMAP_LIST_BUF];
    __shared__ int lcount, lbase;
    const int org[3] = {geo[b].origin[0], geo[b].origin[1], geo[b].origin[2]};
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    if (tid == 0) lcount = 0;
    // the candidates: the bodies, in body order, whose grown box (the cells
    // their flags of epochs n-3 .. n can reach) meets b's cube.  A single
    // lattice's block finds them (the first warp, ballots over 32 bodies at
    // a time); the batched remap takes the preparation kernel's list.  The
    // first REMAP_STAGED records are staged in shared memory.
    if constexpr (SELF_CAND) {
        if (tid < 32) {
            int cnt = 0;
            for (int k0 = 0; k0 < dv.nb; k0 += 32) {
                const int k = k0 + tid;
                bool meets = k < dv.nb;
                for (int a = 0; a < 3 && meets; ++a)
                    meets = spans_meet(org[a], side, geo[k].ebox[a], geo[k].ebox[3 + a], n3[a], per[a]);
                const unsigned bal = __ballot_sync(0xffffffffu, meets);
                if (meets) cid[cnt + __popc(bal & ((1u << tid) - 1u))] = k;
                cnt += __popc(bal);
            }
            if (tid == 0) s_ncand = cnt;
        }
    } else {
        const int nc = geo[b].ncand;
        for (int i = tid; i < nc; i += REMAP_THREADS) cid[i] = dv.cand[b * dv.nb + i];
        if (tid == 0) s_ncand = nc;
    }
    __syncthreads();
    const int ncand = s_ncand;
    {
        constexpr int W = (int)(sizeof(BodyGeom) / sizeof(int));
        const int staged = min(ncand, REMAP_STAGED);
        for (int i = tid; i < staged * W; i += REMAP_THREADS)
            reinterpret_cast<int *>(cg)[i] = reinterpret_cast<const int *>(geo + cid[i / W])[i % W];
    }
    __syncthreads();

    // every lane runs each of its cells, so the ballots below see whole warps
        {
            int xr[REMAP_R], yr[REMAP_R], zr[REMAP_R], idr[REMAP_R];
            long long cr[REMAP_R];
            bool liver[REMAP_R];
#pragma unroll
            for (int r = 0; r < REMAP_R; ++r) {
                const int ci = i0 + r * REMAP_THREADS + tid;
                bool live = ci < cells;
                const int lz = ci / side2, rem = ci - lz * side2;
                const int ly = rem / side, lx = rem - ly * side;
                int x = org[0] + lx, y = org[1] + ly, z = org[2] + lz;
                if (d.px) x = wrap_up(x, d.nx); else live = live && x >= 0 && x < d.nx;
                if (d.py) y = wrap_up(y, d.ny); else live = live && y >= 0 && y < d.ny;
                if (d.pz) z = wrap_up(z, d.nz); else live = live && z >= 0 && z < d.nz;
                const int p3[3] = {x, y, z};
                int id = NO_BODY;
                bool reached = false;           // within STATIC_REACH cells of some body's box
                for (int i = 0; i < ncand && live; ++i) {
                    const int kb = cid[i];
                    const BodyGeom *g = i < REMAP_STAGED ? cg + i : geo + kb;
                    bool in = true;
                    for (int a = 0; a < 3 && in; ++a) {
                        int o = p3[a] - g->ebox[a];
                        if (per[a] && o < 0) o += n3[a];
                        in = o >= 0 && o < g->ebox[3 + a];
                    }
                    if (!in) continue;
                    reached = true;
                    for (int a = 0; a < 3 && in; ++a) {
                        int o = p3[a] - g->box[a];
                        if (per[a] && o < 0) o += n3[a];
                        in = o >= 0 && o < g->box[3 + a];
                    }
                    if (!in) continue;
                    // FP32 screen; cells within its margin of the surface take the FP64 test
                    const int screen = inside_screen(d, g, x, y, z);
                    if (screen == 0 || (screen < 0 && !cell_inside(d, dv.props[kb], sp.body_cur[kb], x, y, z)))
                        continue;
                    if (id != NO_BODY) atomicOr(dv.status, ST_OVERLAP);
                    id = kb;
                }
                // farther than STATIC_REACH from every body's box: the cell holds
                // its static flags in both epoch buffers already (nothing within
                // reach was solid in the last three steps, at most 0.5 cells of
                // motion per step)
                xr[r] = x;
                yr[r] = y;
                zr[r] = z;
                idr[r] = id;
                cr[r] = ((long long)z * d.ny + y) * d.nx + x;
                liver[r] = live && reached;
            }
            // the epoch-(n-1) flags and body id of every row's cell and whether
            // any pull source x - e_a held an obstacle of step n-1 (sources
            // beyond a wall do not count): all loads before any use
            uint8_t prevr[REMAP_R], nearr[REMAP_R], bidr[REMAP_R];
#pragma unroll
            for (int r = 0; r < REMAP_R; ++r) {
                prevr[r] = 0;
                nearr[r] = 0;
                bidr[r] = NO_BODY;
                if (!liver[r] || init_mode) continue;
                const long long c = cr[r];
                const int x = xr[r], y = yr[r], z = zr[r];
                prevr[r] = sp.flags_prev[c];
                bidr[r] = sp.bid_prev[c];
                uint8_t near = 0;
                const long long sy = d.nx, sz = (long long)d.nx * d.ny;
                if (x > 0 && x < d.nx - 1 && y > 0 && y < d.ny - 1 && z > 0 && z < d.nz - 1) {
#pragma unroll
                    for (int a = 1; a < Q; ++a) near |= sp.flags_prev[c - ex(a) - ey(a) * sy - ez(a) * sz];
                } else {
#pragma unroll
                    for (int a = 1; a < Q; ++a) {
                        const int sx_ = x - ex(a), sy_ = y - ey(a), sz_ = z - ez(a);
                        const bool in = !((!d.px && (sx_ < 0 || sx_ >= d.nx)) || (!d.py && (sy_ < 0 || sy_ >= d.ny)) ||
                                          (!d.pz && (sz_ < 0 || sz_ >= d.nz)));
                        const uint8_t v = sp.flags_prev[((long long)wrap_axis(sz_, d.nz) * d.ny + wrap_axis(sy_, d.ny)) * d.nx +
                                                        wrap_axis(sx_, d.nx)];
                        near |= in ? v : 0;
                    }
                }
                nearr[r] = near;
            }
#pragma unroll
            for (int r = 0; r < REMAP_R; ++r) {
                const bool live = liver[r];
                const int id = idr[r];
                const long long c = cr[r];
                uint8_t flags = 0;
                if (live) {
                    const uint8_t solid = id != NO_BODY ? F_SOLID : 0;
                    flags = solid | wall_bit(d, xr[r], yr[r], zr[r]);
                    if (!init_mode) {
                        const uint8_t prev = prevr[r] & F_SOLID;
                        if (prev) flags |= F_SOLID_PREV;
                        if (nearr[r] & F_SOLID) flags |= F_NEAR;
                        if ((solid != 0) != (prev != 0) || (solid && bidr[r] != id)) dv.changed[sp.parity] = 1;
                    }
                    sp.flags_cur[c] = flags;
                    sp.bid_cur[c] = (uint8_t)id;
                }
                // the boundary kernel's cells: a shared-memory atomic per warp
                // (past the buffer, a global one)
                const bool mine = live && !init_mode && !(flags & F_SOLID) && (flags & (F_NEAR | F_SOLID_PREV));
                const unsigned mb = __ballot_sync(0xffffffffu, mine);
                if (mb) {
                    const int leader = __ffs(mb) - 1;
                    int base = 0;
                    if (lane == leader) base = atomicAdd(&lcount, __popc(mb));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    const int pos = base + __popc(mb & ((1u << lane) - 1u));
                    if (mine) {
                        if (pos < REMAP_LIST_BUF) {
                            lbuf[pos] = (uint32_t)c;
                        } else {
                            const int g = atomicAdd(dv.bcount, 1);
                            if (g < dv.blist_cap) dv.blist[g] = (uint32_t)c;
                            else atomicOr(dv.status, ST_LINKS);
                        }
                    }
                }
            }
        }
    __syncthreads();
    if (tid == 0) lbase = lcount ? atomicAdd(dv.bcount, min(lcount, REMAP_LIST_BUF)) : 0;
    __syncthreads();
    const int nl = min(lcount, REMAP_LIST_BUF);
    for (int i = tid; i < nl; i += REMAP_THREADS) {
        if (lbase + i < dv.blist_cap) dv.blist[lbase + i] = lbuf[i];
        else atomicOr(dv.status, ST_LINKS);
    }
}

__global__ void __launch_bounds__(REMAP_THREADS, 4) remap_kernel(const Device dv, const StepPtrs sp, int init_mode) {
    pdl_enter();
    remap_body<true>(dv, sp, launch_blk(), init_mode);
}

__global__ void __launch_bounds__(REMAP_THREADS, 4) remap_batch(const Batch bt) {
    LBM_BATCH_MEMBER(bt);
    remap_body<false>(sdv, ssp, sbk, 0);
}

// Links: block (k, b) scans z-plane k of the cube of side 2 E_b + 3 around
// floor(X_b) and stores the links (x_f, a) with x_f fluid and x_f + e_a a
// cell of body b, in (y, x, a) order, into segment (b, k).  Runs only when
// the remap changed a flag; otherwise the previous lists stand.
__device__ __forceinline__ void links_body(const Device &dv, const StepPtrs &sp, const Blk &bk) {
    if (dv.changed[sp.parity] == 0) return;
    const Domain d = dv.dom;
    const int b = bk.y, k = bk.x;
    const BodyProps pb = dv.props[b];
    const int half = pb.E + 1;
    const int side = 2 * half + 1;
    int *count = dv.seg_count + (long long)b * dv.link_side + k;
    if (k >= side) {
        if (threadIdx.x == 0) *count = 0;
        return;
    }
    const BodyState sb = sp.body_cur[b];
    Link *seg = dv.links + ((long long)b * dv.link_side + k) * dv.seg_cap;
    const int ox = (int)floor(sb.X[0]) - half, oy = (int)floor(sb.X[1]) - half;
    int z = (int)floor(sb.X[2]) - half + k;
    bool zok = true;
    if (d.pz) z = ((z % d.nz) + d.nz) % d.nz; else zok = z >= 0 && z < d.nz;

    __shared__ int warp_tot[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int area = side * side;
    for (int start = 0; start < area; start += blockDim.x) {
        const int l = start + threadIdx.x;
        unsigned mask = 0;
        long long c = 0;
        if (zok && l < area) {
            int x = ox + l % side, y = oy + l / side;
            bool ok = true;
            if (d.px) x = ((x % d.nx) + d.nx) % d.nx; else ok = ok && x >= 0 && x < d.nx;
            if (d.py) y = ((y % d.ny) + d.ny) % d.ny; else ok = ok && y >= 0 && y < d.ny;
            if (ok) {
                c = ((long long)z * d.ny + y) * d.nx + x;
                if (!(sp.flags_cur[c] & F_SOLID)) {
                    for (int a = 1; a < Q; ++a) {
                        int nx_ = x + ex(a), ny_ = y + ey(a), nz_ = z + ez(a);
                        if ((!d.px && (nx_ < 0 || nx_ >= d.nx)) || (!d.py && (ny_ < 0 || ny_ >= d.ny)) ||
                            (!d.pz && (nz_ < 0 || nz_ >= d.nz)))
                            continue;
                        nx_ = wrap_axis(nx_, d.nx); ny_ = wrap_axis(ny_, d.ny); nz_ = wrap_axis(nz_, d.nz);
                        const long long n = ((long long)nz_ * d.ny + ny_) * d.nx + nx_;
                        if ((sp.flags_cur[n] & F_SOLID) && sp.bid_cur[n] == b) mask |= 1u << a;
                    }
                }
            }
        }
        // block-wide exclusive scan of the per-thread link counts
        const int cnt = __popc(mask);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < nwarps; ++w) {
            if (w < warp) before += warp_tot[w];
            total += warp_tot[w];
        }
        int pos = base + before + incl - cnt;
        while (mask) {
            const int a = __ffs(mask) - 1;
            mask &= mask - 1;
            if (pos < dv.seg_cap) seg[pos] = Link{(uint32_t)c, (uint32_t)a};
            else atomicOr(dv.status, ST_LINKS);
            ++pos;
        }
        __syncthreads();
        if (threadIdx.x == 0) base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

__global__ void __launch_bounds__(256) links_kernel(const Device dv, const StepPtrs sp) { links_body(dv, sp, launch_blk()); }

__global__ void __launch_bounds__(256) links_batch(const Batch bt) {
    LBM_BATCH_MEMBER(bt);
    links_body(sdv, ssp, sbk);
}

// a stored deviation in FP32 (exact for FP32, FP16 times its power-of-two
// scale, BF16), without a trip through FP64
template <typename T> __device__ inline float load_dev_f(const T *p, float inv_scale);
template <> __device__ inline float load_dev_f<float>(const float *p, float) { return *p; }
template <> __device__ inline float load_dev_f<__half>(const __half *p, float s) { return __half2float(*p) * s; }
template <> __device__ inline float load_dev_f<__nv_bfloat16>(const __nv_bfloat16 *p, float) {
    return __bfloat162float(*p);
}

template <typename T> __device__ inline double load_dev(const T *p, float inv_scale);
template <> __device__ inline double load_dev<double>(const double *p, float) { return *p; }
template <> __device__ inline double load_dev<float>(const float *p, float) { return (double)*p; }
template <> __device__ inline double load_dev<__half>(const __half *p, float s) {
    return (double)(__half2float(*p) * s);
}
template <> __device__ inline double load_dev<__nv_bfloat16>(const __nv_bfloat16 *p, float) {
    return (double)__bfloat162float(*p);
}

constexpr int FORCE_THREADS = 256;
constexpr int MAX_SEGMENTS = 1024;

// minimum image of a cell difference o (|o| < n + 1) by integer compares
__device__ inline int near_cell_k(int o, int n, int periodic) {
    if (!periodic) return o;
    return 2 * o > n ? o - n : (2 * o < -n ? o + n : o);
}

// periodic minimum image of d for |d| < 3n/2 (two compares, no FP64 floor)
__device__ inline double wrap_near(double d, int n, int periodic) {
    if (!periodic) return d;
    const double h = 0.5 * n;
    return d > h ? d - n : (d < -h ? d + n : d);
}

// Rigid-body step (Algorithm 1, Eq. totalFSwimmer) of body b by one warp
// (all 32 lanes call it).  An FP64 warp instruction costs the same however
// many lanes it carries, so lanes hold components: six load components,
// three axes, nine rotation-matrix entries, four quaternion components.
// Per axis it adds, in order, the momentum-exchange sum, g times the
// volume, the body's drive terms in term order and its springs in spring
// order (body_loads' scratch), then advances by semi-implicit Euler
// (dt = 1) in FP64.  It also writes the geometry record of the new state
// into that state's slot, with its stamp, and checks the new state (walls,
// finite, at most MAX_STEP per step).
__device__ void integrate_body_warp(const Device &dv, const StepPtrs &sp, int b, int with_fluid) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long tstep = *dv.t_dev;
    const BodyProps *pb = dv.props + b;
    const double *st = reinterpret_cast<const double *>(sp.body_cur + b);       // X q V W
    const int ax = lane < 3 ? lane : 0;

    // external force on axis ax: g times the volume, then the body's drive
    // terms in term order and its springs in spring order (loaded first, so
    // that their chains of dependent loads overlap the ones below)
    double Fext = dv.g[ax] * pb->volume;
    if (lane < 3) {
        for (int k = pb->drive_first; k < pb->drive_first + pb->drive_count; ++k) Fext += dv.drive_f[3 * k + ax];
        for (int kk = pb->spring_first; kk < pb->spring_first + pb->spring_count; ++kk) {
            const int k = dv.spring_list[kk];
            const double f = dv.spring_f[3 * k + ax];
            Fext += dv.springs[k].i == b ? f : -f;
        }
    }

    // hydrodynamic load of step n, lane i < 6 component i
    double hyd = 0.0;
    if (with_fluid && dv.precision == 0) {
        if (lane < 6)
            for (int k = 0; k < FORCE_BLOCKS; ++k) hyd += __ldcg(dv.fpart + ((long long)b * FORCE_BLOCKS + k) * 6 + lane);
    } else if (with_fluid) {
        // F = S1 / 36 + Fv, T = (S2 - c x S1) / 36 + Tv - c x Fv with c the
        // centre's position within its cell (the force kernel's terms)
        double fv = 0.0;
        int si = 0;
        if (lane < 6) {
            fv = (double)__ldcg(dv.fx + b * 6 + lane) * (1.0 / (double)(1LL << FIX_BITS));
            si = __ldcg(dv.fi + b * 6 + lane);
            dv.fx[b * 6 + lane] = 0;
            dv.fi[b * 6 + lane] = 0;
        }
        const int i = lane % 3, j = (i + 1) % 3, k = (i + 2) % 3;
        const double s1j = (double)__shfl_sync(FULL, si, j), s1k = (double)__shfl_sync(FULL, si, k);
        const double fvj = __shfl_sync(FULL, fv, j), fvk = __shfl_sync(FULL, fv, k);
        const double *c = dv.geom[sp.parity * dv.nb + b].cfd;
        if (lane < 3) hyd = (double)si * (1.0 / 36.0) + fv;
        else if (lane < 6)
            hyd = ((double)si - (c[j] * s1k - c[k] * s1j)) * (1.0 / 36.0) + fv - (c[j] * fvk - c[k] * fvj);
    }
    double v = hyd;
    if (lane < 6) {
        const double prev = dv.fh[b * 6 + lane];
        dv.fh[b * 6 + lane] = hyd;
        if (dv.avg_force && tstep > 0) v = 0.5 * (hyd + prev);
    }

    // translation, lanes 0..2
    const double F = v + Fext;
    const double Vn = st[7 + ax] + F * pb->inv_m;
    const double Xn = st[ax] + Vn;

    // R(q) of state n, entry (r, c) on lane 3 r + c < 9: 1 - 2 (a^2 + b^2)
    // on the diagonal, 2 (p q +- w u) off it
    const double qw = st[3], qv[3] = {st[4], st[5], st[6]};
    double Rrc;
    {
        const int r = lane < 9 ? lane / 3 : 0, cc = lane < 9 ? lane % 3 : 0;
        double A, Bq, Cq, D, base;
        if (r == cc) {
            A = -qv[(r + 1) % 3]; Bq = qv[(r + 1) % 3];
            Cq = -qv[(r + 2) % 3]; D = qv[(r + 2) % 3];
            base = 1.0;
        } else {
            const bool plus = (r == 1 && cc == 0) || (r == 0 && cc == 2) || (r == 2 && cc == 1);
            A = qv[min(r, cc)]; Bq = qv[max(r, cc)];
            Cq = plus ? qw : -qw; D = qv[3 - r - cc];
            base = 0.0;
        }
        Rrc = base + 2.0 * (A * Bq + Cq * D);
    }
    // Omega += R diag(1/I) R^T T, lanes 0..2
    const double T0 = __shfl_sync(FULL, v, 3), T1 = __shfl_sync(FULL, v, 4), T2 = __shfl_sync(FULL, v, 5);
    const double R0i = __shfl_sync(FULL, Rrc, ax), R1i = __shfl_sync(FULL, Rrc, 3 + ax),
                 R2i = __shfl_sync(FULL, Rrc, 6 + ax);
    const double Tb = (R0i * T0 + R1i * T1 + R2i * T2) * pb->inv_inertia[ax];
    const double Tb0 = __shfl_sync(FULL, Tb, 0), Tb1 = __shfl_sync(FULL, Tb, 1), Tb2 = __shfl_sync(FULL, Tb, 2);
    const double Ri0 = __shfl_sync(FULL, Rrc, 3 * ax), Ri1 = __shfl_sync(FULL, Rrc, 3 * ax + 1),
                 Ri2 = __shfl_sync(FULL, Rrc, 3 * ax + 2);
    const double Wn = st[10 + ax] + (Ri0 * Tb0 + Ri1 * Tb1 + Ri2 * Tb2);

    // q += 1/2 (0, Omega) (x) q, renormalised; lane 0 the scalar part,
    // lane 1 + i the vector component i
    const double W0 = __shfl_sync(FULL, Wn, 0), W1 = __shfl_sync(FULL, Wn, 1), W2 = __shfl_sync(FULL, Wn, 2);
    const double Wv[3] = {W0, W1, W2};
    double q4;
    {
        // lane 0: w - 1/2 (W . v); lane 1 + i: v_i + 1/2 (w W_i + (W x v)_i),
        // one expression with the operands chosen per lane (no divergence)
        const int i = lane >= 1 && lane <= 3 ? lane - 1 : 0, i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        const bool s0 = lane == 0;
        const double base = s0 ? qw : qv[i];
        const double p1 = s0 ? -W0 : qw, r1 = s0 ? qv[0] : Wv[i];
        const double p2 = s0 ? -W1 : Wv[i1], r2 = s0 ? qv[1] : qv[i2];
        const double p3 = s0 ? -W2 : -Wv[i2], r3 = s0 ? qv[2] : qv[i1];
        q4 = base + 0.5 * (p1 * r1 + p2 * r2 + p3 * r3);
    }
    double sq = lane < 4 ? q4 * q4 : 0.0;
    sq += __shfl_xor_sync(FULL, sq, 1);
    sq += __shfl_xor_sync(FULL, sq, 2);
    const double qn = q4 * rsqrt(sq);

    // checks of state n+1
    const bool finite = lane >= 3 || (isfinite(Xn) && isfinite(Vn) && isfinite(Wn));
    const bool all_finite = __all_sync(FULL, finite);
    const bool fast = __any_sync(FULL, lane < 3 && fabs(Vn) > MAX_STEP);

    // the new state, its tape and history entries
    auto put = [&](double *o) {
        if (lane < 3) {
            o[lane] = Xn;
            o[7 + lane] = Vn;
            o[10 + lane] = Wn;
        }
        if (lane < 4) o[3 + lane] = qn;
    };
    put(reinterpret_cast<double *>(sp.body_next + b));
    if (dv.tape) {
        const TapeCtl tc = *dv.tape;
        const long long j = tstep - tc.t0;
        if (tc.on && j >= 0 && j < tc.cap) {
            put(tc.state + ((j + 2) * dv.nb + b) * 13);
            if (lane < 6) tc.force[(j * dv.nb + b) * 6 + lane] = hyd;
        }
    }
    if (dv.hist) put(dv.hist + ((tstep % dv.hist_cap) * dv.nb + b) * 13);

    // the geometry record of state n+1 (its slot is the body buffer it was
    // written to), lanes 0..2 an axis each; the body x axis is column 0 of R(q_{n+1})
    const int slot = sp.parity ^ 1;
    const double nw = __shfl_sync(FULL, qn, 0), nq[3] = {__shfl_sync(FULL, qn, 1), __shfl_sync(FULL, qn, 2),
                                                         __shfl_sync(FULL, qn, 3)};
    // column 0 of R: 1 - 2 (y^2 + z^2), 2 (x y + w z), 2 (x z - w y), one
    // expression base + 2 (A B + C D) with the operands chosen per lane
    double axa;
    {
        const double A = ax == 0 ? -nq[1] : nq[0], B = ax == 0 ? nq[1] : (ax == 1 ? nq[1] : nq[2]);
        const double Cq = ax == 0 ? -nq[2] : (ax == 1 ? nw : -nw), D = ax == 0 ? nq[2] : (ax == 1 ? nq[2] : nq[1]);
        axa = (ax == 0 ? 1.0 : 0.0) + 2.0 * (A * B + Cq * D);
    }
    BodyGeom *g = dv.geom + slot * dv.nb + b;
    const bool out = lane < 3 && outside_walls(dv.dom, *pb, ax, Xn, axa);
    if (lane < 3) geom_axis(dv.dom, *pb, ax, Xn, Vn, Wn, axa, *g);
    if (lane == 0) geom_scalars(*pb, *g);
    put(reinterpret_cast<double *>(dv.gstamp + slot * dv.nb + b));
    const bool any_out = __any_sync(FULL, out);
    if (lane == 0) {
        if (!all_finite) atomicOr(dv.status, ST_NAN);
        else if (fast) atomicOr(dv.status, ST_UNSTABLE);
        if (any_out) atomicOr(dv.status, ST_OUTSIDE);
    }
}

// after every body's step: the clock advances and the next epoch's change
// flag starts clear
__device__ inline void finish_step(const Device &dv, const StepPtrs &sp) {
    *dv.t_dev = *dv.t_dev + 1;
    dv.changed[sp.parity ^ 1] = 0;
    if (dv.bcount) *dv.bcount = 0;          // the next remap refills the boundary kernel's list
}

// round(v 2^FIX_BITS) to the nearest integer, ties away from zero, from the
// bits of v in integer operations (a 64-bit conversion would take the slow
// FP64 pipe); |v| < 2^(62 - FIX_BITS) is the caller's to ensure
__device__ inline long long to_fixed(float v) {
    const unsigned u = __float_as_uint(v);
    const int e = (int)((u >> 23) & 0xffu);
    if (e == 0 || e == 0xff) return 0;
    const long long m = (long long)((u & 0x7fffffu) | 0x800000u);     // v = m 2^(e - 150)
    const int sh = e - 150 + FIX_BITS;
    long long r;
    if (sh >= 0) r = m << sh;
    else if (sh > -25) r = (m + (1LL << (-sh - 1))) >> (-sh);
    else r = 0;
    return (u >> 31) ? -r : r;
}

// Momentum exchange (Eq. hydroF): blocks (k, b), k < FORCE_BLOCKS, split the
// links of body b into contiguous chunks and sum
//   F = sum e_a [2 f~_a(x_f) + 6 w_a rho(x_f) e_-a . u_w(x_f + e_a)],
//   T = sum (x_f + e_a / 2 - X) x F_link
// with f~ of step n (dst) and the body state of step n.  The last of body
// b's blocks to finish runs body b's rigid-body step on its first warp; the
// last body to finish ends the step (clock, change flag).
//
// FP64 storage: every term in FP64; each block reduces with warp shuffles
// in a fixed order and writes its partial sums, which the rigid-body step
// adds in block order (deterministic).
//
// 32/16-bit storage: f~_a = w_a + delta_a splits each link term into a
// constant part 2 w_a e_a and a small variable part v e_a with
// v = 2 delta_a + 6 w_a rho e_-a . u_w.  With the fluid cell at integer
// offset i from the centre's cell and c the centre's position within it
// (x_f - X = i - c), the sums are
//   F = S1 / 36 + Fv,  T = (S2 - c x S1) / 36 + Tv - c x Fv,
//   S1 = sum 72 w_a e_a,  S2 = sum i x 72 w_a e_a   (exact integers),
//   Fv = sum v e_a,  Tv = sum v (i x e_a)           (FP32 terms, each rounded
// to 2^-FIX_BITS and added as 64-bit integers),
// since e_a x e_a = 0.  The large, cancelling constant part never meets a
// rounding, the variable part is ~1e-3 of a term, and integer sums make
// the result independent of the order of the blocks' atomic additions.
template <typename T>
__device__ __forceinline__ void force_body(const Device &dv, const StepPtrs &sp, const Blk &bk) {
    const Domain d = dv.dom;
    const int b = bk.y, kb = bk.x;
    const BodyProps pb = dv.props[b];
    const int side = 2 * (pb.E + 1) + 1;
    const int *counts = dv.seg_count + (long long)b * dv.link_side;
    const Link *links = dv.links + (long long)b * dv.link_side * dv.seg_cap;
    const T *pop = static_cast<const T *>(sp.dst);
    const long long C = d.C;
    const float s = dv.f16_inv_scale;

    // exclusive prefix of the segment counts: thread t holds segments
    // [t per, (t+1) per), per <= 4 (side <= MAX_SEGMENTS), block scan
    __shared__ int prefix[MAX_SEGMENTS + 1];
    __shared__ int seg_warp[FORCE_THREADS / 32];
    {
        const int per = (side + FORCE_THREADS - 1) / FORCE_THREADS;
        const int k0 = threadIdx.x * per;
        int loc[MAX_SEGMENTS / FORCE_THREADS], sum = 0;
#pragma unroll
        for (int i = 0; i < MAX_SEGMENTS / FORCE_THREADS; ++i) {
            const int k = k0 + i;
            loc[i] = (i < per && k < side) ? counts[k] : 0;
            sum += loc[i];
        }
        const int ln = threadIdx.x & 31, wp = threadIdx.x >> 5;
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (ln >= o) incl += v;
        }
        if (ln == 31) seg_warp[wp] = incl;
        __syncthreads();
        int acc = incl - sum;
        for (int w = 0; w < wp; ++w) acc += seg_warp[w];
#pragma unroll
        for (int i = 0; i < MAX_SEGMENTS / FORCE_THREADS; ++i) {
            const int k = k0 + i;
            if (i < per && k < side) prefix[k] = acc;
            acc += loc[i];
        }
        if (threadIdx.x == FORCE_THREADS - 1) prefix[side] = acc;
    }
    __syncthreads();
    const int total = prefix[side];
    const int chunk = (total + FORCE_BLOCKS - 1) / FORCE_BLOCKS;
    const int j0 = kb * chunk, j1 = min(total, j0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    if constexpr (sizeof(T) == 8) {
        const BodyState sb = sp.body_cur[b];
        // body centre wrapped into the domain (once per block)
        const double xw[3] = {d.px ? sb.X[0] - d.nx * floor(sb.X[0] * d.inx) : sb.X[0],
                              d.py ? sb.X[1] - d.ny * floor(sb.X[1] * d.iny) : sb.X[1],
                              d.pz ? sb.X[2] - d.nz * floor(sb.X[2] * d.inz) : sb.X[2]};
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int j = j0 + threadIdx.x; j < j1; j += FORCE_THREADS) {
            int lo = 0, hi = side - 1;       // segment k with prefix[k] <= j < prefix[k+1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (prefix[mid] <= j) lo = mid; else hi = mid - 1;
            }
            const Link lk = links[(long long)lo * dv.seg_cap + (j - prefix[lo])];
            const long long c = lk.cell;
            const int a = (int)lk.dir;
            // cells are 32-bit indices (C < 2^31): 32-bit division
            const unsigned cu = lk.cell, nxu = (unsigned)d.nx, nyu = (unsigned)d.ny;
            const int x = (int)(cu % nxu), y = (int)((cu / nxu) % nyu), z = (int)(cu / (nxu * nyu));
            double rho = 1.0;
            for (int q = 0; q < Q; ++q) rho += load_dev<T>(pop + q * C + c, s);
            const double g_a = wgt(a) + load_dev<T>(pop + a * C + c, s);
            // offsets of the fluid cell, of the link end and of the link midpoint
            const double o0 = wrap_near(x - xw[0], d.nx, d.px);
            const double o1 = wrap_near(y - xw[1], d.ny, d.py);
            const double o2 = wrap_near(z - xw[2], d.nz, d.pz);
            const double e0 = o0 + ex(a), e1 = o1 + ey(a), e2 = o2 + ez(a);
            const double u0 = sb.V[0] + (sb.W[1] * e2 - sb.W[2] * e1);
            const double u1 = sb.V[1] + (sb.W[2] * e0 - sb.W[0] * e2);
            const double u2 = sb.V[2] + (sb.W[0] * e1 - sb.W[1] * e0);
            const double eu = -(ex(a) * u0 + ey(a) * u1 + ez(a) * u2);   // e_-a . u_w
            const double mag = 2.0 * g_a + 6.0 * wgt(a) * rho * eu;
            const double fl[3] = {ex(a) * mag, ey(a) * mag, ez(a) * mag};
            const double m0 = o0 + 0.5 * ex(a), m1 = o1 + 0.5 * ey(a), m2 = o2 + 0.5 * ez(a);
            acc[0] += fl[0]; acc[1] += fl[1]; acc[2] += fl[2];
            acc[3] += m1 * fl[2] - m2 * fl[1];
            acc[4] += m2 * fl[0] - m0 * fl[2];
            acc[5] += m0 * fl[1] - m1 * fl[0];
        }
        __shared__ double part[FORCE_THREADS / 32][6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double v = acc[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) part[warp][i] = v;
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                double v = lane < FORCE_THREADS / 32 ? part[lane][i] : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) dv.fpart[((long long)b * FORCE_BLOCKS + kb) * 6 + i] = v;
            }
        }
    } else {
        const BodyGeom *g = dv.geom + sp.parity * dv.nb + b;       // state n
        const int ci[3] = {g->ci[0], g->ci[1], g->ci[2]};
        const float cf[3] = {g->cf[0], g->cf[1], g->cf[2]};
        const float vf[3] = {g->v[0], g->v[1], g->v[2]}, wf[3] = {g->w[0], g->w[1], g->w[2]};
        long long accx[6] = {0, 0, 0, 0, 0, 0};
        int acci[6] = {0, 0, 0, 0, 0, 0};
        int bad = 0;
        for (int j = j0 + threadIdx.x; j < j1; j += FORCE_THREADS) {
            int lo = 0, hi = side - 1;       // segment k with prefix[k] <= j < prefix[k+1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (prefix[mid] <= j) lo = mid; else hi = mid - 1;
            }
            const Link lk = links[(long long)lo * dv.seg_cap + (j - prefix[lo])];
            const long long c = lk.cell;
            const int a = (int)lk.dir;
            const unsigned cu = lk.cell, nxu = (unsigned)d.nx, nyu = (unsigned)d.ny;
            const int x = (int)(cu % nxu), y = (int)((cu / nxu) % nyu), z = (int)(cu / (nxu * nyu));
            // rho - 1 of the fluid cell: the boundary kernel's record when it
            // collided the cell (nearly every link cell: bodies move far
            // less than a cell a step), else the FP32 sum of the stored
            // deviations (the bulk kernel's cells a body has just reached)
            float drho;
            const uint8_t fc = sp.flags_cur[c];
            if (fc != 0 && !(fc & F_SOLID)) {
                drho = __ldcg(dv.rho_near + c);
            } else {
                drho = 0.0f;
                for (int q = 0; q < Q; ++q) drho += load_dev_f<T>(pop + q * C + c, s);
            }
            const float rho = 1.0f + drho;
            const float da = load_dev_f<T>(pop + a * C + c, s);
            const int i0 = near_cell_k(x - ci[0], d.nx, d.px);
            const int i1 = near_cell_k(y - ci[1], d.ny, d.py);
            const int i2 = near_cell_k(z - ci[2], d.nz, d.pz);
            // u_w at the link end x_f + e_a
            const float e0 = ((float)i0 - cf[0]) + ex(a), e1 = ((float)i1 - cf[1]) + ey(a),
                        e2 = ((float)i2 - cf[2]) + ez(a);
            const float u0 = vf[0] + (wf[1] * e2 - wf[2] * e1);
            const float u1 = vf[1] + (wf[2] * e0 - wf[0] * e2);
            const float u2 = vf[2] + (wf[0] * e1 - wf[1] * e0);
            const float eu = -(ex(a) * u0 + ey(a) * u1 + ez(a) * u2);
            const float w6 = a < 7 ? 1.0f / 3.0f : 1.0f / 6.0f;    // 6 w_a (a > 0)
            const float v = 2.0f * da + w6 * rho * eu;
            // |delta| >= 2 is no fluid state; the bound keeps every sum in range
            if (!(fabsf(v) < 4.0f)) bad |= v != v ? ST_NAN : ST_UNSTABLE;
            const long long vx = to_fixed(v);
            accx[0] += ex(a) * vx;
            accx[1] += ey(a) * vx;
            accx[2] += ez(a) * vx;
            const int c0 = i1 * ez(a) - i2 * ey(a), c1 = i2 * ex(a) - i0 * ez(a), c2 = i0 * ey(a) - i1 * ex(a);
            accx[3] += to_fixed((float)c0 * v);
            accx[4] += to_fixed((float)c1 * v);
            accx[5] += to_fixed((float)c2 * v);
            const int K = a < 7 ? 4 : 2;          // 72 w_a
            acci[0] += K * ex(a);
            acci[1] += K * ey(a);
            acci[2] += K * ez(a);
            acci[3] += K * c0;
            acci[4] += K * c1;
            acci[5] += K * c2;
        }
        if (bad) atomicOr(dv.status, bad);
        __shared__ long long px_[FORCE_THREADS / 32][6];
        __shared__ int pi_[FORCE_THREADS / 32][6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            long long v = accx[i];
            int w = acci[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_down_sync(0xffffffffu, v, o);
                w += __shfl_down_sync(0xffffffffu, w, o);
            }
            if (lane == 0) {
                px_[warp][i] = v;
                pi_[warp][i] = w;
            }
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            const int i = threadIdx.x;
            long long v = 0;
            int w = 0;
            for (int k = 0; k < FORCE_THREADS / 32; ++k) {
                v += px_[k][i];
                w += pi_[k][i];
            }
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(dv.fx + b * 6 + i), (unsigned long long)v);
            if (w) atomicAdd(dv.fi + b * 6 + i, w);
            __threadfence();            // before the block counts itself done
        }
    }
    // the last of body b's blocks integrates body b with its first warp
    // (the drive and spring loads were evaluated beside the bulk kernel);
    // the last body ends the step
    __shared__ int last_of_body;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_of_body = atomicAdd(dv.body_done + b, 1u) == (unsigned)bk.gx - 1;
    }
    __syncthreads();
    if (!last_of_body || threadIdx.x >= 32) return;
    __threadfence();
    integrate_body_warp(dv, sp, b, 1);
    __syncwarp();
    if (threadIdx.x != 0) return;
    dv.body_done[b] = 0u;
    __threadfence();
    if (atomicAdd(dv.blocks_done, 1u) != (unsigned)bk.gy - 1) return;
    __threadfence();
    *dv.blocks_done = 0u;
    finish_step(dv, sp);
}

template <typename T>
__global__ void __launch_bounds__(FORCE_THREADS) force_kernel(const Device dv, const StepPtrs sp) {
    pdl_enter();
    force_body<T>(dv, sp, launch_blk());
}

template <typename T>
__global__ void __launch_bounds__(FORCE_THREADS) force_batch(const Batch bt) {
    LBM_BATCH_MEMBER(bt);
    force_body<T>(sdv, ssp, sbk);
}

// the end of a step of a lattice without bodies: the step counter advances
// (BF16 storage draws its rounding bits from it) and the next epoch's change
// flag starts clear
__global__ void tick_kernel(const Device dv, const StepPtrs sp) {
    if (threadIdx.x == 0) finish_step(dv, sp);
}

// The near tiles of the step of parity q (one block): the marks of that
// parity's previous list are cleared, then every TILE_X-cell tile of an
// x-row that meets the remap cube of a body in `states` grown by one cell is
// marked and listed once.  The cube is the remap's: half-width
// E + REMAP_MARGIN around floor(X).  Also stores the step's index.
__global__ void __launch_bounds__(512) near_tiles_kernel(const Device dv, const BodyState *states, int q,
                                                         int step_offset) {
    const Domain d = dv.dom;
    unsigned *mask = dv.near_mask[q];
    int *list = dv.near_list[q];
    const int old = min(dv.near_count[q], dv.near_cap);
    for (int i = threadIdx.x; i < old; i += blockDim.x) mask[list[i]] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        dv.near_count[q] = 0;
        dv.tstep[q] = *dv.t_dev + step_offset;
    }
    __syncthreads();
    const int ntx = (d.nx + TILE_X - 1) / TILE_X;
    const int n3[3] = {d.nx, d.ny, d.nz}, per[3] = {d.px, d.py, d.pz};
    for (int b = 0; b < dv.nb; ++b) {
        const int half = dv.props[b].E + REMAP_MARGIN + 1;
        const int side = 2 * half + 1;
        int o[3];
        for (int a = 0; a < 3; ++a) o[a] = (int)floor(states[b].X[a]) - half;
        for (int r = threadIdx.x; r < side * side; r += blockDim.x) {
            int y = o[1] + r % side, z = o[2] + r / side;
            if (per[1]) y = ((y % n3[1]) + n3[1]) % n3[1]; else if (y < 0 || y >= n3[1]) continue;
            if (per[2]) z = ((z % n3[2]) + n3[2]) % n3[2]; else if (z < 0 || z >= n3[2]) continue;
            // the row's x range as up to two unwrapped pieces [lo, hi]
            int lo[2], hi[2], pieces = 1;
            if (!per[0]) {
                lo[0] = max(o[0], 0);
                hi[0] = min(o[0] + side - 1, n3[0] - 1);
            } else if (side >= n3[0]) {
                lo[0] = 0;
                hi[0] = n3[0] - 1;
            } else {
                const int x0 = ((o[0] % n3[0]) + n3[0]) % n3[0];
                lo[0] = x0;
                hi[0] = min(x0 + side - 1, n3[0] - 1);
                if (x0 + side - 1 >= n3[0]) {
                    lo[1] = 0;
                    hi[1] = x0 + side - 1 - n3[0];
                    pieces = 2;
                }
            }
            const long long rowt = ((long long)z * n3[1] + y) * ntx;
            for (int k = 0; k < pieces; ++k)
                for (int cx = lo[k] / TILE_X; lo[k] <= hi[k] && cx <= hi[k] / TILE_X; ++cx) {
                    const int t = (int)(rowt + cx);
                    if (atomicExch(mask + t, 1u) == 0u) {
                        const int i = atomicAdd(dv.near_count + q, 1);
                        if (i < dv.near_cap) list[i] = t;
                        else atomicOr(dv.status, ST_LINKS);
                    }
                }
        }
    }
}

// the rigid-body step alone (bodies without fluid), one block: the loads,
// then a warp a body
__global__ void __launch_bounds__(256) integrate_kernel(const Device dv, const StepPtrs sp, int with_fluid) {
    body_loads(dv, sp, threadIdx.x, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int b = threadIdx.x >> 5; b < dv.nb; b += blockDim.x >> 5) integrate_body_warp(dv, sp, b, with_fluid);
    __syncthreads();
    if (threadIdx.x == 0) finish_step(dv, sp);
}

// ---- field export / import -----------------------------------------------

template <typename T, typename O>
__global__ void export_kernel(const Device dv, const T *pop, const uint8_t *flags, const uint8_t *bid,
                              int what, int mask_solid, O *out) {
    const Domain d = dv.dom;
    const long long C = d.C;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const float s = dv.f16_inv_scale;
    const bool solid = mask_solid && (flags[c] & F_SOLID);
    if (what == 2) {
        reinterpret_cast<uint8_t *>(out)[c] = solid ? (uint8_t)(bid[c] + 1) : 0;
        return;
    }
    if (what == 3) {
        for (int a = 0; a < Q; ++a) out[a * C + c] = (O)(wgt(a) + load_dev<T>(pop + a * C + c, s));
        return;
    }
    double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < Q; ++a) {
        const double v = load_dev<T>(pop + a * C + c, s);
        drho += v;
        j[0] += ex(a) * v; j[1] += ey(a) * v; j[2] += ez(a) * v;
    }
    const double rho = 1.0 + drho;
    if (what == 0) {
        out[c] = (O)(solid ? 1.0 : rho);
    } else {
        for (int i = 0; i < 3; ++i) out[i * C + c] = (O)(solid ? 0.0 : (j[i] - 0.5 * dv.g[i]) / rho);
    }
}

// Running time average of the velocity (Sec. 6, the flow fields averaged
// over swimming cycles): each step adds the velocity of the populations it
// wrote, u = (sum e f~ - g/2) / rho (0 in obstacle cells, the value the U
// field reports), to an FP64 sum per cell and component.  The moments are
// FP64 for FP64 storage and FP32 otherwise (FP64 arithmetic is slow on this
// part); the sum is FP64 so that long windows keep their digits.
template <typename T>
__global__ void __launch_bounds__(256) average_kernel(const Device dv, const StepPtrs sp) {
    const long long C = dv.dom.C;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double u[3] = {0.0, 0.0, 0.0};
    if (!(sp.flags_cur[c] & F_SOLID)) {
        const T *pop = static_cast<const T *>(sp.dst);
        if constexpr (sizeof(T) == 8) {
            double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < Q; ++a) {
                const double v = pop[a * C + c];
                drho += v;
                j[0] += ex(a) * v; j[1] += ey(a) * v; j[2] += ez(a) * v;
            }
            for (int i = 0; i < 3; ++i) u[i] = (j[i] - 0.5 * dv.g[i]) / (1.0 + drho);
        } else {
            float drho = 0.0f, j[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const float v = load_dev_f<T>(pop + a * C + c, dv.f16_inv_scale);
                drho += v;
                if (ex(a)) j[0] += ex(a) > 0 ? v : -v;
                if (ey(a)) j[1] += ey(a) > 0 ? v : -v;
                if (ez(a)) j[2] += ez(a) > 0 ? v : -v;
            }
            const float inv = 1.0f / (1.0f + drho);
            for (int i = 0; i < 3; ++i) u[i] = (double)((j[i] - 0.5f * dv.g_f[i]) * inv);
        }
    }
    for (int i = 0; i < 3; ++i) dv.avg_u[i * C + c] += u[i];
    if (c == 0) *dv.avg_n += 1;
}

template <typename T>
__global__ void import_kernel(const Device dv, T *pop, const double *in) {
    const long long C = dv.dom.C;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    for (int a = 0; a < Q; ++a) {
        const double delta = in[a * C + c] - wgt(a);
        if constexpr (sizeof(T) == 8) pop[a * C + c] = delta;
        else if constexpr (sizeof(T) == 4) pop[a * C + c] = (float)delta;
        else if constexpr (std::is_same<T, __half>::value) pop[a * C + c] = __float2half_rn((float)delta * dv.f16_scale);
        else pop[a * C + c] = __float2bfloat16_rn((float)delta);
    }
}

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

void launch_init_flags(const Device &dv, uint8_t *flags0, uint8_t *flags1, uint8_t *bid0, uint8_t *bid1,
                       cudaStream_t s) {
    init_flags_kernel<<<blocks_for(dv.dom.C, 256), 256, 0, s>>>(dv.dom, flags0, flags1, bid0, bid1);
}

void launch_prep(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    prep_kernel<<<1, PREP_THREADS, 0, s>>>(dv, sp);
}

void launch_remap(const Device &dv, const StepPtrs &sp, int init_mode, cudaStream_t s, bool prep) {
    if (prep) launch_prep(dv, sp, s);
    const int side = dv.remap_side;
    launch_kernel(dv.pdl != 0, remap_kernel, dim3((unsigned)remap_blocks(side), dv.nb), dim3(REMAP_THREADS), 0, s,
                  dv, sp, init_mode);
}

void launch_links(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    links_kernel<<<dim3(dv.link_side, dv.nb), 256, 0, s>>>(dv, sp);
    loads_kernel<<<1, 64, 0, s>>>(dv, sp);
}

void launch_force(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const dim3 grid(FORCE_BLOCKS, dv.nb), block(FORCE_THREADS);
    const bool pdl = dv.pdl != 0;
    switch (dv.precision) {
    case 0: launch_kernel(pdl, force_kernel<double>, grid, block, 0, s, dv, sp); break;
    case 1: launch_kernel(pdl, force_kernel<float>, grid, block, 0, s, dv, sp); break;
    case 2: launch_kernel(pdl, force_kernel<__half>, grid, block, 0, s, dv, sp); break;
    default: launch_kernel(pdl, force_kernel<__nv_bfloat16>, grid, block, 0, s, dv, sp); break;
    }
}

void launch_integrate(const Device &dv, const StepPtrs &sp, int with_fluid, cudaStream_t s) {
    integrate_kernel<<<1, 256, 0, s>>>(dv, sp, with_fluid);
}

void launch_tick(const Device &dv, const StepPtrs &sp, cudaStream_t s) { tick_kernel<<<1, 32, 0, s>>>(dv, sp); }

void launch_near_tiles(const Device &dv, const BodyState *states, int q, int step_offset, cudaStream_t s) {
    near_tiles_kernel<<<1, 512, 0, s>>>(dv, states, q, step_offset);
}

long long near_tile_count(const Device &dv) {
    return (long long)((dv.dom.nx + TILE_X - 1) / TILE_X) * dv.dom.ny * dv.dom.nz;
}

int near_tile_cap(const Device &dv, int emax) {
    const long long side = 2LL * (emax + REMAP_MARGIN + 1) + 1;
    const long long per_body = side * side * ((side + TILE_X - 1) / TILE_X + 1);
    return (int)std::min<long long>((long long)dv.nb * per_body, near_tile_count(dv));
}

// the grids of launch_remap, launch_links and launch_force for one lattice
void batch_grid_small(const Device &dv, int k, int g[3]) {
    g[0] = g[1] = g[2] = 0;
    if (dv.nb == 0) return;
    const int side = dv.remap_side;
    switch (k) {
    case BK_PREP: case BK_LOADS: g[0] = g[1] = g[2] = 1; break;
    case BK_REMAP:
        g[0] = remap_blocks(side);
        g[1] = dv.nb; g[2] = 1;
        break;
    case BK_LINKS: g[0] = dv.link_side; g[1] = dv.nb; g[2] = 1; break;
    case BK_FORCE: g[0] = FORCE_BLOCKS; g[1] = dv.nb; g[2] = 1; break;
    default: break;
    }
}

void launch_batch_small(int k, const Batch &bt, unsigned blocks, int precision, cudaStream_t s) {
    if (blocks == 0) return;
    switch (k) {
    case BK_PREP: prep_batch<<<blocks, PREP_THREADS, 0, s>>>(bt); break;
    case BK_REMAP: remap_batch<<<blocks, REMAP_THREADS, 0, s>>>(bt); break;
    case BK_LINKS: links_batch<<<blocks, 256, 0, s>>>(bt); break;
    case BK_LOADS: loads_batch<<<blocks, 64, 0, s>>>(bt); break;
    case BK_FORCE:
        switch (precision) {
        case 0: force_batch<double><<<blocks, FORCE_THREADS, 0, s>>>(bt); break;
        case 1: force_batch<float><<<blocks, FORCE_THREADS, 0, s>>>(bt); break;
        case 2: force_batch<__half><<<blocks, FORCE_THREADS, 0, s>>>(bt); break;
        default: force_batch<__nv_bfloat16><<<blocks, FORCE_THREADS, 0, s>>>(bt); break;
        }
        break;
    default: break;
    }
}

template <typename O>
static void export_typed(const Device &dv, const void *pop, const uint8_t *flags, const uint8_t *bid,
                         int what, int mask_solid, O *out, cudaStream_t s) {
    const unsigned bl = blocks_for(dv.dom.C, 256);
    switch (dv.precision) {
    case 0: export_kernel<double, O><<<bl, 256, 0, s>>>(dv, (const double *)pop, flags, bid, what, mask_solid, out); break;
    case 1: export_kernel<float, O><<<bl, 256, 0, s>>>(dv, (const float *)pop, flags, bid, what, mask_solid, out); break;
    case 2: export_kernel<__half, O><<<bl, 256, 0, s>>>(dv, (const __half *)pop, flags, bid, what, mask_solid, out); break;
    default: export_kernel<__nv_bfloat16, O><<<bl, 256, 0, s>>>(dv, (const __nv_bfloat16 *)pop, flags, bid, what, mask_solid, out); break;
    }
}

void launch_export(const Device &dv, const void *pop, const uint8_t *flags, const uint8_t *bid, int what,
                   int mask_solid, void *out, int dtype, cudaStream_t s) {
    if (dtype == 1) export_typed<float>(dv, pop, flags, bid, what, mask_solid, static_cast<float *>(out), s);
    else export_typed<double>(dv, pop, flags, bid, what, mask_solid, static_cast<double *>(out), s);
}

void launch_average(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const unsigned bl = blocks_for(dv.dom.C, 256);
    switch (dv.precision) {
    case 0: average_kernel<double><<<bl, 256, 0, s>>>(dv, sp); break;
    case 1: average_kernel<float><<<bl, 256, 0, s>>>(dv, sp); break;
    case 2: average_kernel<__half><<<bl, 256, 0, s>>>(dv, sp); break;
    default: average_kernel<__nv_bfloat16><<<bl, 256, 0, s>>>(dv, sp); break;
    }
}

void launch_import_pop(const Device &dv, void *pop, const double *in, cudaStream_t s) {
    const unsigned bl = blocks_for(dv.dom.C, 256);
    switch (dv.precision) {
    case 0: import_kernel<double><<<bl, 256, 0, s>>>(dv, (double *)pop, in); break;
    case 1: import_kernel<float><<<bl, 256, 0, s>>>(dv, (float *)pop, in); break;
    case 2: import_kernel<__half><<<bl, 256, 0, s>>>(dv, (__half *)pop, in); break;
    default: import_kernel<__nv_bfloat16><<<bl, 256, 0, s>>>(dv, (__nv_bfloat16 *)pop, in); break;
    }
}

}  // namespace lbm
