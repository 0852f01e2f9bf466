// kernels.cu -- the per-body kernels of one coupled step and the field
// export / import kernels:
//   remap      map the bodies onto the lattice (Sec. 2.3), epoch flags
//   links      per-body list of fluid->solid links (ballot + block scan)
//   force      momentum-exchange force and torque (Eq. hydroF), FP64,
//              warp-shuffle reduction in a fixed order (deterministic)
//   integrate  drive (Eq. FB1-FB3), springs (Eq. osci_i, osci_j) and the
//              rigid-body time step (Algorithm 1), FP64, one thread a body
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
// then the distance in FP32 from that small, nearly exact offset.  Returns 1
// (inside) or 0 (outside) when the squared distance is farther than
// 2e-2 max(r^2, 1) from r^2 -- orders of magnitude above its FP32 error --
// and -1 otherwise (the FP64 test decides), so the map is the FP64 map bit
// for bit.
__device__ inline int inside_screen(const Domain &d, const BodyProps &p, const int (&ci)[3], const float (&cf)[3],
                                    const float (&a)[3], int x, int y, int z) {
    const int n3[3] = {d.nx, d.ny, d.nz}, per[3] = {d.px, d.py, d.pz}, q3[3] = {x, y, z};
    float o[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        int io = q3[i] - ci[i];
        if (per[i]) io = 2 * io > n3[i] ? io - n3[i] : (2 * io < -n3[i] ? io + n3[i] : io);
        o[i] = (float)io - cf[i];
    }
    const float o0 = o[0], o1 = o[1], o2 = o[2];
    float d2;
    if (p.shape == 0) {
        d2 = o0 * o0 + o1 * o1 + o2 * o2;
    } else {
        const float h = (float)(0.5 * p.l);
        float sp = o0 * a[0] + o1 * a[1] + o2 * a[2];
        sp = sp > h ? h : (sp < -h ? -h : sp);
        const float e0 = o0 - sp * a[0], e1 = o1 - sp * a[1], e2 = o2 - sp * a[2];
        d2 = e0 * e0 + e1 * e1 + e2 * e2;
    }
    const float r2 = (float)(p.r * p.r);
    const float margin = 2e-2f * fmaxf(r2, 1.0f);
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

// Remap: block row blockIdx.y = body b; the threads cover the cube of side
// 2 (E_b + REMAP_MARGIN) + 1 around floor(X_b) at state n.  Every covered
// cell gets its epoch-n flags from the geometry of all bodies and the
// epoch-(n-1) buffer; overlapping cubes write identical values.  Bodies are
// culled with integer boxes first, so the FP64 inside test runs only for
// the bodies whose box holds the cell.
constexpr int REMAP_THREADS = 256;
// A cell farther than this from a body's bounding box [floor(X - reach),
// floor(X + reach)] can hold no flag of that body in epochs n-2 .. n: solid
// cells of epoch n-3 lie within 1.5 cells of the current extent, NEAR adds a
// neighbour's 1.42 cells, and the floor of the upper bound loses up to one.
constexpr int STATIC_REACH = 4;

__global__ void __launch_bounds__(REMAP_THREADS) remap_kernel(const Device dv, const StepPtrs sp, int init_mode) {
    const Domain d = dv.dom;
    const int b = blockIdx.y;
    __shared__ int box[LBM_MAX_BODIES_DEV][6];     // wrapped lower corner, width per axis
    __shared__ int ebox[LBM_MAX_BODIES_DEV][6];    // the same grown by STATIC_REACH cells
    __shared__ int cwi[LBM_MAX_BODIES_DEV][3];     // wrapped centre: cell
    __shared__ float cwf[LBM_MAX_BODIES_DEV][3];   // and offset within it
    __shared__ float ax[LBM_MAX_BODIES_DEV][3];    // body x axis
    __shared__ int origin[3];                      // cell of this block's cube corner
    const int n3[3] = {d.nx, d.ny, d.nz}, per[3] = {d.px, d.py, d.pz};
    if (threadIdx.x == 0) {
        const BodyState sb0 = sp.body_cur[blockIdx.y];
        const int half0 = dv.props[blockIdx.y].E + REMAP_MARGIN;
        for (int a = 0; a < 3; ++a) origin[a] = (int)floor(sb0.X[a]) - half0;
    }
    for (int k = threadIdx.x; k < dv.nb; k += blockDim.x) {
        const BodyState sk = sp.body_cur[k];
        const BodyProps pk = dv.props[k];
        const double reach = pk.r + 0.5 * pk.l;
        {
            const double inv[3] = {d.inx, d.iny, d.inz};
            for (int a = 0; a < 3; ++a) {
                const double c = per[a] ? sk.X[a] - n3[a] * floor(sk.X[a] * inv[a]) : sk.X[a];
                const double fc = floor(c);
                cwi[k][a] = (int)fc;
                cwf[k][a] = (float)(c - fc);
            }
        }
        const double w = sk.q[0], qx = sk.q[1], qy = sk.q[2], qz = sk.q[3];
        ax[k][0] = (float)(1 - 2 * (qy * qy + qz * qz));
        ax[k][1] = (float)(2 * (qx * qy + w * qz));
        ax[k][2] = (float)(2 * (qx * qz - w * qy));
        for (int a = 0; a < 3; ++a) {
            int lo = (int)floor(sk.X[a] - reach), hi = (int)floor(sk.X[a] + reach);
            int width = hi - lo + 1;
            int elo = lo - STATIC_REACH, ewidth = width + 2 * STATIC_REACH;
            if (per[a]) {
                lo %= n3[a];
                if (lo < 0) lo += n3[a];
                if (width > n3[a]) width = n3[a];
                elo %= n3[a];
                if (elo < 0) elo += n3[a];
                if (ewidth > n3[a]) ewidth = n3[a];
            }
            box[k][a] = lo;
            box[k][3 + a] = width;
            ebox[k][a] = elo;
            ebox[k][3 + a] = ewidth;
        }
    }
    __syncthreads();
    const BodyProps pb = dv.props[b];
    const BodyState sb = sp.body_cur[b];
    const int half = pb.E + REMAP_MARGIN;
    const int side = 2 * half + 1;
    const int vol = side * side * side;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l == 0) {
        // a body may not cross a wall (its extent beyond the wall planes)
        double R[3][3];
        quat_to_matrix(sb.q, R);
        for (int k = 0; k < 3; ++k) {
            if (per[k]) continue;
            const double ext = pb.r + (pb.shape == 1 ? 0.5 * pb.l * fabs(R[k][0]) : 0.0);
            if (sb.X[k] - ext < -0.5 || sb.X[k] + ext > n3[k] - 0.5) atomicOr(dv.status, ST_OUTSIDE);
        }
    }
    if (l >= vol) return;
    const int lx = l % side, ly = (l / side) % side, lz = l / (side * side);
    int x = origin[0] + lx;
    int y = origin[1] + ly;
    int z = origin[2] + lz;
    if (d.px) x = ((x % d.nx) + d.nx) % d.nx; else if (x < 0 || x >= d.nx) return;
    if (d.py) y = ((y % d.ny) + d.ny) % d.ny; else if (y < 0 || y >= d.ny) return;
    if (d.pz) z = ((z % d.nz) + d.nz) % d.nz; else if (z < 0 || z >= d.nz) return;
    const long long c = ((long long)z * d.ny + y) * d.nx + x;
    const int p3[3] = {x, y, z};

    int id = NO_BODY;
    bool reached = false;           // within STATIC_REACH cells of some body's box
    for (int k = 0; k < dv.nb; ++k) {
        bool in = true;
        for (int a = 0; a < 3 && in; ++a) {
            int o = p3[a] - ebox[k][a];
            if (per[a] && o < 0) o += n3[a];
            in = o >= 0 && o < ebox[k][3 + a];
        }
        if (!in) continue;
        reached = true;
        for (int a = 0; a < 3 && in; ++a) {
            int o = p3[a] - box[k][a];
            if (per[a] && o < 0) o += n3[a];
            in = o >= 0 && o < box[k][3 + a];
        }
        if (!in) continue;
        // FP32 screen; cells within its margin of the surface take the FP64 test
        const BodyProps pk = dv.props[k];
        const int screen = inside_screen(d, pk, cwi[k], cwf[k], ax[k], x, y, z);
        if (screen == 0 || (screen < 0 && !cell_inside(d, pk, sp.body_cur[k], x, y, z))) continue;
        if (id != NO_BODY) atomicOr(dv.status, ST_OVERLAP);
        id = k;
    }
    // farther than STATIC_REACH from every body's box: the cell holds its
    // static flags in both epoch buffers already (nothing within reach was
    // solid in the last three steps, at most 0.5 cells of motion per step)
    if (!reached) return;
    const uint8_t solid = id != NO_BODY ? F_SOLID : 0;
    uint8_t flags = solid | wall_bit(d, x, y, z);
    if (!init_mode) {
        const uint8_t prev = sp.flags_prev[c] & F_SOLID;
        if (prev) flags |= F_SOLID_PREV;
        // does any pull source x - e_a hold an obstacle of step n-1?  (all
        // 18 loads are independent; sources beyond a wall do not count)
        uint8_t near = 0;
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            const int sx = x - ex(a), sy = y - ey(a), sz = z - ez(a);
            const bool in = !((!d.px && (sx < 0 || sx >= d.nx)) || (!d.py && (sy < 0 || sy >= d.ny)) ||
                              (!d.pz && (sz < 0 || sz >= d.nz)));
            const uint8_t v = sp.flags_prev[((long long)wrap_axis(sz, d.nz) * d.ny + wrap_axis(sy, d.ny)) * d.nx +
                                            wrap_axis(sx, d.nx)];
            near |= in ? v : 0;
        }
        if (near & F_SOLID) flags |= F_NEAR;
        if ((solid != 0) != (prev != 0) || (solid && sp.bid_prev[c] != id)) dv.changed[sp.parity] = 1;
    }
    sp.flags_cur[c] = flags;
    sp.bid_cur[c] = (uint8_t)id;
}

// Links: block (k, b) scans z-plane k of the cube of side 2 E_b + 3 around
// floor(X_b) and stores the links (x_f, a) with x_f fluid and x_f + e_a a
// cell of body b, in (y, x, a) order, into segment (b, k).  Runs only when
// the remap changed a flag; otherwise the previous lists stand.
__global__ void links_kernel(const Device dv, const StepPtrs sp) {
    if (dv.changed[sp.parity] == 0) return;
    const Domain d = dv.dom;
    const int b = blockIdx.y, k = blockIdx.x;
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

// Rigid-body step (Algorithm 1, Eq. totalFSwimmer) for all bodies, run by
// one block of 256 threads.  Phase 1 (threads over drive terms and springs)
// evaluates every drive term (Eq. FB1-FB3) and spring force (Eq. osci_i,
// osci_j) into scratch; phase 2 (thread b) adds, in order, the momentum-
// exchange partial sums, g times the volume, its drive terms in term order
// and its springs in spring order, then advances by semi-implicit Euler
// (dt = 1) in FP64.
__device__ void integrate_block(const Device &dv, const StepPtrs &sp, int with_fluid) {
    const long long tstep = *dv.t_dev;
    const double t = (double)tstep;
    for (int k = threadIdx.x; k < dv.nd; k += blockDim.x) {
        const DriveTerm dt = dv.drives[k];
        double f = 0.0;
        if (!(t < dt.t_on || t >= dt.t_off)) f = dt.amp * sin(dt.omega * t - dt.phase);
        double R[3][3];                                 // the drive acts along R(q) axis
        quat_to_matrix(sp.body_cur[dt.body].q, R);
        for (int i = 0; i < 3; ++i)
            dv.drive_f[3 * k + i] = f * (R[i][0] * dt.axis[0] + R[i][1] * dt.axis[1] + R[i][2] * dt.axis[2]);
    }
    for (int k = threadIdx.x; k < dv.ns; k += blockDim.x) {
        const Spring sp_ = dv.springs[k];
        const BodyState si = sp.body_cur[sp_.i], sj = sp.body_cur[sp_.j];
        const double dd[3] = {si.X[0] - sj.X[0], si.X[1] - sj.X[1], si.X[2] - sj.X[2]};
        const double len = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        const double inv_len = len > 0 ? 1.0 / len : 0.0;
        for (int i = 0; i < 3; ++i)
            dv.spring_f[3 * k + i] = -sp_.k * (len - sp_.rest) * (dd[i] * inv_len) - sp_.gamma * (si.V[i] - sj.V[i]);
    }
    __syncthreads();
    const int b = threadIdx.x;
    if (b < dv.nb) {
        const BodyProps pb = dv.props[b];
        const BodyState s = sp.body_cur[b];
        double R[3][3];
        quat_to_matrix(s.q, R);
        double F[3], Tq[3];
        for (int i = 0; i < 6; ++i) {
            double v = 0.0;
            if (with_fluid)
                for (int k = 0; k < FORCE_BLOCKS; ++k) v += dv.fpart[((long long)b * FORCE_BLOCKS + k) * 6 + i];
            const double prev = dv.fh[b * 6 + i];
            dv.fh[b * 6 + i] = v;
            if (dv.avg_force && tstep > 0) v = 0.5 * (v + prev);
            if (i < 3) F[i] = v + dv.g[i] * pb.volume; else Tq[i - 3] = v;
        }
        for (int k = pb.drive_first; k < pb.drive_first + pb.drive_count; ++k)
            for (int i = 0; i < 3; ++i) F[i] += dv.drive_f[3 * k + i];
        for (int kk = pb.spring_first; kk < pb.spring_first + pb.spring_count; ++kk) {
            const int k = dv.spring_list[kk];
            const bool first = dv.springs[k].i == b;
            for (int i = 0; i < 3; ++i) F[i] += first ? dv.spring_f[3 * k + i] : -dv.spring_f[3 * k + i];
        }
        BodyState n = s;
        for (int i = 0; i < 3; ++i) {
            n.V[i] = s.V[i] + F[i] * pb.inv_m;
            n.X[i] = s.X[i] + n.V[i];
        }
        // Omega += R diag(1/I) R^T T
        double Tb[3], dW[3];
        for (int i = 0; i < 3; ++i)
            Tb[i] = (R[0][i] * Tq[0] + R[1][i] * Tq[1] + R[2][i] * Tq[2]) * pb.inv_inertia[i];
        for (int i = 0; i < 3; ++i) dW[i] = R[i][0] * Tb[0] + R[i][1] * Tb[1] + R[i][2] * Tb[2];
        for (int i = 0; i < 3; ++i) n.W[i] = s.W[i] + dW[i];
        // q += 1/2 (0, Omega) (x) q, renormalised
        const double w = s.q[0], v0 = s.q[1], v1 = s.q[2], v2 = s.q[3];
        const double c0 = n.W[1] * v2 - n.W[2] * v1, c1 = n.W[2] * v0 - n.W[0] * v2,
                     c2 = n.W[0] * v1 - n.W[1] * v0;
        double q4[4] = {w - 0.5 * (n.W[0] * v0 + n.W[1] * v1 + n.W[2] * v2),
                        v0 + 0.5 * (w * n.W[0] + c0), v1 + 0.5 * (w * n.W[1] + c1),
                        v2 + 0.5 * (w * n.W[2] + c2)};
        const double inv_nn = rsqrt(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
        for (int i = 0; i < 4; ++i) n.q[i] = q4[i] * inv_nn;
        bool finite = true;
        for (int i = 0; i < 3; ++i)
            finite = finite && isfinite(n.X[i]) && isfinite(n.V[i]) && isfinite(n.W[i]);
        if (!finite) atomicOr(dv.status, ST_NAN);
        else if (fabs(n.V[0]) > MAX_STEP || fabs(n.V[1]) > MAX_STEP || fabs(n.V[2]) > MAX_STEP)
            atomicOr(dv.status, ST_UNSTABLE);
        sp.body_next[b] = n;
        if (dv.tape) {
            const TapeCtl tc = *dv.tape;
            const long long j = tstep - tc.t0;
            if (tc.on && j >= 0 && j < tc.cap) {
                const double *src = &n.X[0];
                double *st = tc.state + ((j + 2) * dv.nb + b) * 13;
                for (int i = 0; i < 13; ++i) st[i] = src[i];
                for (int i = 0; i < 6; ++i) tc.force[(j * dv.nb + b) * 6 + i] = dv.fh[b * 6 + i];
            }
        }
        if (dv.hist) {
            double *h = dv.hist + ((tstep % dv.hist_cap) * dv.nb + b) * 13;
            const double *src = &n.X[0];
            for (int i = 0; i < 13; ++i) h[i] = src[i];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *dv.t_dev = tstep + 1;
        dv.changed[sp.parity ^ 1] = 0;
    }
}

// Momentum exchange (Eq. hydroF): blocks (k, b), k < FORCE_BLOCKS, split the
// links of body b into contiguous chunks and sum
//   F = sum e_a [2 f~_a(x_f) + 6 w_a rho(x_f) e_-a . u_w(x_f + e_a)],
//   T = sum (x_f + e_a / 2 - X) x F_link
// with f~ of step n (dst) and the body state of step n, in FP64; each block
// reduces with warp shuffles in a fixed order and writes its partial sums.
// The last block to finish then runs the rigid-body step for all bodies,
// adding the partial sums in block order (deterministic).
template <typename T>
__global__ void __launch_bounds__(FORCE_THREADS) force_kernel(const Device dv, const StepPtrs sp) {
    const Domain d = dv.dom;
    const int b = blockIdx.y, kb = blockIdx.x;
    const BodyProps pb = dv.props[b];
    const BodyState sb = sp.body_cur[b];
    const int side = 2 * (pb.E + 1) + 1;
    const int *counts = dv.seg_count + (long long)b * dv.link_side;
    const Link *links = dv.links + (long long)b * dv.link_side * dv.seg_cap;
    const T *pop = static_cast<const T *>(sp.dst);
    const long long C = d.C;
    const float s = dv.f16_inv_scale;
    // body centre wrapped into the domain (once per block)
    const double xw[3] = {d.px ? sb.X[0] - d.nx * floor(sb.X[0] * d.inx) : sb.X[0],
                          d.py ? sb.X[1] - d.ny * floor(sb.X[1] * d.iny) : sb.X[1],
                          d.pz ? sb.X[2] - d.nz * floor(sb.X[2] * d.inz) : sb.X[2]};
    const int ci[3] = {(int)floor(xw[0]), (int)floor(xw[1]), (int)floor(xw[2])};
    const double cfr[3] = {xw[0] - ci[0], xw[1] - ci[1], xw[2] - ci[2]};
    const float vf[3] = {(float)sb.V[0], (float)sb.V[1], (float)sb.V[2]};
    const float wf[3] = {(float)sb.W[0], (float)sb.W[1], (float)sb.W[2]};

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
        if constexpr (sizeof(T) == 8) {
            for (int q = 0; q < Q; ++q) rho += load_dev<T>(pop + q * C + c, s);
        } else {
            float drho = 0.0f;          // FP32 sum of the stored deviations
            for (int q = 0; q < Q; ++q) drho += (float)load_dev<T>(pop + q * C + c, s);
            rho += (double)drho;
        }
        // the link terms in FP64: the force is a small difference of ~1e3
        // terms of size ~0.1 (2 f~_a), which FP32 terms would not keep
        const double g_a = wgt(a) + load_dev<T>(pop + a * C + c, s);
        double o0, o1, o2, mag;
        if constexpr (sizeof(T) == 8) {
            // offsets of the fluid cell, of the link end and of the link midpoint
            o0 = wrap_near(x - xw[0], d.nx, d.px);
            o1 = wrap_near(y - xw[1], d.ny, d.py);
            o2 = wrap_near(z - xw[2], d.nz, d.pz);
            const double e0 = o0 + ex(a), e1 = o1 + ey(a), e2 = o2 + ez(a);
            const double u0 = sb.V[0] + (sb.W[1] * e2 - sb.W[2] * e1);
            const double u1 = sb.V[1] + (sb.W[2] * e0 - sb.W[0] * e2);
            const double u2 = sb.V[2] + (sb.W[0] * e1 - sb.W[1] * e0);
            const double eu = -(ex(a) * u0 + ey(a) * u1 + ez(a) * u2);   // e_-a . u_w
            mag = 2.0 * g_a + 6.0 * wgt(a) * rho * eu;
        } else {
            // offsets from the centre's cell (integer minimum image) and its
            // FP64 fraction; the moving-wall term (~1e-3 of the link) in FP32
            o0 = (double)near_cell_k(x - ci[0], d.nx, d.px) - cfr[0];
            o1 = (double)near_cell_k(y - ci[1], d.ny, d.py) - cfr[1];
            o2 = (double)near_cell_k(z - ci[2], d.nz, d.pz) - cfr[2];
            const float e0 = (float)o0 + ex(a), e1 = (float)o1 + ey(a), e2 = (float)o2 + ez(a);
            const float u0 = vf[0] + (wf[1] * e2 - wf[2] * e1);
            const float u1 = vf[1] + (wf[2] * e0 - wf[0] * e2);
            const float u2 = vf[2] + (wf[0] * e1 - wf[1] * e0);
            const float eu = -(ex(a) * u0 + ey(a) * u1 + ez(a) * u2);
            mag = 2.0 * g_a + (double)((float)(6.0 * wgt(a)) * (float)rho * eu);
        }
        const double fl[3] = {ex(a) * mag, ey(a) * mag, ez(a) * mag};
        const double m0 = o0 + 0.5 * ex(a), m1 = o1 + 0.5 * ey(a), m2 = o2 + 0.5 * ez(a);
        acc[0] += fl[0]; acc[1] += fl[1]; acc[2] += fl[2];
        acc[3] += m1 * fl[2] - m2 * fl[1];
        acc[4] += m2 * fl[0] - m0 * fl[2];
        acc[5] += m0 * fl[1] - m1 * fl[0];
    }
    __shared__ double part[FORCE_THREADS / 32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    // the last block to finish integrates the bodies
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(dv.blocks_done, 1u);
        last = done == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    integrate_block(dv, sp, 1);
    if (threadIdx.x == 0) *dv.blocks_done = 0u;
}

// the rigid-body step alone (bodies without fluid)
__global__ void __launch_bounds__(256) integrate_kernel(const Device dv, const StepPtrs sp, int with_fluid) {
    integrate_block(dv, sp, with_fluid);
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

void launch_remap(const Device &dv, const StepPtrs &sp, int init_mode, cudaStream_t s) {
    const long long side = dv.remap_side;
    const unsigned bx = blocks_for(side * side * side, REMAP_THREADS);
    remap_kernel<<<dim3(bx, dv.nb), REMAP_THREADS, 0, s>>>(dv, sp, init_mode);
}

void launch_links(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    links_kernel<<<dim3(dv.link_side, dv.nb), 256, 0, s>>>(dv, sp);
}

void launch_force(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const dim3 grid(FORCE_BLOCKS, dv.nb);
    switch (dv.precision) {
    case 0: force_kernel<double><<<grid, FORCE_THREADS, 0, s>>>(dv, sp); break;
    case 1: force_kernel<float><<<grid, FORCE_THREADS, 0, s>>>(dv, sp); break;
    case 2: force_kernel<__half><<<grid, FORCE_THREADS, 0, s>>>(dv, sp); break;
    default: force_kernel<__nv_bfloat16><<<grid, FORCE_THREADS, 0, s>>>(dv, sp); break;
    }
}

void launch_integrate(const Device &dv, const StepPtrs &sp, int with_fluid, cudaStream_t s) {
    integrate_kernel<<<1, 256, 0, s>>>(dv, sp, with_fluid);
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
