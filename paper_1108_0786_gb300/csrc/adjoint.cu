// adjoint.cu -- reverse sweep of the coupled step: the transposed Jacobian of
// the rigid-body step (Algorithm 1 with Eq. FB1-FB3, osci_i, osci_j), of the
// momentum-exchange force (Eq. hydroF and its torque), of the LBGK collision
// with Guo's term (Eq. 2), of the refill of uncovered cells and of the stream
// with velocity-corrected bounce-back (Eq. 3, 4 and the moving-wall rule of
// Sec. 2.3).  The obstacle maps of the recorded forward run are held fixed.
//
// Reverse step n (forward step n maps G^{n-1}, S^{n-1}, S^n to G^n, S^{n+1}):
//   adj_integrate  Sh^{n+1} -> Sh^n (rigid-body part), Fh^n, Th^n, dJ/dtheta
//   adj cells      Ph^{n+1} (adjoint of the pre-collision populations of step
//                  n+1) -> Ah^n (adjoint of G^n: the transposed stream, the
//                  bounce-back and refill terms of step n+1 and the force
//                  terms of step n) -> Ph^n = collision^T Ah^n
// The cell part is a pull on the adjoint: cell x gathers Ph^{n+1}_a(x + e_a),
// the reverse of the forward pull.  Cells whose flags are zero in epochs n
// and n+1 (no obstacle in reach, no wall, not uncovered) take a pure gather
// (bulk kernel); the others (bodies' cubes, wall faces) the full rule, with
// the per-body adjoint sums reduced in a fixed order.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int ADJ_THREADS = 256;
// boundary blocks are small: the cube's few link cells carry nearly all of
// the work, and small blocks spread them over more SMs
constexpr int ADJ_BOUNDARY_THREADS = 64;

// density and velocity of step n from the post-collision deviations:
// rho = 1 + sum delta; the collision adds g to the momentum (Guo), so
// rho u = sum e delta - g / 2
template <typename A, typename T>
__device__ inline void moments_post(const T *G, long long C, long long c, const Device &dv, A &rho, A (&u)[3]) {
    A r = 0, j0 = 0, j1 = 0, j2 = 0;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        const A v = (A)G[(long long)b * C + c];
        r += v;
        j0 += (A)ex(b) * v; j1 += (A)ey(b) * v; j2 += (A)ez(b) * v;
    }
    rho = (A)1 + r;
    const A ir = (A)1 / rho;
    u[0] = (j0 - (A)(0.5 * dv.g[0])) * ir;
    u[1] = (j1 - (A)(0.5 * dv.g[1])) * ir;
    u[2] = (j2 - (A)(0.5 * dv.g[2])) * ir;
}

// Transposed Jacobian of the LBGK collision with Guo's forcing at one cell:
// a holds the adjoint of the post-collision populations on entry and that
// of the pre-collision ones on exit.
//   G_b = P_b - omega (P_b - feq_b(rho, u)) + (1 - omega / 2) w_b s_b(u)
//   rho = sum P, u = (sum e P + g / 2) / rho, d u_i / d P_a = (e_ai - u_i) / rho
template <typename A>
__device__ inline void collide_adjoint(A (&a)[Q], A rho, const A (&u)[3], const Device &dv) {
    const A om = (A)dv.omega;
    const A uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    A sr = 0, s0 = 0, s1 = 0, s2 = 0, f0 = 0, f1 = 0, f2 = 0;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        const A eu = (A)ex(b) * u[0] + (A)ey(b) * u[1] + (A)ez(b) * u[2];
        const A wa = (A)wgt(b) * a[b];
        sr += wa * ((A)1 + (A)3 * eu + (A)4.5 * eu * eu - (A)1.5 * uu);
        const A c = (A)3 + (A)9 * eu;
        s0 += wa * (c * (A)ex(b) - (A)3 * u[0]);
        s1 += wa * (c * (A)ey(b) - (A)3 * u[1]);
        s2 += wa * (c * (A)ez(b) - (A)3 * u[2]);
        if (dv.forced) {
            const A eg = (A)(ex(b) * dv.g[0] + ey(b) * dv.g[1] + ez(b) * dv.g[2]);
            f0 += wa * ((A)(-3.0 * dv.g[0]) + (A)9 * (A)ex(b) * eg);
            f1 += wa * ((A)(-3.0 * dv.g[1]) + (A)9 * (A)ey(b) * eg);
            f2 += wa * ((A)(-3.0 * dv.g[2]) + (A)9 * (A)ez(b) * eg);
        }
    }
    const A kf = (A)1 - (A)0.5 * om;
    const A ir = (A)1 / rho;
    const A su0 = (om * rho * s0 + kf * f0) * ir, su1 = (om * rho * s1 + kf * f1) * ir,
            su2 = (om * rho * s2 + kf * f2) * ir;
    const A base = om * sr - (su0 * u[0] + su1 * u[1] + su2 * u[2]);
#pragma unroll
    for (int b = 0; b < Q; ++b)
        a[b] = ((A)1 - om) * a[b] + base + (A)ex(b) * su0 + (A)ey(b) * su1 + (A)ez(b) * su2;
}

// adjoint of the body-surface velocity u_w(p) = V + W x (p - X) for the
// scalar uh . u_w: acc[0..2] += d/dX, acc[3..5] += d/dV, acc[6..8] += d/dW
// (terms formed in S, summed in Acc)
template <typename S, typename Acc>
__device__ inline void adj_surface(const S W[3], const S o[3], const S uh[3], Acc acc[9]) {
    acc[0] += (Acc)(W[1] * uh[2] - W[2] * uh[1]);
    acc[1] += (Acc)(W[2] * uh[0] - W[0] * uh[2]);
    acc[2] += (Acc)(W[0] * uh[1] - W[1] * uh[0]);
    acc[3] += (Acc)uh[0]; acc[4] += (Acc)uh[1]; acc[5] += (Acc)uh[2];
    acc[6] += (Acc)(o[1] * uh[2] - o[2] * uh[1]);
    acc[7] += (Acc)(o[2] * uh[0] - o[0] * uh[2]);
    acc[8] += (Acc)(o[0] * uh[1] - o[1] * uh[0]);
}

// ---- bulk cells: pure gather + transposed collision -------------------------
template <typename A, typename T, bool FIRST>
__global__ void __launch_bounds__(ADJ_THREADS) adj_bulk_kernel(const Device dv, const AdjPtrs ap) {
    const Domain d = dv.dom;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= d.nx || y >= d.ny) return;
    const long long C = d.C;
    const long long c = ((long long)z * d.ny + y) * d.nx + x;
    if (ap.flags_next[c] != 0 || (ap.flags_cur[c] & F_SOLID_PREV)) return;   // a boundary cell
    const A *__restrict__ ain = static_cast<const A *>(ap.ain);
    A a[Q];
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        const int sx = wrap_axis(x + ex(b), d.nx), sy = wrap_axis(y + ey(b), d.ny), sz = wrap_axis(z + ez(b), d.nz);
        a[b] = ain[(long long)b * C + ((long long)sz * d.ny + sy) * d.nx + sx];
    }
    if constexpr (!FIRST) {
        A rho, u[3];
        moments_post<A, T>(static_cast<const T *>(ap.G), C, c, dv, rho, u);
        collide_adjoint<A>(a, rho, u, dv);
    }
    A *__restrict__ aout = static_cast<A *>(ap.aout);
#pragma unroll
    for (int b = 0; b < Q; ++b) aout[(long long)b * C + c] = a[b];
}

// ---- wall-face cells: the full rule, a thread per cell -----------------------
// Block row blockIdx.y = wall face (axis * 2 + side) of a non-periodic axis.
// The body terms of the links of these cells are summed by adj_cube_kernel
// (a face cell next to a body lies in its cube); this kernel writes the
// adjoint of every face cell.  A cell in both is written twice with the
// same rule, this kernel's last.
template <typename A, typename T, bool FIRST>
__global__ void __launch_bounds__(ADJ_BOUNDARY_THREADS) adj_wall_kernel(const Device dv, const AdjPtrs ap) {
    const Domain d = dv.dom;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    int x = 0, y = 0, z = 0;
    bool live = true;
    {
        const int axis = blockIdx.y >> 1, hi = blockIdx.y & 1;
        const int n3[3] = {d.nx, d.ny, d.nz}, per[3] = {d.px, d.py, d.pz};
        if (per[axis]) return;
        const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
        if (l >= n3[ua] * n3[va]) return;
        int p[3];
        p[axis] = hi ? n3[axis] - 1 : 0;
        p[ua] = l % n3[ua];
        p[va] = l / n3[ua];
        x = p[0]; y = p[1]; z = p[2];
    }
    const long long C = d.C;
    const long long c = ((long long)z * d.ny + y) * d.nx + x;
    if (live) {
        const uint8_t fcur = ap.flags_cur[c], fnext = ap.flags_next[c];
        if (fnext == 0 && !(fcur & F_SOLID_PREV)) live = false;     // a bulk cell
        else if (fcur & F_SOLID) {                                    // obstacle at n: no adjoint
            A *aout = static_cast<A *>(ap.aout);
#pragma unroll
            for (int b = 0; b < Q; ++b) aout[(long long)b * C + c] = (A)0;
            if constexpr (!FIRST) static_cast<A *>(ap.rout)[c] = (A)0;
            live = false;
        }
        if (live) {
            const A *__restrict__ ain = static_cast<const A *>(ap.ain);
            const A *__restrict__ rin = static_cast<const A *>(ap.rin);
            const T *__restrict__ G = static_cast<const T *>(ap.G);
            A rho, u[3];
            moments_post<A, T>(G, C, c, dv, rho, u);
            const bool fluid_next = !(fnext & F_SOLID);
            A own[Q], a[Q];
#pragma unroll
            for (int b = 0; b < Q; ++b) own[b] = ain[(long long)b * C + c];
            a[0] = own[0];
            A cr = 0;
#pragma unroll
            for (int b = 1; b < Q; ++b) {
                const int zx = x + ex(b), zy = y + ey(b), zz = z + ez(b);
                const bool wall = (!d.px && (zx < 0 || zx >= d.nx)) || (!d.py && (zy < 0 || zy >= d.ny)) ||
                                  (!d.pz && (zz < 0 || zz >= d.nz));
                if (wall) {                      // Eq. 4 at step n+1
                    a[b] = own[opp(b)];
                    continue;
                }
                const long long zc = ((long long)wrap_axis(zz, d.nz) * d.ny + wrap_axis(zy, d.ny)) * d.nx +
                                     wrap_axis(zx, d.nx);
                const uint8_t fz = ap.flags_cur[zc];
                if (fz & F_SOLID) {
                    // link (x, b) of step n: moving bounce-back of step n+1 and
                    // the momentum exchange of step n share u_w(x + e_b; S^n).
                    // The offset from the body centre is taken in FP64, the
                    // link's terms in the adjoint's precision.
                    const int k = ap.bid_cur[zc];
                    const BodyState &sk = ap.body[k];
                    double od[3];
                    offset_from(d, sk, (double)zx, (double)zy, (double)zz, od);
                    const A o[3] = {(A)od[0], (A)od[1], (A)od[2]};
                    const A W[3] = {(A)sk.W[0], (A)sk.W[1], (A)sk.W[2]};
                    A uw[3];
                    uw[0] = (A)sk.V[0] + (W[1] * o[2] - W[2] * o[1]);
                    uw[1] = (A)sk.V[1] + (W[2] * o[0] - W[0] * o[2]);
                    uw[2] = (A)sk.V[2] + (W[0] * o[1] - W[1] * o[0]);
                    const A ua = -((A)ex(b) * uw[0] + (A)ey(b) * uw[1] + (A)ez(b) * uw[2]);   // e_-b . u_w
                    A mh = 0;
                    if constexpr (!FIRST) {
                        const double *fa = ap.fadj + 6 * k;
                        // (mid - X) x e_b, mid = x + e_b / 2 = (x + e_b) - e_b / 2
                        const A m[3] = {o[0] - (A)(0.5 * ex(b)), o[1] - (A)(0.5 * ey(b)), o[2] - (A)(0.5 * ez(b))};
                        const A t0 = m[1] * (A)ez(b) - m[2] * (A)ey(b), t1 = m[2] * (A)ex(b) - m[0] * (A)ez(b),
                                t2 = m[0] * (A)ey(b) - m[1] * (A)ex(b);
                        mh = (A)ex(b) * (A)fa[0] + (A)ey(b) * (A)fa[1] + (A)ez(b) * (A)fa[2] + t0 * (A)fa[3] +
                             t1 * (A)fa[4] + t2 * (A)fa[5];
                    }
                    const A wh = own[opp(b)];
                    a[b] = wh + (A)2 * mh;
                    cr += (A)(6.0 * wgt(b)) * ua * (wh + mh);
                    // z uncovered at n+1: x (fluid at n and n+1) fed its density
                    if (!(ap.flags_next[zc] & F_SOLID) && fluid_next) cr += rin[zc];
                } else {
                    a[b] = ain[(long long)b * C + zc];
                }
            }
#pragma unroll
            for (int b = 0; b < Q; ++b) a[b] += cr;
            A *__restrict__ aout = static_cast<A *>(ap.aout);
            if constexpr (FIRST) {
#pragma unroll
                for (int b = 0; b < Q; ++b) aout[(long long)b * C + c] = a[b];
            } else {
                collide_adjoint<A>(a, rho, u, dv);
#pragma unroll
                for (int b = 0; b < Q; ++b) aout[(long long)b * C + c] = a[b];
                A rh_out = 0;
                if (fcur & F_SOLID_PREV) {
                    // uncovered at n: P = f_eq(rho_avg, u_w(x; S^n)) of the body
                    // that covered x at n-1, rho_avg over the neighbours fluid
                    // in epochs n-1 and n (rho_avg = rho^n(x))
                    int cnt = 0;
#pragma unroll
                    for (int b = 1; b < Q; ++b) {
                        const int nx_ = x + ex(b), ny_ = y + ey(b), nz_ = z + ez(b);
                        const bool in = !((!d.px && (nx_ < 0 || nx_ >= d.nx)) || (!d.py && (ny_ < 0 || ny_ >= d.ny)) ||
                                          (!d.pz && (nz_ < 0 || nz_ >= d.nz)));
                        const long long nc = ((long long)wrap_axis(nz_, d.nz) * d.ny + wrap_axis(ny_, d.ny)) * d.nx +
                                             wrap_axis(nx_, d.nx);
                        if (in && !(ap.flags_cur[nc] & (F_SOLID | F_SOLID_PREV))) ++cnt;
                    }
                    const int k = ap.bid_prev[c];
                    if (k != NO_BODY) {
                        const BodyState sk = ap.body[k];
                        double o[3], uw[3];
                        offset_from(d, sk, (double)x, (double)y, (double)z, o);
                        uw[0] = sk.V[0] + (sk.W[1] * o[2] - sk.W[2] * o[1]);
                        uw[1] = sk.V[1] + (sk.W[2] * o[0] - sk.W[0] * o[2]);
                        uw[2] = sk.V[2] + (sk.W[0] * o[1] - sk.W[1] * o[0]);
                        const double uu = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
                        double rh = 0.0;
#pragma unroll
                        for (int b = 0; b < Q; ++b) {
                            const double eu = ex(b) * uw[0] + ey(b) * uw[1] + ez(b) * uw[2];
                            rh += (double)a[b] * wgt(b) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
                        }
                        if (cnt) rh_out = (A)(rh / cnt);
                    }
                }
                static_cast<A *>(ap.rout)[c] = rh_out;
            }
        }
    }
}

// ---- boundary cells of the body cubes: a warp per cell -------------------------
// Block (blk, kb) classifies the ADJ_BOUNDARY_THREADS cells blk * 64 ... of
// body kb's cube (cells whose flags are zero in epochs n and n+1 and that
// were not uncovered at n: adj_bulk's; solid at n: zero adjoint; the
// others the full rule, as adj_wall_kernel applies it) and lists the full-rule cells
// in cube order.  Each warp then takes the listed cells w, w + 8, ... with
// lane b the direction b: the pull, wall and link terms of the 18
// directions in parallel, the cell's sums (the density terms, the
// transposed collision's moments, the refill sums, body kb's terms) by
// butterfly shuffles, so every lane holds the same sum and the order is
// fixed.  The block adds its warps' body sums in warp order into
// part[kb][blk] (the layout adj_integrate reads).
constexpr int ADJ_CUBE_WARPS = 8;

template <typename V> __device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename A, typename T, bool FIRST>
__global__ void __launch_bounds__(32 * ADJ_CUBE_WARPS) adj_cube_kernel(const Device dv, const AdjPtrs ap) {
    const Domain d = dv.dom;
    const int kb = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long C = d.C;
    const int half = dv.props[kb].E + REMAP_MARGIN;
    const int side = 2 * half + 1;
    const BodyState &sb = ap.body[kb];
    const int fx = (int)floor(sb.X[0]), fy = (int)floor(sb.X[1]), fz = (int)floor(sb.X[2]);
    // cube cell l -> lattice cell (x, y, z); false outside the cube or the domain
    auto cube_cell = [&](int l, int &x, int &y, int &z) {
        if (l >= side * side * side) return false;
        bool live = true;
        x = fx - half + l % side;
        y = fy - half + (l / side) % side;
        z = fz - half + l / (side * side);
        if (d.px) x = ((x % d.nx) + d.nx) % d.nx; else live = live && x >= 0 && x < d.nx;
        if (d.py) y = ((y % d.ny) + d.ny) % d.ny; else live = live && y >= 0 && y < d.ny;
        if (d.pz) z = ((z % d.nz) + d.nz) % d.nz; else live = live && z >= 0 && z < d.nz;
        return live;
    };
    __shared__ int list[ADJ_BOUNDARY_THREADS];
    __shared__ int wcount[ADJ_BOUNDARY_THREADS / 32];
    __shared__ double wacc[ADJ_CUBE_WARPS][9];
    A *__restrict__ aout = static_cast<A *>(ap.aout);
    // 1. classify this block's cells (the first ADJ_BOUNDARY_THREADS threads)
    bool listed = false;
    const int l = blockIdx.x * ADJ_BOUNDARY_THREADS + tid;
    if (tid < ADJ_BOUNDARY_THREADS) {
        int x, y, z;
        if (cube_cell(l, x, y, z)) {
            const long long c = ((long long)z * d.ny + y) * d.nx + x;
            const uint8_t fcur = ap.flags_cur[c], fnext = ap.flags_next[c];
            if (fnext == 0 && !(fcur & F_SOLID_PREV)) {
                // a bulk cell: adj_bulk's
            } else if (fcur & F_SOLID) {            // obstacle at n: no adjoint
#pragma unroll
                for (int b = 0; b < Q; ++b) aout[(long long)b * C + c] = (A)0;
                if constexpr (!FIRST) static_cast<A *>(ap.rout)[c] = (A)0;
            } else {
                listed = true;
            }
        }
    }
    unsigned lm = 0;                                 // the warp's listed lanes
    if (warp < ADJ_BOUNDARY_THREADS / 32) {
        lm = __ballot_sync(0xffffffffu, listed);
        if (lane == 0) wcount[warp] = __popc(lm);
    }
    __syncthreads();
    if (listed) {
        int base = 0;
        for (int w = 0; w < warp; ++w) base += wcount[w];
        list[base + __popc(lm & ((1u << lane) - 1u))] = l;
    }
    int nlist = 0;
    for (int w = 0; w < ADJ_BOUNDARY_THREADS / 32; ++w) nlist += wcount[w];
    __syncthreads();
    // 2. a warp per listed cell, lane b = direction b
    const bool act = lane < Q;
    const int b = act ? lane : 0;
    const int bx = ex(b), by = ey(b), bz = ez(b), ob = opp(b);
    const A wb = (A)wgt(b);
    const A *__restrict__ ain = static_cast<const A *>(ap.ain);
    const A *__restrict__ rin = static_cast<const A *>(ap.rin);
    const T *__restrict__ G = static_cast<const T *>(ap.G);
    A wsum[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};        // this warp's body-kb terms, cell by cell
    for (int e = warp; e < nlist; e += ADJ_CUBE_WARPS) {
        int x, y, z;
        cube_cell(list[e], x, y, z);
        const long long c = ((long long)z * d.ny + y) * d.nx + x;
        const uint8_t fcur = ap.flags_cur[c], fnext = ap.flags_next[c];
        const bool fluid_next = !(fnext & F_SOLID);
        // density and velocity of step n from the post-collision populations
        const A gv = act ? (A)G[(long long)b * C + c] : (A)0;
        const A rho = (A)1 + warp_sum(gv);
        const A ir = (A)1 / rho;
        const A u0 = (warp_sum((A)bx * gv) - (A)(0.5 * dv.g[0])) * ir;
        const A u1 = (warp_sum((A)by * gv) - (A)(0.5 * dv.g[1])) * ir;
        const A u2 = (warp_sum((A)bz * gv) - (A)(0.5 * dv.g[2])) * ir;
        const A own = act ? ain[(long long)b * C + c] : (A)0;
        const A own_opp = __shfl_sync(0xffffffffu, own, ob);
        A a = own, crb = 0;
        A acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (act && b > 0) {
            const int zx = x + bx, zy = y + by, zz = z + bz;
            const bool wall = (!d.px && (zx < 0 || zx >= d.nx)) || (!d.py && (zy < 0 || zy >= d.ny)) ||
                              (!d.pz && (zz < 0 || zz >= d.nz));
            if (wall) {                              // Eq. 4 at step n+1
                a = own_opp;
            } else {
                const long long zc = ((long long)wrap_axis(zz, d.nz) * d.ny + wrap_axis(zy, d.ny)) * d.nx +
                                     wrap_axis(zx, d.nx);
                const uint8_t fzc = ap.flags_cur[zc];
                if (fzc & F_SOLID) {
                    // link (x, b) of step n: moving bounce-back of step n+1 and
                    // the momentum exchange of step n share u_w(x + e_b; S^n);
                    // the offset from the body centre in FP64, the terms in A
                    const int k = ap.bid_cur[zc];
                    const BodyState &sk = ap.body[k];
                    double od[3];
                    offset_from(d, sk, (double)zx, (double)zy, (double)zz, od);
                    const A o[3] = {(A)od[0], (A)od[1], (A)od[2]};
                    const A W[3] = {(A)sk.W[0], (A)sk.W[1], (A)sk.W[2]};
                    const A uw0 = (A)sk.V[0] + (W[1] * o[2] - W[2] * o[1]);
                    const A uw1 = (A)sk.V[1] + (W[2] * o[0] - W[0] * o[2]);
                    const A uw2 = (A)sk.V[2] + (W[0] * o[1] - W[1] * o[0]);
                    const A ua = -((A)bx * uw0 + (A)by * uw1 + (A)bz * uw2);     // e_-b . u_w
                    A mh = 0;
                    if constexpr (!FIRST) {
                        const double *fa = ap.fadj + 6 * k;
                        // (mid - X) x e_b, mid = x + e_b / 2 = (x + e_b) - e_b / 2
                        const A m0 = o[0] - (A)(0.5 * bx), m1 = o[1] - (A)(0.5 * by), m2 = o[2] - (A)(0.5 * bz);
                        const A t0 = m1 * (A)bz - m2 * (A)by, t1 = m2 * (A)bx - m0 * (A)bz, t2 = m0 * (A)by - m1 * (A)bx;
                        mh = (A)bx * (A)fa[0] + (A)by * (A)fa[1] + (A)bz * (A)fa[2] + t0 * (A)fa[3] + t1 * (A)fa[4] +
                             t2 * (A)fa[5];
                    }
                    const A wh = own_opp;
                    a = wh + (A)2 * mh;
                    crb = (A)6 * wb * ua * (wh + mh);
                    if (k == kb) {
                        const A sc = (A)6 * wb * rho * (wh + mh);
                        const A uh[3] = {-(A)bx * sc, -(A)by * sc, -(A)bz * sc};
                        adj_surface<A, A>(W, o, uh, acc);
                    }
                    // z uncovered at n+1: x (fluid at n and n+1) fed its density
                    if (!(ap.flags_next[zc] & F_SOLID) && fluid_next) crb += rin[zc];
                } else {
                    a = ain[(long long)b * C + zc];
                }
            }
        }
        a += warp_sum(crb);
        if constexpr (FIRST) {
            if (act) aout[(long long)b * C + c] = a;
        } else {
            // the transposed collision (collide_adjoint), its sums over the lanes
            const A om = (A)dv.omega;
            const A uu = u0 * u0 + u1 * u1 + u2 * u2;
            const A eu = (A)bx * u0 + (A)by * u1 + (A)bz * u2;
            const A wa = act ? wb * a : (A)0;
            const A cc = (A)3 + (A)9 * eu;
            const A sr = warp_sum(wa * ((A)1 + (A)3 * eu + (A)4.5 * eu * eu - (A)1.5 * uu));
            const A s0 = warp_sum(wa * (cc * (A)bx - (A)3 * u0));
            const A s1 = warp_sum(wa * (cc * (A)by - (A)3 * u1));
            const A s2 = warp_sum(wa * (cc * (A)bz - (A)3 * u2));
            A f0 = 0, f1 = 0, f2 = 0;
            if (dv.forced) {
                const A eg = (A)(bx * dv.g[0] + by * dv.g[1] + bz * dv.g[2]);
                f0 = warp_sum(wa * ((A)(-3.0 * dv.g[0]) + (A)9 * (A)bx * eg));
                f1 = warp_sum(wa * ((A)(-3.0 * dv.g[1]) + (A)9 * (A)by * eg));
                f2 = warp_sum(wa * ((A)(-3.0 * dv.g[2]) + (A)9 * (A)bz * eg));
            }
            const A kf = (A)1 - (A)0.5 * om;
            const A su0 = (om * rho * s0 + kf * f0) * ir, su1 = (om * rho * s1 + kf * f1) * ir,
                    su2 = (om * rho * s2 + kf * f2) * ir;
            const A base = om * sr - (su0 * u0 + su1 * u1 + su2 * u2);
            a = ((A)1 - om) * a + base + (A)bx * su0 + (A)by * su1 + (A)bz * su2;
            if (act) aout[(long long)b * C + c] = a;
            A rh_out = 0;
            if (fcur & F_SOLID_PREV) {
                // uncovered at n: P = f_eq(rho_avg, u_w(x; S^n)) of the body
                // that covered x at n-1, rho_avg over the neighbours fluid in
                // epochs n-1 and n (rho_avg = rho^n(x))
                bool nf = false;
                if (act && b > 0) {
                    const int nx_ = x + bx, ny_ = y + by, nz_ = z + bz;
                    const bool in = !((!d.px && (nx_ < 0 || nx_ >= d.nx)) || (!d.py && (ny_ < 0 || ny_ >= d.ny)) ||
                                      (!d.pz && (nz_ < 0 || nz_ >= d.nz)));
                    const long long nc = ((long long)wrap_axis(nz_, d.nz) * d.ny + wrap_axis(ny_, d.ny)) * d.nx +
                                         wrap_axis(nx_, d.nx);
                    nf = in && !(ap.flags_cur[nc] & (F_SOLID | F_SOLID_PREV));
                }
                const int cnt = __popc(__ballot_sync(0xffffffffu, nf));
                const int k = ap.bid_prev[c];
                if (k != NO_BODY) {
                    const BodyState &sk = ap.body[k];
                    double o[3], uw[3];
                    offset_from(d, sk, (double)x, (double)y, (double)z, o);
                    uw[0] = sk.V[0] + (sk.W[1] * o[2] - sk.W[2] * o[1]);
                    uw[1] = sk.V[1] + (sk.W[2] * o[0] - sk.W[0] * o[2]);
                    uw[2] = sk.V[2] + (sk.W[0] * o[1] - sk.W[1] * o[0]);
                    const double uuw = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
                    const double rho_d = (double)rho;
                    const double euw = bx * uw[0] + by * uw[1] + bz * uw[2];
                    const double pa = act ? (double)a * wgt(b) : 0.0;
                    const double cw = rho_d * (3.0 + 9.0 * euw);
                    const double rh = warp_sum(pa * (1.0 + 3.0 * euw + 4.5 * euw * euw - 1.5 * uuw));
                    const double uh[3] = {warp_sum(pa * (cw * bx - 3.0 * rho_d * uw[0])),
                                          warp_sum(pa * (cw * by - 3.0 * rho_d * uw[1])),
                                          warp_sum(pa * (cw * bz - 3.0 * rho_d * uw[2]))};
                    if (cnt) rh_out = (A)(rh / cnt);
                    if (k == kb && lane == 0) adj_surface<double, A>(sk.W, o, uh, acc);
                }
            }
            if (lane == 0) static_cast<A *>(ap.rout)[c] = rh_out;
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) wsum[i] += warp_sum(acc[i]);
    }
    // 3. the block's body-kb sums, warps in order
    if (lane == 0)
        for (int i = 0; i < 9; ++i) wacc[warp][i] = (double)wsum[i];
    __syncthreads();
    if (tid < 9) {
        double v = 0.0;
        for (int w = 0; w < ADJ_CUBE_WARPS; ++w) v += wacc[w][tid];
        ap.part[((long long)kb * ap.part_stride + blockIdx.x) * 9 + tid] = v;
    }
}

// ---- rigid-body step, reversed ------------------------------------------------
// Reverse of Algorithm 1 at step t with the state S^n and the hydrodynamic
// load fh^n of the tape:
//   V' = V + F / m, X' = X + V', W' = W + R diag(1/I) R^T T,
//   q' = normalise(q + (0, W') q / 2),
//   F = F_hydro + g vol + sum_d amp_d sin(omega_d t - phase_d) R a_d + springs.
// The terms that depend only on S^n and fh^n (R, F, R^T T, W', q', the drive
// sines, the spring geometry) are made for every step of a segment by
// adj_terms_kernel, a thread per body, drive term or spring and step; the
// serial kernel adj_integrate does the rest, linear in the adjoint.

// state-only terms of steps t0 .. t0 + L - 1: thread (j, i) with i < nb a
// body, then the drive terms, then the springs
__global__ void __launch_bounds__(ADJ_THREADS)
adj_terms_kernel(const Device dv, const BodyState *states, const double *fhs, long long t0, int L,
                 AdjBodyTerms *tb, AdjDriveTerms *td, AdjSpringTerms *ts) {
    const int per = dv.nb + dv.nd + dv.ns;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)L * per) return;
    const int j = (int)(id / per), i = (int)(id % per);
    const BodyState *S = states + (long long)j * dv.nb;
    const double tt = (double)(t0 + j);
    auto drive_value = [&](const DriveTerm &dt, double &sn_, double &cs) {
        sn_ = 0.0;
        cs = 0.0;
        if (tt < dt.t_on || tt >= dt.t_off) return 0.0;
        sincos(dt.omega * tt - dt.phase, &sn_, &cs);
        return dt.amp * sn_;
    };
    if (i < dv.nb) {
        const int b = i;
        const BodyProps pb = dv.props[b];
        const BodyState st = S[b];
        const double *fh = fhs + ((long long)j * dv.nb + b) * 6;
        double R[3][3];
        quat_to_matrix(st.q, R);
        // F: the hydrodynamic force, g times the volume, the body's drive
        // terms in term order and its springs in spring order (the order
        // of the forward's sums)
        double F[3];
        for (int a = 0; a < 3; ++a) F[a] = fh[a] + dv.g[a] * pb.volume;
        for (int k = pb.drive_first; k < pb.drive_first + pb.drive_count; ++k) {
            const DriveTerm dt = dv.drives[k];
            double sn_, cs;
            const double f = drive_value(dt, sn_, cs);
            for (int a = 0; a < 3; ++a)
                F[a] += f * (R[a][0] * dt.axis[0] + R[a][1] * dt.axis[1] + R[a][2] * dt.axis[2]);
        }
        for (int kk = pb.spring_first; kk < pb.spring_first + pb.spring_count; ++kk) {
            const int k = dv.spring_list[kk];
            const Spring sp_ = dv.springs[k];
            const BodyState si = S[sp_.i], sj = S[sp_.j];
            const double dd[3] = {si.X[0] - sj.X[0], si.X[1] - sj.X[1], si.X[2] - sj.X[2]};
            const double len = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
            const double inv_len = len > 0 ? 1.0 / len : 0.0;
            for (int a = 0; a < 3; ++a) {
                const double f = -sp_.k * (len - sp_.rest) * (dd[a] * inv_len) - sp_.gamma * (si.V[a] - sj.V[a]);
                F[a] += sp_.i == b ? f : -f;
            }
        }
        const double *T = fh + 3;
        double beta[3], W1[3];
        for (int a = 0; a < 3; ++a) beta[a] = R[0][a] * T[0] + R[1][a] * T[1] + R[2][a] * T[2];
        for (int a = 0; a < 3; ++a)
            W1[a] = st.W[a] + (R[a][0] * beta[0] * pb.inv_inertia[0] + R[a][1] * beta[1] * pb.inv_inertia[1] +
                               R[a][2] * beta[2] * pb.inv_inertia[2]);
        const double w = st.q[0], v0 = st.q[1], v1 = st.q[2], v2 = st.q[3];
        const double c0 = W1[1] * v2 - W1[2] * v1, c1 = W1[2] * v0 - W1[0] * v2, c2 = W1[0] * v1 - W1[1] * v0;
        const double q4[4] = {w - 0.5 * (W1[0] * v0 + W1[1] * v1 + W1[2] * v2), v0 + 0.5 * (w * W1[0] + c0),
                              v1 + 0.5 * (w * W1[1] + c1), v2 + 0.5 * (w * W1[2] + c2)};
        const double inv_nn = rsqrt(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
        AdjBodyTerms o;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) o.R[3 * r + c] = R[r][c];
        for (int a = 0; a < 3; ++a) {
            o.F[a] = F[a];
            o.beta[a] = beta[a];
            o.W1[a] = W1[a];
        }
        for (int a = 0; a < 4; ++a) o.q1[a] = q4[a] * inv_nn;
        o.inv_nn = inv_nn;
        tb[(long long)j * dv.nb + b] = o;
    } else if (i < dv.nb + dv.nd) {
        const int k = i - dv.nb;
        const DriveTerm dt = dv.drives[k];
        AdjDriveTerms o;
        o.f = drive_value(dt, o.sn, o.cs);
        double R[3][3];
        quat_to_matrix(S[dt.body].q, R);
        for (int a = 0; a < 3; ++a) o.aw[a] = R[a][0] * dt.axis[0] + R[a][1] * dt.axis[1] + R[a][2] * dt.axis[2];
        td[(long long)j * dv.nd + k] = o;
    } else {
        const int k = i - dv.nb - dv.nd;
        const Spring sp_ = dv.springs[k];
        const BodyState si = S[sp_.i], sj = S[sp_.j];
        const double dd[3] = {si.X[0] - sj.X[0], si.X[1] - sj.X[1], si.X[2] - sj.X[2]};
        const double len = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        AdjSpringTerms o;
        o.len = len;
        o.ratio = len > 0 ? (len - sp_.rest) / len : 0.0;
        for (int a = 0; a < 3; ++a) {
            o.dir[a] = len > 0 ? dd[a] / len : 0.0;
            o.dv[a] = si.V[a] - sj.V[a];
        }
        ts[(long long)j * dv.ns + k] = o;
    }
}

__device__ void adj_rot_matrix(const double q[4], const double Rh[3][3], double qh[4]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    qh[2] += -4 * y * Rh[0][0]; qh[3] += -4 * z * Rh[0][0];
    qh[1] += 2 * y * Rh[0][1]; qh[2] += 2 * x * Rh[0][1]; qh[0] += -2 * z * Rh[0][1]; qh[3] += -2 * w * Rh[0][1];
    qh[1] += 2 * z * Rh[0][2]; qh[3] += 2 * x * Rh[0][2]; qh[0] += 2 * y * Rh[0][2]; qh[2] += 2 * w * Rh[0][2];
    qh[1] += 2 * y * Rh[1][0]; qh[2] += 2 * x * Rh[1][0]; qh[0] += 2 * z * Rh[1][0]; qh[3] += 2 * w * Rh[1][0];
    qh[1] += -4 * x * Rh[1][1]; qh[3] += -4 * z * Rh[1][1];
    qh[2] += 2 * z * Rh[1][2]; qh[3] += 2 * y * Rh[1][2]; qh[0] += -2 * x * Rh[1][2]; qh[1] += -2 * w * Rh[1][2];
    qh[1] += 2 * z * Rh[2][0]; qh[3] += 2 * x * Rh[2][0]; qh[0] += -2 * y * Rh[2][0]; qh[2] += -2 * w * Rh[2][0];
    qh[2] += 2 * z * Rh[2][1]; qh[3] += 2 * y * Rh[2][1]; qh[0] += 2 * x * Rh[2][1]; qh[1] += 2 * w * Rh[2][1];
    qh[1] += -4 * x * Rh[2][2]; qh[2] += -4 * y * Rh[2][2];
}

// One block.  Sh^{n+1} = sa_next + the cell sums of reverse step n+1
// (part, in block order); then the reverse step with the state-only terms
// of step n.  Writes Sh^n (rigid-body part plus the lever-arm term Th x
// F_hydro of the torque sum) to sa_cur, (Fh, Th) to fadj and adds
// dJ/dtheta.
__global__ void __launch_bounds__(ADJ_THREADS) adj_integrate_kernel(const Device dv, const AdjBody ab) {
    const int nb = dv.nb;
    const BodyState *S = ab.state;
    // 1. complete Sh^{n+1}: warp w adds body b's block sums, lanes over the
    //    blocks, then a fixed shuffle tree
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int b = warp; b < nb; b += nwarps) {
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = lane; k < ab.part_count; k += 32) {
            const double *p = ab.part + ((long long)b * ab.part_stride + k) * 9;
#pragma unroll
            for (int i = 0; i < 9; ++i) acc[i] += p[i];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
        }
        if (lane == 0) {
            double *sn = ab.sa_next + 13 * b;
            for (int i = 0; i < 3; ++i) { sn[i] += acc[i]; sn[7 + i] += acc[3 + i]; sn[10 + i] += acc[6 + i]; }
        }
    }
    __syncthreads();
    // 2. per body: Euler step and rotation update, reversed
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const BodyProps pb = dv.props[b];
        const BodyState s = S[b];
        const AdjBodyTerms tm = ab.tb[b];
        const double *sn = ab.sa_next + 13 * b;
        const double *fh = ab.fh + 6 * b;
        const double *T = fh + 3;
        double R[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) R[r][c] = tm.R[3 * r + c];
        const double *beta = tm.beta, *W1 = tm.W1, *q1 = tm.q1;
        const double w = s.q[0], v0 = s.q[1], v1 = s.q[2], v2 = s.q[3];
        const double inv_nn = tm.inv_nn;
        double dot = 0.0, qh4[4];
        for (int i = 0; i < 4; ++i) dot += q1[i] * sn[3 + i];
        for (int i = 0; i < 4; ++i) qh4[i] = (sn[3 + i] - q1[i] * dot) * inv_nn;
        double out[13];
        const double qv[3] = {qh4[1], qh4[2], qh4[3]};
        out[3] = qh4[0] + 0.5 * (qv[0] * W1[0] + qv[1] * W1[1] + qv[2] * W1[2]);
        const double t1[3] = {qv[1] * W1[2] - qv[2] * W1[1], qv[2] * W1[0] - qv[0] * W1[2], qv[0] * W1[1] - qv[1] * W1[0]};
        const double vv[3] = {v0, v1, v2};
        for (int i = 0; i < 3; ++i) out[4 + i] = qv[i] - 0.5 * qh4[0] * W1[i] + 0.5 * t1[i];
        const double t2[3] = {vv[1] * qv[2] - vv[2] * qv[1], vv[2] * qv[0] - vv[0] * qv[2], vv[0] * qv[1] - vv[1] * qv[0]};
        double Wh1[3];
        for (int i = 0; i < 3; ++i) Wh1[i] = sn[10 + i] - 0.5 * qh4[0] * vv[i] + 0.5 * w * qv[i] + 0.5 * t2[i];
        double alpha[3];
        for (int i = 0; i < 3; ++i) alpha[i] = R[0][i] * Wh1[0] + R[1][i] * Wh1[1] + R[2][i] * Wh1[2];
        double Th[3];
        for (int i = 0; i < 3; ++i) {
            out[10 + i] = Wh1[i];
            Th[i] = R[i][0] * alpha[0] * pb.inv_inertia[0] + R[i][1] * alpha[1] * pb.inv_inertia[1] +
                    R[i][2] * alpha[2] * pb.inv_inertia[2];
            ab.grad_body[5 * b + 1 + i] += -beta[i] * alpha[i] * pb.inv_inertia[i] * pb.inv_inertia[i];
        }
        double Rh[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Rh[i][j] = Wh1[i] * beta[j] * pb.inv_inertia[j] + T[i] * alpha[j] * pb.inv_inertia[j];
        double Fh[3], F2 = 0.0, gv = 0.0;
        for (int i = 0; i < 3; ++i) {
            const double vh1 = sn[7 + i] + sn[i];
            out[i] = sn[i];
            out[7 + i] = vh1;
            Fh[i] = vh1 * pb.inv_m;
            F2 += vh1 * tm.F[i];
            gv += dv.g[i] * Fh[i];
        }
        ab.grad_body[5 * b] += -F2 * pb.inv_m * pb.inv_m;
        ab.grad_body[5 * b + 4] += gv;
        // lever arm of the torque sum: T = sum (mid - X) x F_link
        out[0] += Th[1] * fh[2] - Th[2] * fh[1];
        out[1] += Th[2] * fh[0] - Th[0] * fh[2];
        out[2] += Th[0] * fh[1] - Th[1] * fh[0];
        // drive terms of this body (F = f R a: dF_i / dR_ij = f a_j)
        for (int k = pb.drive_first; k < pb.drive_first + pb.drive_count; ++k) {
            const double f = ab.td[k].f;                 // zero outside the drive window
            const double *a = dv.drives[k].axis;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Rh[i][j] += f * Fh[i] * a[j];
        }
        double qh[4] = {0, 0, 0, 0};
        adj_rot_matrix(s.q, Rh, qh);
        for (int i = 0; i < 4; ++i) out[3 + i] += qh[i];
        double *sc = ab.sa_cur + 13 * b;
        for (int i = 0; i < 13; ++i) sc[i] = out[i];
        for (int i = 0; i < 3; ++i) { ab.fadj[6 * b + i] = Fh[i]; ab.fadj[6 * b + 3 + i] = Th[i]; }
    }
    __syncthreads();
    // 3. drive-term and spring gradients (one thread per term), then the
    //    spring terms of each body's adjoint (thread b, its springs in order)
    const double tt = (double)ab.t;
    for (int k = threadIdx.x; k < dv.nd; k += blockDim.x) {
        const DriveTerm dt = dv.drives[k];
        if (tt < dt.t_on || tt >= dt.t_off) continue;
        const AdjDriveTerms tdk = ab.td[k];
        const double *fa = ab.fadj + 6 * dt.body;
        const double proj = fa[0] * tdk.aw[0] + fa[1] * tdk.aw[1] + fa[2] * tdk.aw[2];
        ab.grad_drive[2 * k] += tdk.sn * proj;
        ab.grad_drive[2 * k + 1] += -dt.amp * tdk.cs * proj;
    }
    for (int k = threadIdx.x; k < dv.ns; k += blockDim.x) {
        const Spring sp_ = dv.springs[k];
        const AdjSpringTerms tsk = ab.ts[k];
        double fh[3], dvv = 0.0, fd = 0.0;
        for (int i = 0; i < 3; ++i) {
            fh[i] = ab.fadj[6 * sp_.i + i] - ab.fadj[6 * sp_.j + i];
            dvv += fh[i] * tsk.dv[i];
        }
        ab.grad_spring[3 * k + 2] += -dvv;
        if (tsk.len > 0) {
            for (int i = 0; i < 3; ++i) fd += fh[i] * tsk.dir[i];
            ab.grad_spring[3 * k] += -(tsk.len - sp_.rest) * fd;
            ab.grad_spring[3 * k + 1] += sp_.k * fd;
        }
    }
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const BodyProps pb = dv.props[b];
        double *sc = ab.sa_cur + 13 * b;
        for (int kk = pb.spring_first; kk < pb.spring_first + pb.spring_count; ++kk) {
            const int k = dv.spring_list[kk];
            const Spring sp_ = dv.springs[k];
            const AdjSpringTerms tsk = ab.ts[k];
            const double sign = sp_.i == b ? 1.0 : -1.0;
            double fh[3], fd = 0.0;
            for (int i = 0; i < 3; ++i) fh[i] = ab.fadj[6 * sp_.i + i] - ab.fadj[6 * sp_.j + i];
            for (int i = 0; i < 3; ++i) sc[7 + i] += -sign * sp_.gamma * fh[i];
            if (!(tsk.len > 0)) continue;
            for (int i = 0; i < 3; ++i) fd += fh[i] * tsk.dir[i];
            for (int i = 0; i < 3; ++i)
                sc[i] += sign * (-sp_.k * (fd * tsk.dir[i] + tsk.ratio * (fh[i] - fd * tsk.dir[i])));
        }
    }
}

// sa[b] += the cell sums part[b][0..count) (the last reverse step)
__global__ void adj_reduce_kernel(int nb, const double *part, int stride, int count, double *sa) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double *s = sa + 13 * b;
    for (int k = 0; k < count; ++k) {
        const double *p = part + ((long long)b * stride + k) * 9;
        for (int i = 0; i < 3; ++i) { s[i] += p[i]; s[7 + i] += p[3 + i]; s[10 + i] += p[6 + i]; }
    }
}

template <typename A, typename T, bool FIRST>
void launch_bulk_cells(const Device &dv, const AdjPtrs &ap, cudaStream_t s) {
    const dim3 blk(128, 2);
    const dim3 grid((dv.dom.nx + 127) / 128, (dv.dom.ny + 1) / 2, dv.dom.nz);
    adj_bulk_kernel<A, T, FIRST><<<grid, blk, 0, s>>>(dv, ap);
}

template <typename A, typename T, bool FIRST>
void launch_boundary_cells(const Device &dv, const AdjPtrs &ap, cudaStream_t s) {
    if (dv.nb > 0)
        adj_cube_kernel<A, T, FIRST><<<dim3(ap.part_stride, dv.nb), 32 * ADJ_CUBE_WARPS, 0, s>>>(dv, ap);
    if (!(dv.dom.px && dv.dom.py && dv.dom.pz)) {
        const long long nx = dv.dom.nx, ny = dv.dom.ny, nz = dv.dom.nz;
        const long long area = std::max(ny * nz, std::max(nx * nz, nx * ny));
        adj_wall_kernel<A, T, FIRST>
            <<<dim3((unsigned)((area + ADJ_BOUNDARY_THREADS - 1) / ADJ_BOUNDARY_THREADS), 6), ADJ_BOUNDARY_THREADS, 0,
               s>>>(dv, ap);
    }
}

}  // namespace

int adjoint_part_stride(const Device &dv) {
    const long long side = dv.remap_side;
    return (int)((side * side * side + ADJ_BOUNDARY_THREADS - 1) / ADJ_BOUNDARY_THREADS);
}

void launch_adj_integrate(const Device &dv, const AdjBody &ab, cudaStream_t s) {
    adj_integrate_kernel<<<1, ADJ_THREADS, 0, s>>>(dv, ab);
}

void launch_adj_terms(const Device &dv, const BodyState *states, const double *fh, long long t0, int L,
                      AdjBodyTerms *tb, AdjDriveTerms *td, AdjSpringTerms *ts, cudaStream_t s) {
    const long long n = (long long)L * (dv.nb + dv.nd + dv.ns);
    if (n > 0)
        adj_terms_kernel<<<(unsigned)((n + ADJ_THREADS - 1) / ADJ_THREADS), ADJ_THREADS, 0, s>>>(dv, states, fh, t0, L,
                                                                                                 tb, td, ts);
}

void launch_adj_bulk(const Device &dv, const AdjPtrs &ap, bool first, cudaStream_t s) {
    if (dv.precision == LBM_PREC_F64) {
        if (first) launch_bulk_cells<double, double, true>(dv, ap, s);
        else launch_bulk_cells<double, double, false>(dv, ap, s);
    } else {
        if (first) launch_bulk_cells<float, float, true>(dv, ap, s);
        else launch_bulk_cells<float, float, false>(dv, ap, s);
    }
}

void launch_adj_boundary(const Device &dv, const AdjPtrs &ap, bool first, cudaStream_t s) {
    if (dv.precision == LBM_PREC_F64) {
        if (first) launch_boundary_cells<double, double, true>(dv, ap, s);
        else launch_boundary_cells<double, double, false>(dv, ap, s);
    } else {
        if (first) launch_boundary_cells<float, float, true>(dv, ap, s);
        else launch_boundary_cells<float, float, false>(dv, ap, s);
    }
}

void launch_adj_reduce(const Device &dv, const double *part, int stride, int count, double *sa, cudaStream_t s) {
    if (dv.nb > 0) adj_reduce_kernel<<<(dv.nb + 127) / 128, 128, 0, s>>>(dv.nb, part, stride, count, sa);
}

}  // namespace lbm
