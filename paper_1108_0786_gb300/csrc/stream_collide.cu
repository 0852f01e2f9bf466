// stream_collide.cu -- the fused D3Q19 stream + bounce-back + refill + LBGK
// kernel of one coupled step (Eq. 1-4 of the paper and the moving-wall rule
// and reconstruction of Sec. 2.3).  This kernel moves >99% of the bytes of a
// step and is bound by HBM bandwidth: per cell it reads 19 populations and a
// flag byte and writes 19 populations (2 * 19 * sizeof(T) + 1 bytes).
//
// Pull scheme, two grids (src = step n-1, dst = step n).  For a cell x that
// is fluid at n:
//   - fast path (flag byte 0): f_b(x) = f~_b(x - e_b) for all 19 b;
//   - x was solid at n-1 (uncovered): f_b = f_eq(rho_avg, u_w(x; state n)),
//     rho_avg the mean density of the D3Q19 neighbours that are fluid in both
//     epochs (1 if none);
//   - otherwise, for each b whose source y = x - e_b lies beyond a no-slip
//     wall: f_b = f~_{-b}(x) (Eq. 4); if y was solid at n-1:
//     f_b = f~_{-b}(x) + 6 w_b rho(x) e_b . u_w(y; state n-1), rho(x) the
//     density of x at n-1;
// then rho, u (Guo: u = (sum e f + g/2) / rho), LBGK relaxation to the
// second-order equilibrium plus Guo's forcing term, and the store of
// f~(x, n).  Solid cells store deviation 0.
//
// Populations are stored as deviations delta = f - w from the rest
// equilibrium, so that FP32 and 16-bit storage keep the small velocity
// signal; the collision runs in FP64 for FP64 storage and in FP32 otherwise.
//
// Memory access: each thread handles V consecutive cells of an x row; every
// population is fetched as one aligned V-wide vector per thread (coalesced
// 128-bit loads for V * sizeof(T) = 16), and the +-1 x shift of the pull is
// completed with a warp shuffle from the neighbouring lane (a scalar load at
// row and warp ends).  Every population byte is read once and written once.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int SC_THREADS = 128;

template <int BYTES> struct Raw;
template <> struct Raw<2> { using type = unsigned short; };
template <> struct Raw<4> { using type = unsigned int; };
template <> struct Raw<8> { using type = uint2; };
template <> struct Raw<16> { using type = uint4; };

// storage codecs: deviation value <-> compute type
template <typename T> struct Codec;
template <> struct Codec<double> {
    using C = double;
    __device__ static C ld(double v, float) { return v; }
    __device__ static double st(C v, float) { return v; }
};
template <> struct Codec<float> {
    using C = float;
    __device__ static C ld(float v, float) { return v; }
    __device__ static float st(C v, float) { return v; }
};
template <> struct Codec<__half> {
    using C = float;
    __device__ static C ld(__half v, float inv_scale) { return __half2float(v) * inv_scale; }
    __device__ static __half st(C v, float scale) { return __float2half_rn(v * scale); }
};
template <> struct Codec<__nv_bfloat16> {
    using C = float;
    __device__ static C ld(__nv_bfloat16 v, float) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 st(C v, float) { return __float2bfloat16_rn(v); }
};

template <typename T, int V>
__device__ __forceinline__ void load_vec(const T *p, T (&out)[V]) {
    using R = typename Raw<sizeof(T) * V>::type;
    R r = __ldg(reinterpret_cast<const R *>(p));
    memcpy(&out, &r, sizeof(R));
}

template <typename T, int V>
__device__ __forceinline__ void store_vec(T *p, const T (&in)[V]) {
    using R = typename Raw<sizeof(T) * V>::type;
    R r;
    memcpy(&r, &in, sizeof(R));
    *reinterpret_cast<R *>(p) = r;
}

template <typename T>
__device__ __forceinline__ T shfl_up1(T v) {
    if constexpr (sizeof(T) == 8) {
        unsigned long long b;
        memcpy(&b, &v, 8);
        b = __shfl_up_sync(0xffffffffu, b, 1);
        memcpy(&v, &b, 8);
    } else {
        unsigned int b = 0;
        memcpy(&b, &v, sizeof(T));
        b = __shfl_up_sync(0xffffffffu, b, 1);
        memcpy(&v, &b, sizeof(T));
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T shfl_down1(T v) {
    if constexpr (sizeof(T) == 8) {
        unsigned long long b;
        memcpy(&b, &v, 8);
        b = __shfl_down_sync(0xffffffffu, b, 1);
        memcpy(&v, &b, 8);
    } else {
        unsigned int b = 0;
        memcpy(&b, &v, sizeof(T));
        b = __shfl_down_sync(0xffffffffu, b, 1);
        memcpy(&v, &b, sizeof(T));
    }
    return v;
}

template <typename T, int V>
__global__ void __launch_bounds__(SC_THREADS)
stream_collide_kernel(const Device dv, const StepPtrs sp) {
    using Cd = typename Codec<T>::C;
    const Domain d = dv.dom;
    const long long C = d.C;
    const int nxq = d.nx / V;
    const long long nq = C / V;
    long long q = (long long)blockIdx.x * SC_THREADS + threadIdx.x;
    const bool active = q < nq;
    if (!active) q = nq - 1;             // keep the whole warp in the shuffles
    const int lane = threadIdx.x & 31;
    const int x0 = (int)(q % nxq) * V;
    const long long row = q / nxq;
    const int y = (int)(row % d.ny);
    const int z = (int)(row / d.ny);
    const int ym = y == 0 ? d.ny - 1 : y - 1, yp = y == d.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? d.nz - 1 : z - 1, zp = z == d.nz - 1 ? 0 : z + 1;
    const long long c0 = row * d.nx + x0;
    const T *__restrict__ src = static_cast<const T *>(sp.src);
    T *__restrict__ dst = static_cast<T *>(sp.dst);
    const float inv_scale = dv.f16_inv_scale, scale = dv.f16_scale;

    uint8_t fl[V];
    {
        uint8_t raw[V];
        if constexpr (V == 1) {
            raw[0] = sp.flags_cur[c0];
        } else {
            load_vec<uint8_t, V>(sp.flags_cur + c0, raw);
        }
#pragma unroll
        for (int i = 0; i < V; ++i) fl[i] = raw[i];
    }

    // ---- pull: f_b(x) = f~_b(x - e_b) -----------------------------------
    Cd f[Q][V];
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        const int ys = ey(b) > 0 ? ym : (ey(b) < 0 ? yp : y);
        const int zs = ez(b) > 0 ? zm : (ez(b) < 0 ? zp : z);
        const T *plane = src + (long long)b * C + ((long long)zs * d.ny + ys) * d.nx;
        T A[V];
        load_vec<T, V>(plane + x0, A);
        if (ex(b) == 0) {
#pragma unroll
            for (int i = 0; i < V; ++i) f[b][i] = Codec<T>::ld(A[i], inv_scale);
        } else if (ex(b) > 0) {          // source at x - 1
            T left = shfl_up1(A[V - 1]);
            if (lane == 0 || x0 == 0) left = plane[x0 == 0 ? d.nx - 1 : x0 - 1];
            f[b][0] = Codec<T>::ld(left, inv_scale);
#pragma unroll
            for (int i = 1; i < V; ++i) f[b][i] = Codec<T>::ld(A[i - 1], inv_scale);
        } else {                          // source at x + 1
            T right = shfl_down1(A[0]);
            if (lane == 31 || x0 + V == d.nx) right = plane[x0 + V == d.nx ? 0 : x0 + V];
#pragma unroll
            for (int i = 0; i < V - 1; ++i) f[b][i] = Codec<T>::ld(A[i + 1], inv_scale);
            f[b][V - 1] = Codec<T>::ld(right, inv_scale);
        }
    }

    // ---- cells next to obstacles or walls ----------------------------------
    unsigned solid_mask = 0;
    unsigned any = 0;
#pragma unroll
    for (int i = 0; i < V; ++i) any |= fl[i];
    if (any) {
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const uint8_t fc = fl[i];
            if (fc == 0) continue;
            if (fc & F_SOLID) {
                solid_mask |= 1u << i;
                continue;
            }
            const int xc = x0 + i;
            const long long c = c0 + i;
            if (fc & F_SOLID_PREV) {
                // uncovered cell: f = f_eq(rho_avg, u_w(x)) with the state of step n
                double sum = 0.0;
                int cnt = 0;
                for (int a = 1; a < Q; ++a) {
                    int nx_ = xc + ex(a), ny_ = y + ey(a), nz_ = z + ez(a);
                    if ((!d.px && (nx_ < 0 || nx_ >= d.nx)) || (!d.py && (ny_ < 0 || ny_ >= d.ny)) ||
                        (!d.pz && (nz_ < 0 || nz_ >= d.nz)))
                        continue;
                    nx_ = wrap_axis(nx_, d.nx); ny_ = wrap_axis(ny_, d.ny); nz_ = wrap_axis(nz_, d.nz);
                    const long long yc = ((long long)nz_ * d.ny + ny_) * d.nx + nx_;
                    if (sp.flags_cur[yc] & (F_SOLID | F_SOLID_PREV)) continue;
                    Cd drho = 0;
                    for (int bb = 0; bb < Q; ++bb) drho += Codec<T>::ld(src[bb * C + yc], inv_scale);
                    sum += 1.0 + (double)drho;
                    ++cnt;
                }
                const double rho = cnt ? sum / cnt : 1.0;
                const int k = sp.bid_prev[c];
                double u[3] = {0.0, 0.0, 0.0};
                if (k != NO_BODY) surface_velocity(d, sp.body_cur[k], xc, y, z, u);
                const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
                for (int b = 0; b < Q; ++b) {
                    const double eu = ex(b) * u[0] + ey(b) * u[1] + ez(b) * u[2];
                    f[b][i] = (Cd)(wgt(b) * (rho - 1.0) + wgt(b) * rho * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
                }
            } else {
                // bounce-back at walls (Eq. 4) and at obstacles of step n-1
                Cd rho_x = -1;
#pragma unroll
                for (int b = 1; b < Q; ++b) {
                    int sx = xc - ex(b), sy = y - ey(b), sz = z - ez(b);
                    const Cd back = Codec<T>::ld(src[(long long)opp(b) * C + c], inv_scale);
                    if ((!d.px && (sx < 0 || sx >= d.nx)) || (!d.py && (sy < 0 || sy >= d.ny)) ||
                        (!d.pz && (sz < 0 || sz >= d.nz))) {
                        f[b][i] = back;
                        continue;
                    }
                    sx = wrap_axis(sx, d.nx); sy = wrap_axis(sy, d.ny); sz = wrap_axis(sz, d.nz);
                    const long long sc = ((long long)sz * d.ny + sy) * d.nx + sx;
                    if (!(sp.flags_prev[sc] & F_SOLID)) continue;
                    if (rho_x < 0) {
                        Cd drho = 0;
                        for (int a = 0; a < Q; ++a) drho += Codec<T>::ld(src[(long long)a * C + c], inv_scale);
                        rho_x = (Cd)1 + drho;
                    }
                    const int k = sp.bid_prev[sc];
                    double u[3] = {0.0, 0.0, 0.0};
                    if (k != NO_BODY) surface_velocity(d, sp.body_prev[k], sx, sy, sz, u);
                    const Cd eu = (Cd)(ex(b) * u[0] + ey(b) * u[1] + ez(b) * u[2]);
                    f[b][i] = back + (Cd)(6.0 * wgt(b)) * rho_x * eu;
                }
            }
        }
    }

    // ---- LBGK collision (Eq. 2) with Guo's forcing ---------------------------
    Cd rho[V], drho[V], ux[V], uy[V], uz[V], usq[V];
#pragma unroll
    for (int i = 0; i < V; ++i) {
        Cd s = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            s += f[b][i];
            if (ex(b)) jx += ex(b) > 0 ? f[b][i] : -f[b][i];
            if (ey(b)) jy += ey(b) > 0 ? f[b][i] : -f[b][i];
            if (ez(b)) jz += ez(b) > 0 ? f[b][i] : -f[b][i];
        }
        drho[i] = s;
        rho[i] = (Cd)1 + s;
        const Cd inv = (Cd)1 / rho[i];
        ux[i] = (jx + (Cd)(0.5 * dv.g[0])) * inv;
        uy[i] = (jy + (Cd)(0.5 * dv.g[1])) * inv;
        uz[i] = (jz + (Cd)(0.5 * dv.g[2])) * inv;
        usq[i] = ux[i] * ux[i] + uy[i] * uy[i] + uz[i] * uz[i];
    }
    const Cd om = (Cd)dv.omega;
    const Cd guo = (Cd)(1.0 - 0.5 * dv.omega);
    const Cd gx = (Cd)dv.g[0], gy = (Cd)dv.g[1], gz = (Cd)dv.g[2];
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        const Cd w = (Cd)wgt(b);
        T out[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const Cd eu = (Cd)ex(b) * ux[i] + (Cd)ey(b) * uy[i] + (Cd)ez(b) * uz[i];
            const Cd deq = w * (drho[i] + rho[i] * ((Cd)3 * eu + (Cd)4.5 * eu * eu - (Cd)1.5 * usq[i]));
            Cd o = f[b][i] - om * (f[b][i] - deq);
            if (dv.forced) {
                const Cd eg = (Cd)ex(b) * gx + (Cd)ey(b) * gy + (Cd)ez(b) * gz;
                const Cd ug = ux[i] * gx + uy[i] * gy + uz[i] * gz;
                o += guo * w * ((Cd)3 * (eg - ug) + (Cd)9 * eu * eg);
            }
            if (solid_mask & (1u << i)) o = 0;
            out[i] = Codec<T>::st(o, scale);
        }
        if (active) store_vec<T, V>(dst + (long long)b * C + c0, out);
    }
}

template <typename T, int V>
void launch_typed(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const long long nq = dv.dom.C / V;
    const unsigned blocks = (unsigned)((nq + SC_THREADS - 1) / SC_THREADS);
    stream_collide_kernel<T, V><<<blocks, SC_THREADS, 0, s>>>(dv, sp);
}

}  // namespace

int stream_collide_vector_width(const Device &dv) {
    const int nx = dv.dom.nx;
    switch (dv.precision) {
    case 0: return nx % 2 == 0 ? 2 : 1;               // FP64: 16-byte vectors
    case 1: return nx % 4 == 0 ? 4 : 1;               // FP32
    default: return nx % 8 == 0 ? 8 : 1;              // FP16 / BF16
    }
}

void launch_stream_collide(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const int v = stream_collide_vector_width(dv);
    switch (dv.precision) {
    case 0:
        if (v == 2) launch_typed<double, 2>(dv, sp, s); else launch_typed<double, 1>(dv, sp, s);
        break;
    case 1:
        if (v == 4) launch_typed<float, 4>(dv, sp, s); else launch_typed<float, 1>(dv, sp, s);
        break;
    case 2:
        if (v == 8) launch_typed<__half, 8>(dv, sp, s); else launch_typed<__half, 1>(dv, sp, s);
        break;
    default:
        if (v == 8) launch_typed<__nv_bfloat16, 8>(dv, sp, s); else launch_typed<__nv_bfloat16, 1>(dv, sp, s);
        break;
    }
}

}  // namespace lbm
