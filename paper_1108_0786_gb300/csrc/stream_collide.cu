// stream_collide.cu -- the fused D3Q19 stream + bounce-back + refill + LBGK
// update of one coupled step (Eq. 1-4 of the paper, and the moving-wall rule
// and the reconstruction of uncovered cells of Sec. 2.3).  It moves >99% of
// the bytes of a step and is bound by HBM bandwidth: per cell it reads 19
// populations and a flag byte and writes 19 populations
// (2 * 19 * sizeof(T) + 1 bytes).
//
// Two kernels write the populations of step n (pull scheme, two grids: src =
// step n-1, dst = step n):
//
//  bulk      every cell with a zero flag byte: f_b(x) = f~_b(x - e_b) for
//            all 19 b, LBGK relaxation to the second-order equilibrium with
//            Guo's forcing, store; solid cells store deviation 0.  No
//            data-dependent paths, so the kernel stays small and light.
//  boundary  only the fluid cells whose flag byte is non-zero (they lie in
//            the cubes around the bodies or on wall faces; the bulk kernel
//            leaves them alone, so the two kernels may run concurrently):
//              - x was solid at n-1 (uncovered): f_b = f_eq(rho_avg, u_w(x)),
//                rho_avg the mean density of the D3Q19 neighbours that are
//                fluid in both epochs (1 if none), u_w at the state of step n;
//              - otherwise per b: if the source y = x - e_b lies beyond a
//                no-slip wall, f_b = f~_{-b}(x) (Eq. 4); if y was solid at
//                n-1, f_b = f~_{-b}(x) + 6 w_b rho(x) e_b . u_w(y) with rho(x)
//                the density of x at n-1 and u_w at the state of step n-1;
//            then the same LBGK collision.
//
// Populations are stored as deviations delta = f - w from the rest
// equilibrium (16-bit formats: FP16 scaled by 2^10, BF16 unscaled), so the
// small velocity signal survives FP32 and 16-bit storage; the collision runs
// in FP64 for FP64 storage and in FP32 otherwise.
//
// Memory access of the bulk kernel: thread (tx, ty) of block (bx, by, z)
// handles V consecutive cells of row (y, z); each population is fetched as
// one aligned V-wide vector, and the +-1 x shift of the pull is completed
// with a warp shuffle from the neighbouring lane (a scalar load at row and
// warp ends).  Every population byte is read once and written once.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

template <int BYTES> struct Raw;
template <> struct Raw<1> { using type = unsigned char; };
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
__device__ __forceinline__ T shfl(T v, int delta, bool up) {
    if constexpr (sizeof(T) == 8) {
        unsigned long long b;
        memcpy(&b, &v, 8);
        b = up ? __shfl_up_sync(0xffffffffu, b, delta) : __shfl_down_sync(0xffffffffu, b, delta);
        memcpy(&v, &b, 8);
    } else {
        unsigned int b = 0;
        memcpy(&b, &v, sizeof(T));
        b = up ? __shfl_up_sync(0xffffffffu, b, delta) : __shfl_down_sync(0xffffffffu, b, delta);
        memcpy(&v, &b, sizeof(T));
    }
    return v;
}

// LBGK collision of one cell in place (deviation form):
//   drho = sum delta, rho = 1 + drho, u = (sum e delta + g/2) / rho,
//   delta_eq_b = w_b (drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)),
//   delta~_b = delta_b + (delta_eq_b - delta_b) / tau
//              + (1 - 1/(2 tau)) w_b (3 (e_b - u) . g + 9 (e_b . u)(e_b . g)).
// In exact arithmetic the increments delta~_b - delta_b carry zero mass and
// momentum exactly g.  With FP32 storage the rounded velocity that enters the
// equilibrium would make each collision a small momentum source in every
// cell, constant in a steady flow, and the slow viscous mode of a channel
// integrates it into a ~1e-5 velocity error.  The FP32 update therefore sums
// mass and momentum of the increments (small numbers, so the sums are
// accurate) and moves the defect to the +-x, +-y, +-z pairs and the rest
// population: only the value-dependent rounding of the final additions
// remains.  FP64 keeps the plain update, as do the 16-bit formats, whose
// storage rounding (2^-9 .. 2^-11 relative) dwarfs this effect.
// CLOSE selects that closure.  PAIRED evaluates opposite directions (b, b + 1)
// together: they share w, (e.u)^2 and e.g up to sign, so
// deq = w (base + 4.5 rho (e.u)^2 +- 3 rho e.u) saves a fifth of the
// arithmetic; otherwise one direction at a time.  Both forms compute the
// same expression (FP32 takes the paired one; the 16-bit kernels schedule
// the per-direction one better).
// explicit fused multiply-adds: this file is compiled without implicit
// contraction (-fmad=false), so every kernel that runs a cell's arithmetic --
// any launch shape, the batched ensemble kernels, the boundary kernel --
// rounds it identically, and the FMAs the collision wants are spelled out
__device__ __forceinline__ float mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return __fma_rn(a, b, c); }

// e_b . (x, y, z) over the non-zero components of e_b only, in x, y, z
// order (a zero component would still cost a multiply and an add: 0 * z is
// not 0 for every z)
template <typename R>
__device__ __forceinline__ R edot(int b, R x, R y, R z) {
    R r = 0;
    bool any = false;
    if (ex(b)) { r = ex(b) > 0 ? x : -x; any = true; }
    if (ey(b)) { const R t = ey(b) > 0 ? y : -y; r = any ? r + t : t; any = true; }
    if (ez(b)) { const R t = ez(b) > 0 ? z : -z; r = any ? r + t : t; }
    return r;
}

template <typename Cd, bool CLOSE, bool PAIRED = CLOSE>
__device__ __forceinline__ void collide(Cd (&f)[Q], const Device &dv) {
    Cd s = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        s += f[b];
        if (ex(b)) jx += ex(b) > 0 ? f[b] : -f[b];
        if (ey(b)) jy += ey(b) > 0 ? f[b] : -f[b];
        if (ez(b)) jz += ez(b) > 0 ? f[b] : -f[b];
    }
    const Cd rho = (Cd)1 + s;
    const Cd inv = (Cd)1 / rho;
    // FP32 takes the parameters rounded once on the host (no FP64 conversion per cell)
    const bool f32 = sizeof(Cd) == 4;
    const Cd gx = f32 ? (Cd)dv.g_f[0] : (Cd)dv.g[0], gy = f32 ? (Cd)dv.g_f[1] : (Cd)dv.g[1],
             gz = f32 ? (Cd)dv.g_f[2] : (Cd)dv.g[2];
    const Cd ux = mad((Cd)0.5, gx, jx) * inv, uy = mad((Cd)0.5, gy, jy) * inv, uz = mad((Cd)0.5, gz, jz) * inv;
    const Cd usq = mad(ux, ux, mad(uy, uy, uz * uz));
    const Cd om = f32 ? (Cd)dv.omega_f : (Cd)dv.omega;
    const Cd guo = f32 ? (Cd)dv.guo_f : (Cd)(1.0 - 0.5 * dv.omega);
    const Cd ug = mad(ux, gx, mad(uy, gy, uz * gz));
    const Cd base = mad((Cd)(-1.5) * rho, usq, s);     // deviation of f_eq without the e.u terms, over w
    Cd m = 0, px = 0, py = 0, pz = 0;
    // one relaxation: the increment of direction b towards deq (+ Guo's term
    // gt), kept for the conservation closure or applied directly
    auto relax = [&](int b, Cd deq, Cd gt) {
        if constexpr (CLOSE) {
            const Cd d = dv.forced ? mad(om, deq - f[b], gt) : om * (deq - f[b]);
            m += d;
            if (ex(b)) px += ex(b) > 0 ? d : -d;
            if (ey(b)) py += ey(b) > 0 ? d : -d;
            if (ez(b)) pz += ez(b) > 0 ? d : -d;
            f[b] += d;
        } else {
            Cd o = mad(-om, f[b] - deq, f[b]);
            if (dv.forced) o += gt;
            f[b] = o;
        }
    };
    if constexpr (!PAIRED) {
        // one direction at a time (the form the 16-bit kernels schedule best)
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            const Cd w = (Cd)wgt(b);
            const Cd eu = edot(b, ux, uy, uz);
            const Cd deq = w * mad(rho, mad((Cd)4.5 * eu, eu, mad((Cd)3, eu, (Cd)(-1.5) * usq)), s);
            Cd gt = 0;
            if (dv.forced) {
                const Cd eg = edot(b, gx, gy, gz);
                gt = guo * w * mad((Cd)9 * eu, eg, (Cd)3 * (eg - ug));
            }
            relax(b, deq, gt);
        }
    } else {
    {
        const Cd w = (Cd)wgt(0);
        relax(0, w * base, dv.forced ? guo * w * ((Cd)(-3) * ug) : (Cd)0);
    }
#pragma unroll
    for (int b = 1; b < Q; b += 2) {
        const Cd w = (Cd)wgt(b);
        const Cd eu = edot(b, ux, uy, uz);
        const Cd a = mad((Cd)4.5 * rho * eu, eu, base);
        const Cd c = (Cd)3 * rho * eu;
        Cd g1 = 0, g2 = 0;
        if (dv.forced) {
            const Cd eg = edot(b, gx, gy, gz);
            const Cd sym = mad((Cd)9 * eu, eg, (Cd)(-3) * ug), asym = (Cd)3 * eg;
            g1 = guo * w * (sym + asym);
            g2 = guo * w * (sym - asym);
        }
        relax(b, w * (a + c), g1);
        relax(b + 1, w * (a - c), g2);
    }
    }
    if constexpr (CLOSE) {
        const Cd hx = (Cd)0.5 * (gx - px), hy = (Cd)0.5 * (gy - py), hz = (Cd)0.5 * (gz - pz);
        f[1] += hx; f[2] -= hx;
        f[3] += hy; f[4] -= hy;
        f[5] += hz; f[6] -= hz;
        f[0] -= m;
    }
}

// LBGK (+ Guo) of one cell for 16-bit storage, the form with the fewest
// instructions (these kernels are bound by instruction issue, not by HBM):
// opposite directions (b, b + 1) are paired, the moments come from pair
// sums and differences, and each relaxation is one FMA,
//   f~_b = (1 - omega) f_b + (omega w_b) (a +- c) [+ (1 - omega/2) w_b (s +- t)],
//   a = drho - 1.5 rho u.u + 4.5 rho (e.u)^2,  c = 3 rho e.u,
//   s = 9 (e.u)(e.g) - 3 u.g,  t = 3 e.g,
// the same expression as collide<> (other roundings).  SCALED: f holds
// k delta (k = f16_scale, a power of two) on entry and exit, so the scale
// enters only rho, u and the per-cell constants, never a population.
template <bool SCALED>
__device__ __forceinline__ void collide_lean(float (&f)[Q], const Device &dv) {
    const float k = SCALED ? dv.f16_scale : 1.0f, ik = SCALED ? dv.f16_inv_scale : 1.0f;
    float s = f[0], jx = 0.0f, jy = 0.0f, jz = 0.0f;
    float del[Q / 2];
#pragma unroll
    for (int p = 0; p < Q / 2; ++p) {
        const int b = 2 * p + 1;
        s += f[b] + f[b + 1];
        del[p] = f[b] - f[b + 1];
        if (ex(b)) jx += ex(b) > 0 ? del[p] : -del[p];
        if (ey(b)) jy += ey(b) > 0 ? del[p] : -del[p];
        if (ez(b)) jz += ez(b) > 0 ? del[p] : -del[p];
    }
    const float rho = fmaf(s, ik, 1.0f);
    const float inv = ik / rho;
    const float kh = 0.5f * k;
    const float gx = dv.g_f[0], gy = dv.g_f[1], gz = dv.g_f[2];
    const float ux = fmaf(kh, gx, jx) * inv, uy = fmaf(kh, gy, jy) * inv, uz = fmaf(kh, gz, jz) * inv;
    const float usq = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float kr = k * rho;
    const float base = fmaf(-1.5f * kr, usq, s);       // k (drho - 1.5 rho u.u)
    const float A = 4.5f * kr, Cc = 3.0f * kr;
    const float om1 = dv.om1_f;
    const bool forced = dv.forced;
    const float ug3 = forced ? -3.0f * k * fmaf(ux, gx, fmaf(uy, gy, uz * gz)) : 0.0f;
    f[0] = fmaf(om1, f[0], forced ? fmaf(dv.gw_f[0], ug3, dv.ow_f[0] * base) : dv.ow_f[0] * base);
#pragma unroll
    for (int p = 0; p < Q / 2; ++p) {
        const int b = 2 * p + 1;
        const int wc = b < 7 ? 1 : 2;
        const float eu = edot(b, ux, uy, uz);
        const float a = fmaf(A, eu * eu, base);
        const float c = Cc * eu;
        const float ow = dv.ow_f[wc];
        float r1 = ow * (a + c), r2 = ow * (a - c);
        if (forced) {
            const float eg = edot(b, gx, gy, gz);
            const float sym = fmaf(9.0f * k * eu, eg, ug3), asym = 3.0f * k * eg;
            const float gw = dv.gw_f[wc];
            r1 = fmaf(gw, sym + asym, r1);
            r2 = fmaf(gw, sym - asym, r2);
        }
        f[b] = fmaf(om1, f[b], r1);
        f[b + 1] = fmaf(om1, f[b + 1], r2);
    }
}

// 16-bit storage without a per-population scale: FP16 keeps k delta, so the
// stored value itself is what collide_lean<true> works on
template <typename T> __device__ __forceinline__ float raw_ld(T v);
template <> __device__ __forceinline__ float raw_ld<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float raw_ld<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }


// ---- stochastic rounding of BF16 storage ------------------------------------
// BF16 keeps 8 significant bits.  Rounded to nearest, a population whose
// update is below half an ulp is rounded back to the same value every step:
// slow terms are lost and the flow settles at a biased state (Guo's term in
// the channel workload adds ~2e-8 a step to populations whose ulp is ~2e-7).
// BF16 stores therefore round up with a probability equal to the fraction of
// the ulp that is dropped: the rounding error has zero mean, and the slow
// terms accumulate as they do in FP32.  The random bits come from a
// counter-based hash of (cell, step), so a cell's rounding depends neither
// on the launch shape nor on which kernel stores the cell: 8 bits for each
// population, bytes of five 32-bit words per cell.
struct Dither {
    unsigned h[5];
};

// MurmurHash3's 32-bit finalizer (Appleby): a bijective integer mixer
__device__ __forceinline__ unsigned fmix32(unsigned x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

// the five words of a cell and step: the finalizer of a key of (cell, step),
// then four steps of a 32-bit linear congruential generator (the
// multiplier and increment of Numerical Recipes' quick generator), each
// output xor-shifted so that its low bytes carry the state's high bits
__device__ __forceinline__ Dither bf16_dither(long long c, long long t) {
    const unsigned key = (unsigned)c * 0x9E3779B1u ^ ((unsigned)t * 0x85EBCA77u + (unsigned)(t >> 32));
    Dither d;
    unsigned x = fmix32(key);
    d.h[0] = x;
#pragma unroll
    for (int k = 1; k < 5; ++k) {
        x = x * 1664525u + 1013904223u;
        d.h[k] = x ^ (x >> 15);
    }
    return d;
}

// v rounded stochastically to BF16 with byte a % 4 of word a / 4 of d, its
// bits in the upper half of the result: adding 8 random bits and half a
// step of them below the kept bits, then truncating, rounds the magnitude
// up with the probability of the dropped fraction (to 2^-9 of an ulp)
__device__ __forceinline__ unsigned bf16_sr_word(float v, const Dither &d, int a) {
    const unsigned r = __byte_perm(d.h[a >> 2], 0x80u, 0x5504u | ((unsigned)(a & 3) << 4));   // byte << 8 | 0x80
    return __float_as_uint(v) + r;
}

// the same BF16 bits in the low half
__device__ __forceinline__ unsigned bf16_sr_bits(float v, const Dither &d, int a) {
    return bf16_sr_word(v, d, a) >> 16;
}

// a 16-bit population as stored: FP16 rounded to nearest, BF16 rounded
// stochastically (the dither is used only for BF16)
template <typename T> __device__ __forceinline__ T store16(float v, const Dither &d, int a);
template <> __device__ __forceinline__ __half store16<__half>(float v, const Dither &, int) {
    return __float2half_rn(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 store16<__nv_bfloat16>(float v, const Dither &d, int a) {
    return __ushort_as_bfloat16((unsigned short)bf16_sr_bits(v, d, a));
}

// the dither of cell c in the step whose index *t holds (read only for BF16)
template <typename T> __device__ __forceinline__ Dither dither_for(long long c, const long long *t) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) return bf16_dither(c, *t);
    else return Dither{};
}

template <typename T, int V, int BX, int BY, bool FLAT = false>
__device__ __forceinline__ void bulk_body(const Device &dv, const StepPtrs &sp, const Blk &bk) {
    using Cd = typename Codec<T>::C;
    const Domain d = dv.dom;
    const int nxq = d.nx / V;
    int xq, y;
    bool active;
    if constexpr (FLAT) {
        // the z-plane's V-cell groups in row order, BX * BY a block: a warp's
        // lanes may cross a row end, where the x-neighbour fallbacks below
        // (first and last cell of a row) take over from the shuffles
        const int per_plane = nxq * d.ny;
        int q = bk.x * (BX * BY) + threadIdx.y * BX + threadIdx.x;
        active = q < per_plane;
        q = min(q, per_plane - 1);
        xq = q % nxq;
        y = q / nxq;
    } else {
        xq = bk.x * BX + threadIdx.x;
        y = bk.y * BY + threadIdx.y;
        active = xq < nxq && y < d.ny;
        xq = min(xq, nxq - 1);          // inactive lanes still join the shuffles
        y = min(y, d.ny - 1);
    }
    const int z = bk.z;
    const int lane = threadIdx.x & 31;
    const int x0 = xq * V;
    const int ym = y == 0 ? d.ny - 1 : y - 1, yp = y == d.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? d.nz - 1 : z - 1, zp = z == d.nz - 1 ? 0 : z + 1;
    const long long C = d.C;
    const long long c0 = ((long long)z * d.ny + y) * d.nx + x0;
    const T *__restrict__ src = static_cast<const T *>(sp.src);
    T *__restrict__ dst = static_cast<T *>(sp.dst);
    const float inv_scale = dv.f16_inv_scale, scale = dv.f16_scale;

    uint8_t fl[V];
    load_vec<uint8_t, V>(sp.flags_cur + c0, fl);
    // 16-bit storage: stored values as they are (collide_lean takes FP16's scale)
    constexpr bool raw16 = sizeof(T) == 2;
    auto ld = [&](T v) -> Cd {
        if constexpr (raw16) return raw_ld<T>(v);
        else return Codec<T>::ld(v, inv_scale);
    };

    Cd f[Q][V];
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        const int ys = ey(b) > 0 ? ym : (ey(b) < 0 ? yp : y);
        const int zs = ez(b) > 0 ? zm : (ez(b) < 0 ? zp : z);
        const T *row = src + (long long)b * C + ((long long)zs * d.ny + ys) * d.nx;
        T A[V];
        load_vec<T, V>(row + x0, A);
        if (ex(b) == 0) {
#pragma unroll
            for (int i = 0; i < V; ++i) f[b][i] = ld(A[i]);
        } else if (ex(b) > 0) {          // pull from x - 1
            T left = shfl(A[V - 1], 1, true);
            if (lane == 0 || x0 == 0) left = row[x0 == 0 ? d.nx - 1 : x0 - 1];
            f[b][0] = ld(left);
#pragma unroll
            for (int i = 1; i < V; ++i) f[b][i] = ld(A[i - 1]);
        } else {                          // pull from x + 1
            T right = shfl(A[0], 1, false);
            if (lane == 31 || x0 + V == d.nx) right = row[x0 + V == d.nx ? 0 : x0 + V];
#pragma unroll
            for (int i = 0; i < V - 1; ++i) f[b][i] = ld(A[i + 1]);
            f[b][V - 1] = ld(right);
        }
    }

#pragma unroll
    for (int i = 0; i < V; ++i) {
        Cd g[Q];
#pragma unroll
        for (int b = 0; b < Q; ++b) g[b] = f[b][i];
        if constexpr (raw16) collide_lean<std::is_same<T, __half>::value>(g, dv);
        else collide<Cd, std::is_same<T, float>::value>(g, dv);
        const bool solid = fl[i] & F_SOLID;
#pragma unroll
        for (int b = 0; b < Q; ++b) f[b][i] = solid ? (Cd)0 : g[b];
    }
    // overlapped steps: a tile near a body is the near kernel's
    const bool far = !sp.far_skip || sp.far_skip[((long long)z * d.ny + y) * ((d.nx + TILE_X - 1) / TILE_X) +
                                                 x0 / TILE_X] == 0u;
    if (!active || !far) return;
    // BF16 rounds stochastically (one cell per thread for 16-bit storage here)
    static_assert(!raw16 || V == 1, "16-bit storage with several cells per thread uses bulk16_kernel");
    static_assert(TILE_X % V == 0, "a thread's cells lie in one tile");
    const Dither dz = raw16 ? dither_for<T>(c0, sp.tstep) : Dither{};
    auto st = [&](Cd v, int b) -> T {
        if constexpr (raw16) return store16<T>(v, dz, b);
        else return Codec<T>::st(v, scale);
    };
    // fluid cells with a non-zero flag byte belong to the boundary kernel,
    // which may run concurrently: leave them alone
    bool all_mine = true;
#pragma unroll
    for (int i = 0; i < V; ++i) all_mine = all_mine && (fl[i] == 0 || (fl[i] & F_SOLID));
    if (all_mine) {
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            T out[V];
#pragma unroll
            for (int i = 0; i < V; ++i) out[i] = st(f[b][i], b);
            store_vec<T, V>(dst + (long long)b * C + c0, out);
        }
        return;
    }
#pragma unroll
    for (int b = 0; b < Q; ++b)
#pragma unroll
        for (int i = 0; i < V; ++i)
            if (fl[i] == 0 || (fl[i] & F_SOLID)) dst[(long long)b * C + c0 + i] = st(f[b][i], b);
}

// MINB == 1 leaves the register budget to the compiler (an explicit minimum
// of one block lets it spend far more registers than it needs)
template <typename T, int V, int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB == 1 ? 0 : MINB)
bulk_kernel(const Device dv, const StepPtrs sp) {
    pdl_enter();
    bulk_body<T, V, BX, BY>(dv, sp, launch_blk());
}

// a batched bulk block takes BATCH_PZ consecutive z-planes of its member:
// the member lookup at its start (a few dependent loads and barriers with
// no population traffic in flight) is paid once for all of them
constexpr int BATCH_PZ = 4;

template <typename T, int V, int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB == 1 ? 0 : MINB) bulk_batch(const Batch bt) {
    LBM_BATCH_MEMBER(bt);
    const int z0 = sbk.z * BATCH_PZ, z1 = min(z0 + BATCH_PZ, sdv.dom.nz);
    for (int z = z0; z < z1; ++z) {
        Blk pb = sbk;
        pb.z = z;
        bulk_body<T, V, BX, BY, true>(sdv, ssp, pb);
    }
}

// 16-bit values packed two to a 32-bit word (the lower address in the low
// half): widening to FP32 and narrowing back (round to nearest even)
template <typename T> __device__ __forceinline__ float half_lo(unsigned w);
template <typename T> __device__ __forceinline__ float half_hi(unsigned w);
template <typename T> __device__ __forceinline__ unsigned half_bits(float v);
template <> __device__ __forceinline__ float half_lo<__half>(unsigned w) {
    return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
}
template <> __device__ __forceinline__ float half_hi<__half>(unsigned w) {
    return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
}
template <> __device__ __forceinline__ unsigned half_bits<__half>(float v) {
    return __half_as_ushort(__float2half_rn(v));
}
template <> __device__ __forceinline__ float half_lo<__nv_bfloat16>(unsigned w) { return __uint_as_float(w << 16); }
template <> __device__ __forceinline__ float half_hi<__nv_bfloat16>(unsigned w) {
    return __uint_as_float(w & 0xffff0000u);
}
// the stored bits of population a of a cell: FP16 to nearest, BF16 stochastically
template <typename T> __device__ __forceinline__ unsigned store_bits(float v, const Dither &d, int a) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) return bf16_sr_bits(v, d, a);
    else return half_bits<T>(v);
}

// The bulk kernel for 16-bit storage, V (even) cells per thread.  The
// populations stay packed two to a word (the thread's cells 2j and 2j + 1
// in word j) from load to store, half the registers of widened values, so
// that more warps -- or more bytes per warp -- keep HBM requests in flight.
// A shift along x is a byte permute of adjacent words (and of one word
// shuffled from the neighbouring lane); a cell's 19 values are widened to
// FP32 just before its collision (collide_lean, the row-staged kernel's
// arithmetic) and narrowed back into their half-words after it.
template <typename T, int V, int BX, int BY, bool FLAT = false>
__device__ __forceinline__ void bulk16_body(const Device &dv, const StepPtrs &sp, const Blk &bk) {
    static_assert(sizeof(T) == 2 && V % 2 == 0, "two 16-bit cells a word");
    constexpr int W = V / 2;
    using RawV = typename Raw<2 * V>::type;
    const Domain d = dv.dom;
    const int nxq = d.nx / V;
    int xq, y;
    bool active;
    if constexpr (FLAT) {
        // the z-plane's V-cell groups in row order, BX * BY a block: a warp's
        // lanes may cross a row end, where the x-neighbour fallbacks below
        // (first and last cell of a row) take over from the shuffles
        const int per_plane = nxq * d.ny;
        int q = bk.x * (BX * BY) + threadIdx.y * BX + threadIdx.x;
        active = q < per_plane;
        q = min(q, per_plane - 1);
        xq = q % nxq;
        y = q / nxq;
    } else {
        xq = bk.x * BX + threadIdx.x;
        y = bk.y * BY + threadIdx.y;
        active = xq < nxq && y < d.ny;
        xq = min(xq, nxq - 1);          // inactive lanes still join the shuffles
        y = min(y, d.ny - 1);
    }
    const int z = bk.z;
    const int lane = threadIdx.x & 31;
    const int x0 = xq * V;
    const int ym = y == 0 ? d.ny - 1 : y - 1, yp = y == d.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? d.nz - 1 : z - 1, zp = z == d.nz - 1 ? 0 : z + 1;
    const long long C = d.C;
    const long long c0 = ((long long)z * d.ny + y) * d.nx + x0;
    const unsigned short *__restrict__ src = static_cast<const unsigned short *>(sp.src);
    unsigned short *__restrict__ dst = static_cast<unsigned short *>(sp.dst);

    uint8_t fl[V];
    load_vec<uint8_t, V>(sp.flags_cur + c0, fl);

    unsigned w[Q][W];
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        const int ys = ey(b) > 0 ? ym : (ey(b) < 0 ? yp : y);
        const int zs = ez(b) > 0 ? zm : (ez(b) < 0 ? zp : z);
        const unsigned short *row = src + (long long)b * C + ((long long)zs * d.ny + ys) * d.nx;
        unsigned R[W];
        {
            const RawV r = __ldg(reinterpret_cast<const RawV *>(row + x0));
            memcpy(&R, &r, sizeof(R));
        }
        if (ex(b) == 0) {
#pragma unroll
            for (int j = 0; j < W; ++j) w[b][j] = R[j];
        } else if (ex(b) > 0) {          // pull from x - 1: the left neighbour's last half-word first
            unsigned lw = __shfl_up_sync(0xffffffffu, R[W - 1], 1);
            if (lane == 0 || x0 == 0) lw = (unsigned)row[x0 == 0 ? d.nx - 1 : x0 - 1] << 16;
            w[b][0] = __byte_perm(lw, R[0], 0x5432);
#pragma unroll
            for (int j = 1; j < W; ++j) w[b][j] = __byte_perm(R[j - 1], R[j], 0x5432);
        } else {                          // pull from x + 1: the right neighbour's first half-word last
            unsigned rw = __shfl_down_sync(0xffffffffu, R[0], 1);
            if (lane == 31 || x0 + V == d.nx) rw = (unsigned)row[x0 + V == d.nx ? 0 : x0 + V];
#pragma unroll
            for (int j = 0; j < W - 1; ++j) w[b][j] = __byte_perm(R[j], R[j + 1], 0x5432);
            w[b][W - 1] = __byte_perm(R[W - 1], rw, 0x5432);
        }
    }

#pragma unroll
    for (int i = 0; i < V; ++i) {
        const int j = i >> 1;
        const bool hi = i & 1;
        float g[Q];
#pragma unroll
        for (int b = 0; b < Q; ++b) g[b] = hi ? half_hi<T>(w[b][j]) : half_lo<T>(w[b][j]);
        collide_lean<std::is_same<T, __half>::value>(g, dv);
        const bool solid = fl[i] & F_SOLID;
        const Dither dz = dither_for<T>(c0 + i, sp.tstep);
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            if constexpr (std::is_same<T, __nv_bfloat16>::value) {
                // the rounded bits are the upper half of the sum: select them
                const unsigned h = solid ? 0u : bf16_sr_word(g[b], dz, b);
                w[b][j] = hi ? __byte_perm(w[b][j], h, 0x7610) : __byte_perm(h, w[b][j], 0x7632);
            } else {
                const unsigned h = solid ? 0u : store_bits<T>(g[b], dz, b);
                w[b][j] = hi ? __byte_perm(w[b][j], h, 0x5410) : __byte_perm(h, w[b][j], 0x7610);
            }
        }
    }
    // overlapped steps: a tile near a body is the near kernel's
    static_assert(TILE_X % V == 0, "a thread's cells lie in one tile");
    const bool far = !sp.far_skip || sp.far_skip[((long long)z * d.ny + y) * ((d.nx + TILE_X - 1) / TILE_X) +
                                                 x0 / TILE_X] == 0u;
    if (!active || !far) return;
    // fluid cells with a non-zero flag byte belong to the boundary kernel,
    // which may run concurrently: leave them alone
    bool all_mine = true;
#pragma unroll
    for (int i = 0; i < V; ++i) all_mine = all_mine && (fl[i] == 0 || (fl[i] & F_SOLID));
    if (all_mine) {
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            RawV r;
            memcpy(&r, &w[b], sizeof(r));
            *reinterpret_cast<RawV *>(dst + (long long)b * C + c0) = r;
        }
        return;
    }
#pragma unroll
    for (int b = 0; b < Q; ++b)
#pragma unroll
        for (int i = 0; i < V; ++i)
            if (fl[i] == 0 || (fl[i] & F_SOLID))
                dst[(long long)b * C + c0 + i] = (unsigned short)((i & 1) ? w[b][i >> 1] >> 16 : w[b][i >> 1] & 0xffffu);
}

template <typename T, int V, int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB == 1 ? 0 : MINB)
bulk16_kernel(const Device dv, const StepPtrs sp) {
    pdl_enter();
    bulk16_body<T, V, BX, BY>(dv, sp, launch_blk());
}

template <typename T, int V, int BX, int BY, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB == 1 ? 0 : MINB) bulk16_batch(const Batch bt) {
    LBM_BATCH_MEMBER(bt);
    const int z0 = sbk.z * BATCH_PZ, z1 = min(z0 + BATCH_PZ, sdv.dom.nz);
    for (int z = z0; z < z1; ++z) {
        Blk pb = sbk;
        pb.z = z;
        bulk16_body<T, V, BX, BY, true>(sdv, ssp, pb);
    }
}

// Velocity of body b's surface at lattice point p in the compute type R:
// FP64 throughout for FP64 storage; otherwise the minimum-image offset in
// FP64 and V + W x offset in R (the moving-wall term is ~1e-4 and its R
// rounding sits below the storage's)
template <typename R>
__device__ inline void wall_velocity(const Domain &d, const BodyState &b, int px, int py, int pz, R (&u)[3]) {
    if constexpr (sizeof(R) == 8) {
        double w[3];
        surface_velocity(d, b, px, py, pz, w);
        u[0] = w[0]; u[1] = w[1]; u[2] = w[2];
    } else {
        double od[3];
        offset_from(d, b, (double)px, (double)py, (double)pz, od);
        const R o0 = (R)od[0], o1 = (R)od[1], o2 = (R)od[2];
        const R w0 = (R)b.W[0], w1 = (R)b.W[1], w2 = (R)b.W[2];
        u[0] = (R)b.V[0] + (w1 * o2 - w2 * o1);
        u[1] = (R)b.V[1] + (w2 * o0 - w0 * o2);
        u[2] = (R)b.V[2] + (w0 * o1 - w1 * o0);
    }
}

// a body for the moving-wall term: the centre wrapped into the domain and
// split into its cell (int) and the offset within it (FP32), velocity and
// angular velocity in FP32 (copied from the step's geometry record)
struct WallBody {
    int ic[3];
    float frac[3], v[3], w[3];
};

__device__ inline WallBody wall_body(const BodyGeom &g) {
    WallBody r;
    for (int i = 0; i < 3; ++i) {
        r.ic[i] = g.ci[i];
        r.frac[i] = g.cf[i];
        r.v[i] = g.v[i];
        r.w[i] = g.w[i];
    }
    return r;
}

__device__ inline int near_cell(int o, int n, int periodic) {
    if (!periodic) return o;
    return 2 * o > n ? o - n : (2 * o < -n ? o + n : o);
}

// V + W x (p - X) in FP32; the minimum-image offset is an integer difference
// of cells wrapped by compares minus the centre's fraction (exact to FP32
// rounding of a few-cell offset)
__device__ inline void wall_velocity_wrapped(const Domain &d, const WallBody &b, int px, int py, int pz,
                                             float (&u)[3]) {
    const float o0 = (float)near_cell(px - b.ic[0], d.nx, d.px) - b.frac[0];
    const float o1 = (float)near_cell(py - b.ic[1], d.ny, d.py) - b.frac[1];
    const float o2 = (float)near_cell(pz - b.ic[2], d.nz, d.pz) - b.frac[2];
    u[0] = b.v[0] + (b.w[1] * o2 - b.w[2] * o1);
    u[1] = b.v[1] + (b.w[2] * o0 - b.w[0] * o2);
    u[2] = b.v[2] + (b.w[0] * o1 - b.w[1] * o0);
}

// Cells with a non-zero flag byte: refill, bounce-back at walls and moving
// obstacles, then LBGK.  mode 0: the cells the remap listed (fluid with
// F_NEAR or F_SOLID_PREV), one a thread, on a grid sized for the longest
// possible list; mode 1: block row y = wall face (axis * 2 + side), the
// face's cells.  A cell in
// both sets, or listed twice, is computed more than once with the same
// result.  Every load a cell needs is issued before any of them is used, so
// a thread waits for memory about twice instead of once per direction.
template <typename T>
__device__ __forceinline__ void boundary_body(const Device &dv, const StepPtrs &sp, const Blk &bk, int mode) {
    using Cd = typename Codec<T>::C;
    const Domain d = dv.dom;
    // 32/16-bit storage: the bodies of step n-1 with their centres wrapped
    // into the domain, so that a link's minimum-image offset is an integer
    // difference, two compares and the FP32 position within the cell
    __shared__ WallBody wb[sizeof(T) == 8 ? 1 : LBM_MAX_BODIES_DEV];
    const int l = bk.x * blockDim.x + threadIdx.x;
    // the count may pass the capacity after an overflow (reported as an error): never read past it
    const int listed = mode == 0 ? (int)min((long long)*dv.bcount, dv.blist_cap) : 0;
    if (mode == 0 && (int)(bk.x * blockDim.x) >= listed) return;      // the whole block is past the list
    if constexpr (sizeof(T) != 8) {
        for (int k = threadIdx.x; k < dv.nb; k += blockDim.x) wb[k] = wall_body(dv.geom[(sp.parity ^ 1) * dv.nb + k]);
        __syncthreads();
    }
    int x, y, z;
    if (mode == 0) {
        if (l >= listed) return;
        const unsigned cl = dv.blist[l];          // C < 2^31: 32-bit division
        const unsigned nxu = (unsigned)d.nx, nyu = (unsigned)d.ny;
        x = (int)(cl % nxu);
        y = (int)((cl / nxu) % nyu);
        z = (int)(cl / (nxu * nyu));
    } else {
        const int axis = bk.y >> 1, hi = bk.y & 1;
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
    const uint8_t fc = sp.flags_cur[c];
    if (fc == 0 || (fc & F_SOLID)) return;
    const T *__restrict__ src = static_cast<const T *>(sp.src);
    const float s = dv.f16_inv_scale;
    Cd f[Q];
    if (fc & F_SOLID_PREV) {
        // uncovered cell: f = f_eq(rho_avg, u_w(x)) with the state of step n;
        // rho_avg over the D3Q19 neighbours fluid in both epochs (1 if none)
        long long nc[Q];
        bool ok[Q];
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            const int nx_ = x + ex(a), ny_ = y + ey(a), nz_ = z + ez(a);
            ok[a] = !((!d.px && (nx_ < 0 || nx_ >= d.nx)) || (!d.py && (ny_ < 0 || ny_ >= d.ny)) ||
                      (!d.pz && (nz_ < 0 || nz_ >= d.nz)));
            nc[a] = ((long long)wrap_axis(nz_, d.nz) * d.ny + wrap_axis(ny_, d.ny)) * d.nx + wrap_axis(nx_, d.nx);
        }
#pragma unroll
        for (int a = 1; a < Q; ++a) ok[a] = ok[a] && !(sp.flags_cur[nc[a]] & (F_SOLID | F_SOLID_PREV));
        const int k = sp.bid_prev[c];
        if constexpr (sizeof(T) == 8) {
            double sum = 0.0;
            int cnt = 0;
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                Cd drho = 0;
#pragma unroll
                for (int bb = 0; bb < Q; ++bb) drho += Codec<T>::ld(src[bb * C + nc[a]], s);
                if (ok[a]) {
                    sum += 1.0 + (double)drho;
                    ++cnt;
                }
            }
            const double rho = cnt ? sum / cnt : 1.0;
            double u[3] = {0.0, 0.0, 0.0};
            if (k != NO_BODY) surface_velocity(d, sp.body_cur[k], x, y, z, u);
            const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
            for (int b = 0; b < Q; ++b) {
                const double eu = ex(b) * u[0] + ey(b) * u[1] + ez(b) * u[2];
                f[b] = (Cd)(wgt(b) * (rho - 1.0) + wgt(b) * rho * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
            }
        } else {
            // FP32: the mean of the neighbours' density deviations (small
            // numbers: no 1 + drho is ever rounded), u_w of state n
            float dsum = 0.0f;
            int cnt = 0;
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                float drho = 0.0f;
#pragma unroll
                for (int bb = 0; bb < Q; ++bb) drho += Codec<T>::ld(src[bb * C + nc[a]], s);
                if (ok[a]) {
                    dsum += drho;
                    ++cnt;
                }
            }
            const float drho = cnt ? dsum / (float)cnt : 0.0f;
            const float rho = 1.0f + drho;
            float u[3] = {0.0f, 0.0f, 0.0f};
            if (k != NO_BODY) wall_velocity_wrapped(d, wall_body(dv.geom[sp.parity * dv.nb + k]), x, y, z, u);
            const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
            for (int b = 0; b < Q; ++b) {
                const float w = (float)wgt(b);
                const float eu = ex(b) * u[0] + ey(b) * u[1] + ez(b) * u[2];
                f[b] = w * drho + w * rho * (3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
            }
        }
    } else {
        // bounce-back at walls (Eq. 4) and at obstacles of step n-1
        Cd own[Q];
        Cd drho = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            own[a] = Codec<T>::ld(src[(long long)a * C + c], s);
            drho += own[a];
        }
        const Cd rho_x = (Cd)1 + drho;
        f[0] = own[0];
#pragma unroll
        for (int b = 1; b < Q; ++b) {
            const int sx = x - ex(b), sy = y - ey(b), sz = z - ez(b);
            const bool wall = (!d.px && (sx < 0 || sx >= d.nx)) || (!d.py && (sy < 0 || sy >= d.ny)) ||
                              (!d.pz && (sz < 0 || sz >= d.nz));
            const long long sc = ((long long)wrap_axis(sz, d.nz) * d.ny + wrap_axis(sy, d.ny)) * d.nx +
                                 wrap_axis(sx, d.nx);
            const uint8_t fp = sp.flags_prev[sc];
            const Cd pulled = Codec<T>::ld(src[(long long)b * C + sc], s);
            Cd v = pulled;
            if (wall) {
                v = own[opp(b)];                                             // Eq. 4
            } else if (fp & F_SOLID) {
                const int k = sp.bid_prev[sc];
                Cd u[3] = {0, 0, 0};
                if (k != NO_BODY) {
                    if constexpr (sizeof(T) == 8) wall_velocity<Cd>(d, sp.body_prev[k], sx, sy, sz, u);
                    else wall_velocity_wrapped(d, wb[k], sx, sy, sz, u);
                }
                const Cd eu = (Cd)ex(b) * u[0] + (Cd)ey(b) * u[1] + (Cd)ez(b) * u[2];
                v = own[opp(b)] + (Cd)(6.0 * wgt(b)) * rho_x * eu;          // moving wall
            }
            f[b] = v;
        }
    }
    if constexpr (sizeof(T) != 8) {
        // rho - 1 of the cell for the momentum exchange (the collision keeps
        // it); a lattice without bodies has no momentum exchange and no
        // record (a wall-face cell is listed here all the same)
        if (dv.nb > 0) {
            Cd drho = 0;
#pragma unroll
            for (int b = 0; b < Q; ++b) drho += f[b];
            dv.rho_near[c] = (float)drho;
        }
    }
    collide<Cd, std::is_same<T, float>::value>(f, dv);
    T *__restrict__ dst = static_cast<T *>(sp.dst);
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        const Dither dz = bf16_dither(c, *sp.tstep);
#pragma unroll
        for (int b = 0; b < Q; ++b) dst[(long long)b * C + c] = store16<T>(f[b], dz, b);
    } else {
#pragma unroll
        for (int b = 0; b < Q; ++b) dst[(long long)b * C + c] = Codec<T>::st(f[b], dv.f16_scale);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) boundary_kernel(const Device dv, const StepPtrs sp, int mode) {
    boundary_body<T>(dv, sp, launch_blk(), mode);
}

// a batched launch of one mode over the members
template <typename T>
__global__ void __launch_bounds__(256) boundary_batch(const Batch bt, int mode) {
    LBM_BATCH_MEMBER(bt);
    boundary_body<T>(sdv, ssp, sbk, mode);
}

// ---- TMA row-staged variant ---------------------------------------------------
//
// Persistent blocks walk the x-rows (y, z) of the lattice (row r = blockIdx.x
// + i gridDim.x).  For each row one thread issues 20 bulk copies
// (cp.async.bulk, completed on an mbarrier with the byte count): the 19
// source rows, direction b from the neighbour row (y - ey_b, z - ez_b) of
// plane b, and the row's flag bytes, into one of NSTAGE shared-memory stages;
// NSTAGE rows are in flight.  The threads then pull f_b(x) = row_b[x - ex_b]
// from shared memory, collide with the same code as the register variant
// and store -- the same arithmetic, the same bits.  Every wait on an
// mbarrier is bounded: past the limit the block records ST_TIMEOUT, waits
// (bounded again) for its copies in flight and returns.

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bulk copy global -> shared of `bytes` (a multiple of 16, both addresses
// 16-byte aligned), completing `bytes` transactions on bar
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

constexpr int TMA_THREADS = 256;
constexpr long long TMA_WAIT_CYCLES = 1LL << 31;     // ~1 s of SM clock before a block gives up
constexpr long long TMA_EXPIRE_CYCLES = 1LL << 16;   // the bound of the expired-wait check (~30 us)
constexpr int TMA_HEADER = 128;                      // mbarriers, ahead of the stages

__host__ __device__ constexpr size_t tma_stage_bytes(int nx, int elem) { return (size_t)Q * nx * elem + (size_t)nx; }

template <typename T, int NSTAGE, int MINB, int ROWS>
__global__ void __launch_bounds__(TMA_THREADS, MINB) bulk_tma_kernel(const Device dv, const StepPtrs sp) {
    pdl_enter();
    using Cd = typename Codec<T>::C;
    static_assert((NSTAGE + 1) * sizeof(uint64_t) <= TMA_HEADER, "the mbarriers fit the header");
    extern __shared__ __align__(128) unsigned char smem[];
    const Domain d = dv.dom;
    const int nx = d.nx;
    const unsigned row_bytes = (unsigned)(nx * sizeof(T));
    const unsigned flag_off = Q * row_bytes;
    const unsigned row_stage = (unsigned)tma_stage_bytes(nx, sizeof(T));     // one x-row's sources + flags
    const unsigned stage_bytes = ROWS * row_stage;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    unsigned char *stages = smem + TMA_HEADER;
    const long long rows = (long long)d.ny * d.nz;
    const long long first = blockIdx.x;
    const long long nmine = rows > first ? (rows - 1 - first) / gridDim.x + 1 : 0;
    const long long ngroups = (nmine + ROWS - 1) / ROWS;     // a stage holds ROWS of this block's rows
    const T *__restrict__ src = static_cast<const T *>(sp.src);
    T *__restrict__ dst = static_cast<T *>(sp.dst);
    const long long C = d.C;
    const float inv_scale = dv.f16_inv_scale, scale = dv.f16_scale;
    const int ntx = (nx + TILE_X - 1) / TILE_X;

    if (threadIdx.x == 0) {
        // bar[NSTAGE] is never arrived at: with dv.expire_waits the first
        // wait of every block is on it, so that its bounded wait runs out
        for (int st = 0; st <= NSTAGE; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](long long g) {          // thread 0: rows of group g into stage g % NSTAGE
        const int st = (int)(g % NSTAGE);
        const int nr = (int)min((long long)ROWS, nmine - g * ROWS);
        unsigned char *buf0 = stages + (size_t)st * stage_bytes;
        mbar_expect_tx(&bar[st], nr * row_stage);
        for (int rr = 0; rr < nr; ++rr) {
            const long long r = first + (g * ROWS + rr) * gridDim.x;
            const int y = (int)(r % d.ny), z = (int)(r / d.ny);
            unsigned char *buf = buf0 + (size_t)rr * row_stage;
#pragma unroll
            for (int b = 0; b < Q; ++b) {
                const int ys = wrap_axis(y - ey(b), d.ny), zs = wrap_axis(z - ez(b), d.nz);
                bulk_copy(buf + b * row_bytes, src + (long long)b * C + ((long long)zs * d.ny + ys) * nx,
                          row_bytes, &bar[st]);
            }
            bulk_copy(buf + flag_off, sp.flags_cur + r * nx, (unsigned)nx, &bar[st]);
        }
    };
    if (threadIdx.x == 0)
        for (long long g = 0; g < ngroups && g < NSTAGE; ++g) issue(g);

    long long g = 0;
    bool ok = true;
    for (; g < ngroups; ++g) {
        const int st = (int)(g % NSTAGE);
        const unsigned parity = (unsigned)((g / NSTAGE) & 1);
        const long long t0 = clock64();
        bool ready = false;
        if (dv.expire_waits && g == 0) {
            while (!(ready = mbar_try_wait(&bar[NSTAGE], 0)) && clock64() - t0 < TMA_EXPIRE_CYCLES) {
            }
        } else {
            while (!(ready = mbar_try_wait(&bar[st], parity)) && clock64() - t0 < TMA_WAIT_CYCLES) {
            }
        }
        ok = __syncthreads_and(ready);
        if (!ok) break;
        const int nr = (int)min((long long)ROWS, nmine - g * ROWS);
        for (int rr = 0; rr < nr; ++rr) {
            const unsigned char *buf = stages + (size_t)st * stage_bytes + (size_t)rr * row_stage;
            const T *rowb = reinterpret_cast<const T *>(buf);
            const uint8_t *fl = buf + flag_off;
            const long long r = first + (g * ROWS + rr) * gridDim.x;
            const long long c0 = r * nx;
            for (int x = threadIdx.x; x < nx; x += TMA_THREADS) {
                const uint8_t f8 = fl[x];
                if (f8 != 0 && !(f8 & F_SOLID)) continue;      // the boundary kernel's cell
                if (sp.far_skip && sp.far_skip[r * ntx + x / TILE_X]) continue;    // the near kernel's
                if (f8 & F_SOLID) {
#pragma unroll
                    for (int b = 0; b < Q; ++b) dst[(long long)b * C + c0 + x] = Codec<T>::st((Cd)0, scale);
                    continue;
                }
                Cd f[Q];
#pragma unroll
                for (int b = 0; b < Q; ++b) {
                    int xs = x - ex(b);
                    xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
                    if constexpr (sizeof(T) == 2) f[b] = raw_ld<T>(rowb[b * nx + xs]);
                    else f[b] = Codec<T>::ld(rowb[b * nx + xs], inv_scale);
                }
                if constexpr (sizeof(T) == 2) {
                    collide_lean<std::is_same<T, __half>::value>(f, dv);
                    const Dither dz = dither_for<T>(c0 + x, sp.tstep);
#pragma unroll
                    for (int b = 0; b < Q; ++b) dst[(long long)b * C + c0 + x] = store16<T>(f[b], dz, b);
                } else {
                    collide<Cd, std::is_same<T, float>::value>(f, dv);
#pragma unroll
                    for (int b = 0; b < Q; ++b) dst[(long long)b * C + c0 + x] = Codec<T>::st(f[b], scale);
                }
            }
        }
        __syncthreads();                         // stage st is free again
        if (threadIdx.x == 0 && g + NSTAGE < ngroups) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(g + NSTAGE);
        }
    }
    if (!ok && threadIdx.x == 0) {
        atomicOr(dv.status, ST_TIMEOUT);
        // the copies still in flight target this block's shared memory
        for (long long j = g; j < ngroups && j < g + NSTAGE; ++j) {
            const long long t0 = clock64();
            while (!mbar_try_wait(&bar[j % NSTAGE], (unsigned)((j / NSTAGE) & 1)) &&
                   clock64() - t0 < TMA_WAIT_CYCLES) {
            }
        }
    }
}

template <typename T, int NSTAGE, int PER_SM, int ROWS = 1>
size_t tma_smem_bytes(int nx) { return TMA_HEADER + (size_t)NSTAGE * ROWS * tma_stage_bytes(nx, sizeof(T)); }

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <typename T, int NSTAGE, int PER_SM, int ROWS = 1>
void launch_tma(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const size_t bytes = tma_smem_bytes<T, NSTAGE, PER_SM, ROWS>(dv.dom.nx);
    const long long rows = (long long)dv.dom.ny * dv.dom.nz;
    const long long grid = std::min<long long>(rows, (long long)sm_count() * PER_SM);
    launch_kernel(dv.pdl != 0, bulk_tma_kernel<T, NSTAGE, PER_SM, ROWS>, dim3((unsigned)grid), dim3(TMA_THREADS), bytes,
                  s, dv, sp);
}

template <typename T, int NSTAGE, int PER_SM, int ROWS = 1>
bool tma_fits(int nx) {
    return nx % 16 == 0 && tma_smem_bytes<T, NSTAGE, PER_SM, ROWS>(nx) * PER_SM <= 227u * 1024u;
}

template <typename T, int NSTAGE, int PER_SM, int ROWS = 1>
void tma_prepare() {
    cudaFuncSetAttribute(bulk_tma_kernel<T, NSTAGE, PER_SM, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
}

template <typename T, int V, int BX, int BY, int MINB>
void launch_bulk(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const int nxq = dv.dom.nx / V;
    dim3 grid((nxq + BX - 1) / BX, (dv.dom.ny + BY - 1) / BY, dv.dom.nz);
    launch_kernel(dv.pdl != 0, bulk_kernel<T, V, BX, BY, MINB>, grid, dim3(BX, BY), 0, s, dv, sp);
}

template <typename T, int V, int BX, int BY, int MINB>
void launch_bulk16(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const int nxq = dv.dom.nx / V;
    dim3 grid((nxq + BX - 1) / BX, (dv.dom.ny + BY - 1) / BY, dv.dom.nz);
    launch_kernel(dv.pdl != 0, bulk16_kernel<T, V, BX, BY, MINB>, grid, dim3(BX, BY), 0, s, dv, sp);
}

template <typename T, int V, int MINB>
void launch_shape16(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const int nxq = dv.dom.nx / V;
    if (nxq >= 128) launch_bulk16<T, V, 128, 2, MINB>(dv, sp, s);
    else launch_bulk16<T, V, 32, 8, MINB>(dv, sp, s);
}

// launch shapes: V cells per thread in blocks of 256 threads (BX a multiple
// of 32 along x); MINB > 1 caps the registers so that MINB blocks fit an SM
template <typename T, int V, int MINB>
void launch_shape(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const int nxq = dv.dom.nx / V;
    if (nxq >= 128) launch_bulk<T, V, 128, 2, MINB>(dv, sp, s);
    else launch_bulk<T, V, 32, 8, MINB>(dv, sp, s);
}

using Launcher = void (*)(const Device &, const StepPtrs &, cudaStream_t);
struct Variant {
    int precision, vec, minb;       // vec -1: TMA row-staged, minb = resident blocks per SM
    Launcher fn;
    bool (*fits)(int nx);           // staged variants: shared memory and alignment for this nx
};

// the compiled variants of the bulk kernel; the first entry of a precision
// and width is its default
const Variant kVariants[] = {
    {0, 1, 1, launch_shape<double, 1, 1>},
    {0, 2, 1, launch_shape<double, 2, 1>},
    {1, 2, 1, launch_shape<float, 2, 1>},
    {1, 2, 4, launch_shape<float, 2, 4>},
    {1, 1, 1, launch_shape<float, 1, 1>},
    {1, 4, 1, launch_shape<float, 4, 1>},
    {2, 4, 1, launch_shape16<__half, 4, 1>},
    {2, 4, 2, launch_shape16<__half, 4, 2>},
    {2, 4, 3, launch_shape16<__half, 4, 3>},
    {2, 8, 1, launch_shape16<__half, 8, 1>},
    {2, 8, 2, launch_shape16<__half, 8, 2>},
    {2, 2, 1, launch_shape16<__half, 2, 1>},
    {2, 2, 4, launch_shape16<__half, 2, 4>},
    {2, 1, 1, launch_shape<__half, 1, 1>},
    {3, 4, 1, launch_shape16<__nv_bfloat16, 4, 1>},
    {3, 4, 2, launch_shape16<__nv_bfloat16, 4, 2>},
    {3, 4, 3, launch_shape16<__nv_bfloat16, 4, 3>},
    {3, 8, 1, launch_shape16<__nv_bfloat16, 8, 1>},
    {3, 8, 2, launch_shape16<__nv_bfloat16, 8, 2>},
    {3, 2, 1, launch_shape16<__nv_bfloat16, 2, 1>},
    {3, 2, 4, launch_shape16<__nv_bfloat16, 2, 4>},
    {3, 1, 1, launch_shape<__nv_bfloat16, 1, 1>},
    {0, -1, 1, launch_tma<double, 2, 1>, tma_fits<double, 2, 1>},
    {1, -1, 1, launch_tma<float, 4, 1>, tma_fits<float, 4, 1>},
    {1, -1, 2, launch_tma<float, 2, 2>, tma_fits<float, 2, 2>},
    {2, -1, 2, launch_tma<__half, 2, 2, 2>, tma_fits<__half, 2, 2, 2>},
    {2, -1, 3, launch_tma<__half, 2, 3>, tma_fits<__half, 2, 3>},
    {2, -1, 4, launch_tma<__half, 2, 4>, tma_fits<__half, 2, 4>},
    {3, -1, 2, launch_tma<__nv_bfloat16, 2, 2, 2>, tma_fits<__nv_bfloat16, 2, 2, 2>},
    {3, -1, 3, launch_tma<__nv_bfloat16, 2, 3>, tma_fits<__nv_bfloat16, 2, 3>},
    {3, -1, 4, launch_tma<__nv_bfloat16, 2, 4>, tma_fits<__nv_bfloat16, 2, 4>},
};
const Variant *find_variant(int precision, int vec, int minb) {
    const Variant *first = nullptr;
    for (const Variant &v : kVariants) {
        if (v.precision != precision || v.vec != vec) continue;
        if (!first) first = &v;
        if (minb == 0 || v.minb == minb) return minb == 0 ? first : &v;
    }
    return nullptr;
}

template <typename T>
void launch_boundary(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    if (dv.nb > 0) {
        // the list's length is on the device: blocks past it return at once
        const long long side = dv.remap_side;
        const long long most = (long long)dv.nb * side * side * side;
        const unsigned bx = (unsigned)((most + 255) / 256);
        boundary_kernel<T><<<bx, 256, 0, s>>>(dv, sp, 0);
    }
    if (!(dv.dom.px && dv.dom.py && dv.dom.pz)) {
        const long long nx = dv.dom.nx, ny = dv.dom.ny, nz = dv.dom.nz;
        const long long area = std::max(ny * nz, std::max(nx * nz, nx * ny));
        boundary_kernel<T><<<dim3((unsigned)((area + 255) / 256), 6), 256, 0, s>>>(dv, sp, 1);
    }
}

}  // namespace

bool valid_vector_width(const Device &dv, int v) {
    if (v == -1) {
        const Variant *x = find_variant(dv.precision, -1, 0);
        return x && x->fits(dv.dom.nx);
    }
    return v >= 1 && dv.dom.nx % v == 0 && find_variant(dv.precision, v, 0) != nullptr;
}

bool valid_variant(const Device &dv, int v, int minb) {
    if (!valid_vector_width(dv, v)) return false;
    const Variant *x = find_variant(dv.precision, v, minb);
    return x && (!x->fits || x->fits(dv.dom.nx));
}

void prepare_bulk_variants() {
    static bool done = false;
    if (done) return;
    tma_prepare<double, 2, 1>();
    tma_prepare<float, 4, 1>();
    tma_prepare<float, 2, 2>();
    tma_prepare<__half, 2, 2, 2>();
    tma_prepare<__half, 2, 3>();
    tma_prepare<__half, 2, 4>();
    tma_prepare<__nv_bfloat16, 2, 2, 2>();
    tma_prepare<__nv_bfloat16, 2, 3>();
    tma_prepare<__nv_bfloat16, 2, 4>();
    done = true;
}

int default_vector_width(const Device &dv) {
    const int pref = dv.precision == 0 ? 1 : (dv.precision == 1 ? 2 : 4);
    for (int v = pref; v > 1; v >>= 1)
        if (dv.dom.nx % v == 0) return v;
    return 1;
}

int list_variants(const Device &dv, int *vec, int *minb, int max) {
    int n = 0;
    for (const Variant &v : kVariants)
        if (v.precision == dv.precision && (v.fits ? v.fits(dv.dom.nx) : dv.dom.nx % v.vec == 0) && n < max) {
            vec[n] = v.vec;
            minb[n] = v.minb;
            ++n;
        }
    return n;
}

void launch_stream_collide(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const Variant *v = find_variant(dv.precision, dv.vec, dv.minb);
    if (!v) v = find_variant(dv.precision, 1, 0);
    v->fn(dv, sp, s);
}

void launch_boundary_fix(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    switch (dv.precision) {
    case 0: launch_boundary<double>(dv, sp, s); break;
    case 1: launch_boundary<float>(dv, sp, s); break;
    case 2: launch_boundary<__half>(dv, sp, s); break;
    default: launch_boundary<__nv_bfloat16>(dv, sp, s); break;
    }
}

// ---- overlapped steps: the near tiles -----------------------------------------

namespace {

// one listed near tile of the step a block (TILE_X threads, one cell each):
// the bulk kernel's arithmetic on the cells whose flag byte is zero or solid
// (the same bits as any launch shape of it)
template <typename T>
__global__ void __launch_bounds__(TILE_X) near_bulk_kernel(const Device dv, const StepPtrs sp) {
    if ((int)blockIdx.x >= dv.near_count[sp.parity]) return;
    const int t = dv.near_list[sp.parity][blockIdx.x];
    const int ntx = (dv.dom.nx + TILE_X - 1) / TILE_X;
    const int row = t / ntx;
    const Blk bk{t % ntx, row % dv.dom.ny, row / dv.dom.ny, ntx, dv.dom.ny, dv.dom.nz};
    StepPtrs own = sp;
    own.far_skip = nullptr;
    bulk_body<T, 1, TILE_X, 1>(dv, own, bk);
}

}  // namespace

void launch_near_bulk(const Device &dv, const StepPtrs &sp, cudaStream_t s) {
    const unsigned blocks = (unsigned)dv.near_cap;
    switch (dv.precision) {
    case 0: near_bulk_kernel<double><<<blocks, TILE_X, 0, s>>>(dv, sp); break;
    case 1: near_bulk_kernel<float><<<blocks, TILE_X, 0, s>>>(dv, sp); break;
    case 2: near_bulk_kernel<__half><<<blocks, TILE_X, 0, s>>>(dv, sp); break;
    default: near_bulk_kernel<__nv_bfloat16><<<blocks, TILE_X, 0, s>>>(dv, sp); break;
    }
}

// ---- batched launches (ensembles) ------------------------------------------

namespace {

constexpr int BATCH_BX = 32, BATCH_BY = 8;      // 256 threads a block, a plane's cells in row order

template <typename T, int V, int MINB = 1>
void bulk_batch_launch(const Batch &bt, unsigned blocks, cudaStream_t s) {
    if constexpr (sizeof(T) == 2 && V % 2 == 0)
        bulk16_batch<T, V, BATCH_BX, BATCH_BY, MINB><<<blocks, dim3(BATCH_BX, BATCH_BY), 0, s>>>(bt);
    else
        bulk_batch<T, V, BATCH_BX, BATCH_BY, MINB><<<blocks, dim3(BATCH_BX, BATCH_BY), 0, s>>>(bt);
}

struct BatchShape {
    int precision, vec;
    void (*fn)(const Batch &, unsigned, cudaStream_t);
};

// per precision, index 0 and 1 are one and two cells a thread (the
// untuned choice is 1, else 0), two cells with the registers capped for 3
// resident blocks an SM in FP32 (the compiler's own choice leaves room for
// two); the shapes after them cap the registers for 3 or 4 resident blocks
// (those that spill little at the cap)
const BatchShape kBatchShapes[] = {
    {0, 1, bulk_batch_launch<double, 1>},  {0, 2, bulk_batch_launch<double, 2>},
    {1, 1, bulk_batch_launch<float, 1>},   {1, 2, bulk_batch_launch<float, 2, 3>},
    {1, 4, bulk_batch_launch<float, 4>},   {1, 2, bulk_batch_launch<float, 2, 4>},
    {2, 1, bulk_batch_launch<__half, 1>},  {2, 2, bulk_batch_launch<__half, 2>},
    {2, 4, bulk_batch_launch<__half, 4>},  {2, 2, bulk_batch_launch<__half, 2, 4>},
    {2, 4, bulk_batch_launch<__half, 4, 3>},
    {3, 1, bulk_batch_launch<__nv_bfloat16, 1>}, {3, 2, bulk_batch_launch<__nv_bfloat16, 2>},
    {3, 4, bulk_batch_launch<__nv_bfloat16, 4>}, {3, 2, bulk_batch_launch<__nv_bfloat16, 2, 4>},
    {3, 4, bulk_batch_launch<__nv_bfloat16, 4, 3>},
};

const BatchShape *batch_shape(int precision, int i) {
    for (const BatchShape &b : kBatchShapes)
        if (b.precision == precision && i-- == 0) return &b;
    return nullptr;
}

}  // namespace

int batch_bulk_shape(int precision, int i) {
    const BatchShape *b = batch_shape(precision, i);
    return b ? b->vec : 0;
}

void batch_grid_cells(const Device &dv, int k, int variant, int g[3]) {
    g[0] = g[1] = g[2] = 0;
    const Domain &d = dv.dom;
    if (k == BK_BOUNDARY && dv.nb > 0) {
        const long long side = dv.remap_side;
        g[0] = (int)((dv.nb * side * side * side + 255) / 256);
        g[1] = g[2] = 1;
    } else if (k == BK_WALLS && !(d.px && d.py && d.pz)) {
        const long long nx = d.nx, ny = d.ny, nz = d.nz;
        const long long area = std::max(ny * nz, std::max(nx * nz, nx * ny));
        g[0] = (int)((area + 255) / 256);
        g[1] = 6;
        g[2] = 1;
    } else if (k == BK_BULK) {
        const BatchShape *b = batch_shape(dv.precision, variant);
        if (!b || d.nx % b->vec) return;
        // a z-plane's V-cell groups in row order (no lanes idle at row ends),
        // BATCH_PZ planes a block
        g[0] = (int)(((long long)(d.nx / b->vec) * d.ny + BATCH_BX * BATCH_BY - 1) / (BATCH_BX * BATCH_BY));
        g[1] = 1;
        g[2] = (d.nz + BATCH_PZ - 1) / BATCH_PZ;
    }
}

void launch_batch_cells(int k, int variant, const Batch &bt, unsigned blocks, int precision, cudaStream_t s) {
    if (blocks == 0) return;
    if (k == BK_BULK) {
        const BatchShape *b = batch_shape(precision, variant);
        if (b) b->fn(bt, blocks, s);
        return;
    }
    const int mode = k == BK_WALLS ? 1 : 0;
    switch (precision) {
    case 0: boundary_batch<double><<<blocks, 256, 0, s>>>(bt, mode); break;
    case 1: boundary_batch<float><<<blocks, 256, 0, s>>>(bt, mode); break;
    case 2: boundary_batch<__half><<<blocks, 256, 0, s>>>(bt, mode); break;
    default: boundary_batch<__nv_bfloat16><<<blocks, 256, 0, s>>>(bt, mode); break;
    }
}

bool needs_boundary_fix(const Device &dv) {
    return dv.nb > 0 || !(dv.dom.px && dv.dom.py && dv.dom.pz);
}

}  // namespace lbm
