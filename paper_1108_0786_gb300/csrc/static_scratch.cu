// static_scratch.cu -- momentum-exchange force and torque per body for
// callers that cannot allocate device memory.
//
// This is a variant of the force kernel of kernels.cu.  The regular step
// keeps its link lists and per-block partial sums in memory the handle
// allocates; here the caller passes only its inputs (post-collision
// populations, the obstacle-cell field, body states) and its output, and
// the per-block partial sums go to a file-scope device array of fixed size.
// No cudaMalloc, cudaFree or allocating library routine is called.
//
// The array is shared by every call on a device and keeps the contents of
// the last call: each call writes every record it later reads, so nothing
// has to start at zero, but two calls that overlap on the GPU (for example
// on two streams) race on the array and give wrong results.
#include <mutex>

#include <cuda.h>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;

// per-block partial sums (6 doubles each), LBM_STATIC_SCRATCH_RECORDS records
static __device__ __align__(256) double g_force_partials[LBM_STATIC_SCRATCH_RECORDS * 6];

std::mutex g_setup_mutex;
struct ScratchAddr {
    unsigned long long ctx_id;  // context the address belongs to (0: none yet)
    double *addr;
};
ScratchAddr g_partials_addr[NA_MAX_DEVICES] = {};

// Identifier of the current context, from the driver through the runtime's
// entry-point lookup (no link against the driver library); 0 if the driver
// does not offer it.
unsigned long long current_context_id() {
    typedef CUresult (*GetCurrent)(CUcontext *);
    typedef CUresult (*GetId)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the array in the current context.  Host code cannot use
// the symbol itself as a device pointer; the address is looked up once per
// device with that device current, and again whenever the device's context
// has changed (after cudaDeviceReset the module is loaded anew, possibly at
// another address).  Without a context identifier (no context current yet,
// or a driver without the query) it is looked up on every call.
cudaError_t partials_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchAddr &slot = g_partials_addr[dev];
    if (id == 0 || slot.ctx_id != id || !slot.addr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_force_partials);
        if (e != cudaSuccess) return e;
        slot.addr = static_cast<double *>(p);
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return cudaSuccess;
}

// Cells the scan covers along one axis: the cube's side, or the whole axis
// when a periodic axis is shorter than the side (a wrapped cube would visit
// its cells twice and add their links twice).
inline int scan_extent(int side, int n, int periodic) { return periodic && n < side ? n : side; }

// Block (k, b): cells k*256 .. of the box of extents (sx, sy, sz) that
// starts at floor(X_b) - hw (the cube of side 2 hw + 1 around floor(X_b),
// cut to one period on short periodic axes); every fluid cell adds the
// links (x_f, a) whose end x_f + e_a is a cell of body b (Eq. hydroF,
// torque about the body centre at the link midpoint), and the block writes
// its fixed-order sum to record b * blocks + k.
__global__ void __launch_bounds__(NA_THREADS)
static_partials_kernel(const double *pop, const uint8_t *flags, const double *bodies, Domain d, int hw,
                       int sx, int sy, int sz, int blocks, double *partials) {
    const int b = blockIdx.y, k = blockIdx.x;
    BodyState sb;
    {
        const double *s = bodies + 13 * b;
        for (int i = 0; i < 3; ++i) { sb.X[i] = s[i]; sb.V[i] = s[7 + i]; sb.W[i] = s[10 + i]; }
        for (int i = 0; i < 4; ++i) sb.q[i] = s[3 + i];
    }
    const long long l = (long long)k * NA_THREADS + threadIdx.x;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if (l < (long long)sx * sy * sz) {
        int x = (int)floor(sb.X[0]) - hw + (int)(l % sx);
        int y = (int)floor(sb.X[1]) - hw + (int)((l / sx) % sy);
        int z = (int)floor(sb.X[2]) - hw + (int)(l / ((long long)sx * sy));
        bool ok = true;
        if (d.px) x = ((x % d.nx) + d.nx) % d.nx; else ok = ok && x >= 0 && x < d.nx;
        if (d.py) y = ((y % d.ny) + d.ny) % d.ny; else ok = ok && y >= 0 && y < d.ny;
        if (d.pz) z = ((z % d.nz) + d.nz) % d.nz; else ok = ok && z >= 0 && z < d.nz;
        const long long c = ((long long)z * d.ny + y) * d.nx + x;
        if (ok && flags[c] == 0) {
            double rho = -1.0;
            for (int a = 1; a < Q; ++a) {
                int nx_ = x + ex(a), ny_ = y + ey(a), nz_ = z + ez(a);
                if ((!d.px && (nx_ < 0 || nx_ >= d.nx)) || (!d.py && (ny_ < 0 || ny_ >= d.ny)) ||
                    (!d.pz && (nz_ < 0 || nz_ >= d.nz)))
                    continue;
                nx_ = wrap_axis(nx_, d.nx); ny_ = wrap_axis(ny_, d.ny); nz_ = wrap_axis(nz_, d.nz);
                if (flags[((long long)nz_ * d.ny + ny_) * d.nx + nx_] != b + 1) continue;
                if (rho < 0) {
                    rho = 0.0;
                    for (int q = 0; q < Q; ++q) rho += pop[q * d.C + c];
                }
                double u[3];
                surface_velocity(d, sb, x + ex(a), y + ey(a), z + ez(a), u);
                const double eu = -(ex(a) * u[0] + ey(a) * u[1] + ez(a) * u[2]);
                const double mag = 2.0 * pop[a * d.C + c] + 6.0 * wgt(a) * rho * eu;
                const double fl[3] = {ex(a) * mag, ey(a) * mag, ez(a) * mag};
                double o[3];
                offset_from(d, sb, x + 0.5 * ex(a), y + 0.5 * ey(a), z + 0.5 * ez(a), o);
                acc[0] += fl[0]; acc[1] += fl[1]; acc[2] += fl[2];
                acc[3] += o[1] * fl[2] - o[2] * fl[1];
                acc[4] += o[2] * fl[0] - o[0] * fl[2];
                acc[5] += o[0] * fl[1] - o[1] * fl[0];
            }
        }
    }
    __shared__ double part[NA_THREADS / 32][6];
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
            double v = lane < NA_THREADS / 32 ? part[lane][i] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) partials[((long long)b * blocks + k) * 6 + i] = v;
        }
    }
}

// thread b adds its records in block order
__global__ void static_sum_kernel(const double *partials, int nb, int blocks, double *out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    for (int i = 0; i < 6; ++i) {
        double v = 0.0;
        for (int k = 0; k < blocks; ++k) v += partials[((long long)b * blocks + k) * 6 + i];
        out[b * 6 + i] = v;
    }
}

}  // namespace
}  // namespace lbm

#pragma GCC visibility push(default)
extern "C" int lbm_momentum_exchange_static(const double *pop, const unsigned char *flags, const double *bodies,
                                            int nb, int nx, int ny, int nz, int bc, int half_width, double *out,
                                            void *stream) {
    if (!pop || !flags || !bodies || !out) return LBM_E_ARG;
    if (nb < 1 || nb > LBM_MAX_BODIES || nx < 1 || ny < 1 || nz < 1 || bc < 0 || bc > 7) return LBM_E_ARG;
    const long long C = (long long)nx * ny * nz;
    if (C > (1LL << 31) - 1) return LBM_E_ARG;
    if (half_width < 1 || half_width > LBM_STATIC_SCRATCH_MAX_HALF_WIDTH) return LBM_E_ARG;
    const int side = 2 * half_width + 1;
    const int sx = lbm::scan_extent(side, nx, bc & 1), sy = lbm::scan_extent(side, ny, bc & 2),
              sz = lbm::scan_extent(side, nz, bc & 4);
    const int blocks = (int)(((long long)sx * sy * sz + lbm::NA_THREADS - 1) / lbm::NA_THREADS);
    if ((long long)blocks * nb > LBM_STATIC_SCRATCH_RECORDS) return LBM_E_ARG;
    double *partials = nullptr;
    if (lbm::partials_address(&partials) != cudaSuccess) return LBM_E_CUDA;
    const lbm::Domain d{nx, ny, nz, (bc & 1) ? 1 : 0, (bc & 2) ? 1 : 0, (bc & 4) ? 1 : 0, C,
                        1.0 / nx, 1.0 / ny, 1.0 / nz};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lbm::static_partials_kernel<<<dim3(blocks, nb), lbm::NA_THREADS, 0, s>>>(pop, flags, bodies, d, half_width,
                                                                            sx, sy, sz, blocks, partials);
    lbm::static_sum_kernel<<<(nb + 127) / 128, 128, 0, s>>>(partials, nb, blocks, out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}
#pragma GCC visibility pop
