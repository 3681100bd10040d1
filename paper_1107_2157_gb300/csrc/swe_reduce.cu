// swe_reduce.cu -- FP64 reductions over a state plane: the mass
// sum(h) dx dy and the CFL time step (Sec. 3).
//
// Both run in two launches: a fixed grid of kRedBlocks blocks writes one
// FP64 partial per block to a scratch buffer, then one block combines the
// partials in a fixed order.  The assignment of cells to threads and the
// combining tree depend only on (nx, ny), so results are bitwise
// reproducible.  The CFL per-cell terms use explicitly rounded FP64
// operations (no contraction), so the minimum is the exact minimum of
// correctly rounded per-cell bounds.
#include "swe_device.cuh"

namespace swe {

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

size_t reduce_scratch_doubles() { return 2 * (size_t)kRedBlocks + 16; }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum / min; every thread gets the result.
template <bool MIN>
__device__ double block_reduce(double v)
{
    __shared__ double part[32];
    v = MIN ? warp_min(v) : warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (lane < nw) ? part[lane] : (MIN ? __longlong_as_double(0x7ff0000000000000ll) : 0.0);
    v = MIN ? warp_min(v) : warp_sum(v);
    __syncthreads();
    return v;
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) mass_partial_kernel(const T *__restrict__ H, int nx, int ny,
                                                                   long long pitch, double *partial)
{
    double s = 0.0;
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
        const T *row = H + (size_t)j * (size_t)pitch;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) s += (double)row[i];
    }
    s = block_reduce<false>(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) sum_final_kernel(const double *partial, int n, double scale, double *out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    s = block_reduce<false>(s);
    if (threadIdx.x == 0) out[0] = s * scale;
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) cfl_partial_kernel(const T *__restrict__ H, const T *__restrict__ U,
                                                                  const T *__restrict__ V, int nx, int ny,
                                                                  long long pitch, double dx, double dy, double g,
                                                                  double *pmin, double *pbad)
{
    double best = __longlong_as_double(0x7ff0000000000000ll);  // +inf
    double bad = 0.0;
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
        const size_t ro = (size_t)j * (size_t)pitch;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const double h = (double)H[ro + i];
            const double u = (double)U[ro + i];
            const double v = (double)V[ro + i];
            if (!(h > 0.0) || !isfinite(h) || !isfinite(u) || !isfinite(v)) {
                bad += 1.0;
                continue;
            }
            const double c = __dsqrt_rn(__dmul_rn(g, h));
            const double tx = __ddiv_rn(dx, __dadd_rn(c, fabs(__ddiv_rn(u, h))));
            const double ty = __ddiv_rn(dy, __dadd_rn(c, fabs(__ddiv_rn(v, h))));
            best = fmin(best, fmin(tx, ty));
        }
    }
    best = block_reduce<true>(best);
    bad = block_reduce<false>(bad);
    if (threadIdx.x == 0) {
        pmin[blockIdx.x] = best;
        pbad[blockIdx.x] = bad;
    }
}

__global__ void __launch_bounds__(1024) cfl_final_kernel(const double *pmin, const double *pbad, int n, double cfl,
                                                         double *out)
{
    double best = __longlong_as_double(0x7ff0000000000000ll);
    double bad = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        best = fmin(best, pmin[i]);
        bad += pbad[i];
    }
    best = block_reduce<true>(best);
    bad = block_reduce<false>(bad);
    if (threadIdx.x == 0) {
        out[0] = __dmul_rn(cfl, best);
        out[1] = bad;
    }
}

static int red_blocks(int ny) { return ny < kRedBlocks ? ny : kRedBlocks; }

cudaError_t launch_mass(int dtype, const void *H, int nx, int ny, long long pitch, double dxdy, double *scratch,
                        double *out_dev, cudaStream_t s)
{
    const int nb = red_blocks(ny);
    if (dtype == SWE_F64)
        mass_partial_kernel<double><<<nb, kRedThreads, 0, s>>>(static_cast<const double *>(H), nx, ny, pitch, scratch);
    else
        mass_partial_kernel<float><<<nb, kRedThreads, 0, s>>>(static_cast<const float *>(H), nx, ny, pitch, scratch);
    sum_final_kernel<<<1, 1024, 0, s>>>(scratch, nb, dxdy, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_cfl(int dtype, const void *H, const void *U, const void *V, int nx, int ny, long long pitch,
                       double dx, double dy, double g, double cfl, double *scratch, double *out_dev, cudaStream_t s)
{
    const int nb = red_blocks(ny);
    double *pmin = scratch, *pbad = scratch + kRedBlocks;
    if (dtype == SWE_F64)
        cfl_partial_kernel<double><<<nb, kRedThreads, 0, s>>>(static_cast<const double *>(H),
                                                              static_cast<const double *>(U),
                                                              static_cast<const double *>(V), nx, ny, pitch, dx, dy, g,
                                                              pmin, pbad);
    else
        cfl_partial_kernel<float><<<nb, kRedThreads, 0, s>>>(static_cast<const float *>(H),
                                                             static_cast<const float *>(U),
                                                             static_cast<const float *>(V), nx, ny, pitch, dx, dy, g,
                                                             pmin, pbad);
    cfl_final_kernel<<<1, 1024, 0, s>>>(pmin, pbad, nb, cfl, out_dev);
    return cudaGetLastError();
}

}  // namespace swe

// ---------------------------------------------------------------------------
// swe_mass_noalloc: the mass reduction above with its partial sums in a
// file-scope device array instead of a context's cudaMalloc'd scratch, for
// callers that may not allocate device memory.
// ---------------------------------------------------------------------------
#include <mutex>

namespace swe {

// One partial sum per block of mass_partial_kernel (at most kRedBlocks).
static __device__ __align__(256) double g_noalloc_partials[kRedBlocks];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device, looked up
// once per device.  In host code the array's name is only a host-side
// stand-in, so the kernels must be given this address.
static cudaError_t noalloc_partials(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace swe

extern "C" swe_status swe_mass_noalloc(int dtype, const void *h, int nx, int ny, long long ld, double dx, double dy,
                                       double *mass_dev, void *stream)
{
    using namespace swe;
    if (dtype != SWE_F32 && dtype != SWE_F64) return SWE_EINVAL;
    if (!h || !mass_dev) return SWE_EINVAL;
    if (nx < 1 || ny < 1 || nx > SWE_NOALLOC_MAX_DIM || ny > SWE_NOALLOC_MAX_DIM || ld < nx) return SWE_EINVAL;
    if (!(dx > 0.0) || !(dy > 0.0) || !isfinite(dx) || !isfinite(dy)) return SWE_EINVAL;
    double *partials = nullptr;
    cudaError_t e = noalloc_partials(&partials);
    if (e != cudaSuccess) return SWE_ECUDA;
    // every partial the final kernel reads is written first: nothing to clear
    e = launch_mass(dtype, h, nx, ny, ld, dx * dy, partials, mass_dev, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SWE_OK : SWE_ECUDA;
}
