// swe_packed.cu -- the packed-state variant of the one-step kernel: each
// cell's (h, hu, hv) is stored as one 16-byte vector (h, hu, hv, 0) instead
// of in three planes -- the packing Sec. 5 credits for the speed of its
// hand-optimised OpenCL kernel.  One TMA box per tile, one 16-byte load per
// cell; 32 bytes of HBM traffic per cell-update against the planes' 24.
// The same strip routine and face/update functions as the plane kernels
// (swe_tile.cuh), so the same bits.  FP32 only.
#include <mutex>

#include "swe_tile.cuh"

namespace swe {

using PackedCfg = TiledCfg<float, 4, 8>;  // 128 x 32 cells per CTA, 4 warps
constexpr size_t kPackedBoxBytes = (size_t)PackedCfg::BW * PackedCfg::BH * 16;
constexpr size_t kPackedSmem = (kPackedBoxBytes + 127) / 128 * 128 + 128;

__global__ void __launch_bounds__(128) lw_packed_kernel(const __grid_constant__ CUtensorMap m, float4 *__restrict__ out,
                                                        int nx, int ny, long long ppitch, Coef<float> k, int *err,
                                                        const DevCoef<float> *kd)
{
    if (!take_dev_coef(kd, k)) return;
    using C = PackedCfg;
    constexpr int VX = C::VX;
    extern __shared__ __align__(128) unsigned char smem[];
    const float4 *box = reinterpret_cast<const float4 *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (kPackedBoxBytes + 127) / 128 * 128);
    const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(bar, (uint32_t)kPackedBoxBytes);
        tma_load_3d(smem, &m, bar, 0, x0 - C::AX, y0 - 1);
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait_bounded(bar, 0, err))) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cx = lane * VX, gx = x0 + cx;
    const int rb = warp * C::ROWS, re = min(rb + C::ROWS, ny - y0);
    auto store = [&](int r, const float(&oh)[VX], const float(&ou)[VX], const float(&ov)[VX]) {
        if (gx < nx) {
            // whole vectors: cells past nx land in the row padding (ppitch is a multiple of 8 cells)
            float4 *o = out + (size_t)(y0 + r) * (size_t)ppitch + gx;
#pragma unroll
            for (int q = 0; q < VX; ++q) o[q] = make_float4(oh[q], ou[q], ov[q], 0.0f);
        }
    };
    if (x0 == 0 || x0 + C::TX >= nx)
        strip_compute_box<float, VX, true>(PackedBox{box}, C::BW, C::AX, 1, rb, re, cx, gx, nx, ny, y0, k, store);
    else
        strip_compute_box<float, VX, false>(PackedBox{box}, C::BW, C::AX, 1, rb, re, cx, gx, nx, ny, y0, k, store);
}

// (h, hu, hv) planes <-> packed cells, over the nx x ny interior.
__global__ void pack_state_kernel(const float *__restrict__ h, const float *__restrict__ u, const float *__restrict__ v,
                                  long long pitch, float4 *__restrict__ out, long long ppitch, int nx, int ny)
{
    const long long total = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long y = e / nx, x = e % nx, o = y * pitch + x;
        out[y * ppitch + x] = make_float4(h[o], u[o], v[o], 0.0f);
    }
}

__global__ void unpack_state_kernel(const float4 *__restrict__ in, long long ppitch, float *__restrict__ h,
                                    float *__restrict__ u, float *__restrict__ v, long long pitch, int nx, int ny)
{
    const long long total = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long y = e / nx, x = e % nx, o = y * pitch + x;
        const float4 c = in[y * ppitch + x];
        h[o] = c.x;
        u[o] = c.y;
        v[o] = c.z;
    }
}

void packed_box(int *bw, int *bh)
{
    *bw = PackedCfg::BW;
    *bh = PackedCfg::BH;
}

cudaError_t launch_packed(const CUtensorMap *map, void *out, int nx, int ny, long long ppitch, double dx, double dy,
                          double dt, double g, int *err, cudaStream_t s, const void *kd)
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(lw_packed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPackedSmem);
    });
    if (attr != cudaSuccess) return attr;
    const Coef<float> k = make_coef<float>(dx, dy, dt, g);
    const dim3 grid((nx + PackedCfg::TX - 1) / PackedCfg::TX, (ny + PackedCfg::TY - 1) / PackedCfg::TY);
    lw_packed_kernel<<<grid, 128, kPackedSmem, s>>>(*map, static_cast<float4 *>(out), nx, ny, ppitch, k, err,
                                                    static_cast<const DevCoef<float> *>(kd));
    return cudaGetLastError();
}

cudaError_t launch_pack(const void *h, const void *u, const void *v, long long pitch, void *out, long long ppitch,
                        int nx, int ny, bool unpack, cudaStream_t s)
{
    if (unpack)
        unpack_state_kernel<<<1184, 256, 0, s>>>(static_cast<const float4 *>(out), ppitch, (float *)h, (float *)u,
                                                 (float *)v, pitch, nx, ny);
    else
        pack_state_kernel<<<1184, 256, 0, s>>>(static_cast<const float *>(h), static_cast<const float *>(u),
                                               static_cast<const float *>(v), pitch, static_cast<float4 *>(out),
                                               ppitch, nx, ny);
    return cudaGetLastError();
}

}  // namespace swe
