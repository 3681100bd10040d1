// swe_reduce.cu -- FP64 reductions over a state plane: the mass
// sum(h) dx dy and the CFL time step (Sec. 3).
//
// A launch reduces one grid or many (blockIdx.y = instance): a fixed number
// of blocks per grid writes one FP64 partial per block to a scratch buffer,
// then one block per grid combines that grid's partials in a fixed order.
// The assignment of cells to threads and the combining tree depend only on
// the grid's size and the block count, so results are bitwise reproducible.
// The CFL per-cell terms use explicitly rounded FP64 operations (no
// contraction), so the minimum is the exact minimum of correctly rounded
// per-cell bounds.
//
// GB300 runs FP64 arithmetic at a small fraction of its FP32 and integer
// rates, so the FP32 reductions keep FP64 operations off the per-cell path:
// the mass sums FP32 depths exactly in 64-bit integers (ExactSum32) and the
// CFL step screens cells with FP32 estimates before any FP64 evaluation.
#include <algorithm>

#include "swe_device.cuh"
#include "swe_exact_sum.h"

namespace swe {

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

size_t reduce_scratch_doubles() { return 5 * (size_t)kRedBlocks + 32; }

// Scratch needed to reduce n grids with B blocks each.
size_t reduce_scratch_doubles_many(int n, int B) { return 5 * (size_t)n * (size_t)B + 6 * (size_t)n + 16; }

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

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reduction (sum, or min / max of non-negative values when MIN /
// MAX is set); every thread gets the result.
template <bool MIN, bool MAX = false>
__device__ double block_reduce(double v)
{
    __shared__ double part[32];
    v = MIN ? warp_min(v) : (MAX ? warp_max(v) : warp_sum(v));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (lane < nw) ? part[lane] : (MIN ? __longlong_as_double(0x7ff0000000000000ll) : 0.0);
    v = MIN ? warp_min(v) : (MAX ? warp_max(v) : warp_sum(v));
    __syncthreads();
    return v;
}

// Fetches the grid this block reduces: the by-value one, or grids[blockIdx.y].
template <bool MANY>
__device__ __forceinline__ RedGrid red_grid(const RedGrid &one, const RedGrid *__restrict__ many)
{
    if (MANY) return many[blockIdx.y];
    return one;
}

// Streams the 16-byte vectors of NP FP32 planes over the rows of block b
// (rows b, b + B, ...; rows 16-byte aligned), Q vectors per thread and plane
// per round.  The next round's loads are issued before the current round is
// used, so the arithmetic runs under the memory latency.  f receives one
// vector of each plane; the row tails (nx % 4 cells) are left to the caller.
template <int NP, int Q, typename F>
__device__ __forceinline__ void stream_rows4(const float *const (&P)[NP], long long pitch, int nx, int ny, int b,
                                             int B, F &&f)
{
    const int T = blockDim.x, tid = threadIdx.x;
    const int nv = nx / 4, per_round = Q * T;
    const int rpr = (nv + per_round - 1) / per_round;  // rounds per row
    const int rows = b < ny ? (ny - 1 - b) / B + 1 : 0;
    const int n = rows * rpr;
    float4 A[NP][Q], Z[NP][Q];
    auto load = [&](int i, float4(&buf)[NP][Q]) {
        const int k = i / rpr, c = i - k * rpr;
        const size_t ro = (size_t)(b + (size_t)k * B) * (size_t)pitch;
        const int v0 = c * per_round + tid;
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int v = v0 + q * T;
                buf[p][q] = v < nv ? __ldg(reinterpret_cast<const float4 *>(P[p] + ro) + v) : make_float4(0, 0, 0, 0);
            }
    };
    auto use = [&](int i, const float4(&buf)[NP][Q]) {
        const int v0 = (i % rpr) * per_round + tid;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (v0 + q * T >= nv) continue;
            if constexpr (NP == 1)
                f(buf[0][q]);
            else
                f(buf[0][q], buf[1][q], buf[2][q]);
        }
    };
    if (n > 0) load(0, A);
    int i = 0;
    for (; i + 1 < n; i += 2) {
        load(i + 1, Z);
        use(i, A);
        if (i + 2 < n) load(i + 2, A);
        use(i + 1, Z);
    }
    if (i < n) use(i, A);
}

// Mass partials.  Each block takes rows blockIdx.x, blockIdx.x + gridDim.x,
// ...; with VEC the threads read 16-byte vectors (4 FP32 / 2 FP64 values,
// the row base and stride being 16-byte aligned) -- FP32 through
// stream_rows4, four per thread per round -- and the row tail scalar.  FP32
// depths are summed exactly (ExactSum32); FP64 depths in two FP64
// accumulators per thread.
template <typename T, bool VEC, bool MANY>
__global__ void __launch_bounds__(kRedThreads) mass_partial_kernel(RedGrid one, const RedGrid *__restrict__ many,
                                                                   double *partial)
{
    constexpr int N = 16 / sizeof(T);
    constexpr bool F32 = sizeof(T) == 4;
    const RedGrid G = red_grid<MANY>(one, many);
    const T *H = static_cast<const T *>(G.h);
    double s0 = 0.0, s1 = 0.0;
    ExactSum32 ex;
    if constexpr (F32 && VEC) {
        const float *planes[1] = {static_cast<const float *>(G.h)};
        stream_rows4<1, 4>(planes, G.pitch, G.nx, G.ny, blockIdx.x, gridDim.x,
                           [&](const float4 &x) { ex.add4(x.x, x.y, x.z, x.w); });
    }
    for (int j = blockIdx.x; j < G.ny; j += gridDim.x) {
        const T *row = H + (size_t)j * (size_t)G.pitch;
        int i0 = 0;
        if (F32 && VEC) {
            i0 = (G.nx / 4) * 4;
        } else if (VEC) {
            const int nv = G.nx / N;
            for (int v0 = threadIdx.x; v0 < nv; v0 += 4 * blockDim.x) {
                if constexpr (F32) {
                    float4 x[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int v = v0 + q * blockDim.x;
                        x[q] = v < nv ? __ldg(reinterpret_cast<const float4 *>(row) + v) : make_float4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (v0 + q * (int)blockDim.x < nv) ex.add4(x[q].x, x[q].y, x[q].z, x[q].w);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int v = v0 + q * blockDim.x;
                        if (v < nv) {
                            const double2 x = __ldg(reinterpret_cast<const double2 *>(row) + v);
                            s0 += (double)x.x;
                            s1 += (double)x.y;
                        }
                    }
                }
            }
            i0 = nv * N;
        }
        for (int i = i0 + threadIdx.x; i < G.nx; i += blockDim.x) {
            if constexpr (F32)
                ex.add1((float)row[i]);
            else
                s0 += (double)row[i];
        }
    }
    const double s = block_reduce<false>(F32 ? ex.value() : s0 + s1);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// One block per grid: out[2*g] = (sum of the grid's B partials) * dx * dy.
template <bool MANY>
__global__ void __launch_bounds__(1024) sum_final_kernel(RedGrid one, const RedGrid *__restrict__ many,
                                                         const double *partial, int B, double *out)
{
    const RedGrid G = MANY ? many[blockIdx.x] : one;
    const double *p = partial + (size_t)blockIdx.x * B;
    double s = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) s += p[i];
    s = block_reduce<false>(s);
    if (threadIdx.x == 0) out[2 * (size_t)blockIdx.x] = s * G.dx * G.dy;
}

// ---------------------------------------------------------------------------
// CFL time step.  dt = cfl * min over cells of min(dx / sx, dy / sy) with
// sx = sqrt(g h) + |hu / h|, sy = sqrt(g h) + |hv / h|, all FP64.  A correctly
// rounded division is monotone, so min over cells of fl(dx / sx) equals
// fl(dx / max sx): only the exact FP64 maxima Sx, Sy are needed.  GB300's
// FP64 units are slow, so pass 1 finds FP32 estimates of the maxima (relative
// error far below 2^-16) and pass 2 evaluates the exact FP64 sx, sy only for
// cells whose estimate lies within 2^-16 of the estimated maximum; no other
// cell can hold the maximum.  A thread reuses its last exact value when it
// meets the same (h, momentum) bits again, so flat regions cost one FP64
// evaluation per thread.
//
// Pass 2 splits each block's rows into S column chunks, one CTA each, so
// the few blocks that hold candidates are read by S CTAs in parallel; the
// exact maxima meet in one slot per grid through an atomic maximum on their
// bit patterns (non-negative doubles order as unsigned integers), which
// gives the same result in any order.
//
// The blocks of a grid that hold candidates are listed by the pass-1 final
// kernel, and pass 2 runs a fixed, small grid of CTAs over the items (listed
// block, column chunk) of that list.
//
// Scratch layout for n grids of B blocks (P = n*B doubles per array):
// [0,P) ax  [P,2P) ay  [2P,3P) bad  [3P,3P+3n) thresholds (thx, thy, bad)
// [3P+3n, 3P+5n) exact (sx, sy) maxima per grid
// [3P+5n, 4P+5n) candidate blocks of each grid (B slots per grid)
// [4P+5n, 4P+6n) the number of candidates of each grid.
// ---------------------------------------------------------------------------
constexpr float kCflSlack = 1.0f / 65536.0f;

// Depth not positive, or a value not finite (checked in the data's own type).
template <typename T>
__device__ __forceinline__ bool cell_bad(T h, T u, T v)
{
    return !(h > T(0)) || !isfinite(h) || !isfinite(u) || !isfinite(v);
}

// FP32 estimate of a cell's sx and sy (pass 1 and the pass-2 screen use
// this one function: explicitly rounded operations, the same bits in both).
__device__ __forceinline__ void cfl_estimate(float h, float u, float v, float g32, float &ex, float &ey)
{
    const float inv = rcp(h);
    const float c = __fsqrt_rn(__fmul_rn(g32, h));
    ex = __fadd_rn(c, fabsf(__fmul_rn(u, inv)));
    ey = __fadd_rn(c, fabsf(__fmul_rn(v, inv)));
}

// Visits every cell of the block's rows (rows blockIdx.x, blockIdx.x +
// gridDim.x, ...) in the data's own type.  With VEC (FP32 planes, 16-byte
// aligned rows) a thread loads two 16-byte vectors of each plane at a time
// and takes the row tail one cell at a time.
// ``b`` and ``B`` (the row blocks) replace blockIdx.x and gridDim.x, and the
// visit covers column chunk ``sc`` of ``S`` equal chunks of each row.
template <typename T, bool VEC, typename F>
__device__ __forceinline__ void for_cells(const RedGrid &G, F &&f, int b = -1, int B = 0, int sc = 0, int S = 1)
{
    const T *H = static_cast<const T *>(G.h), *U = static_cast<const T *>(G.u), *V = static_cast<const T *>(G.v);
    if (b < 0) {
        b = blockIdx.x;
        B = gridDim.x;
    }
    for (int j = b; j < G.ny; j += B) {
        const size_t ro = (size_t)j * (size_t)G.pitch;
        if constexpr (VEC && sizeof(T) == 4) {
            const float4 *h4 = reinterpret_cast<const float4 *>(H + ro);
            const float4 *u4 = reinterpret_cast<const float4 *>(U + ro);
            const float4 *v4 = reinterpret_cast<const float4 *>(V + ro);
            const int nv_all = G.nx / 4, cw = (nv_all + S - 1) / S;
            const int nv = min(nv_all, (sc + 1) * cw);
            for (int v0 = sc * cw + threadIdx.x; v0 < nv; v0 += 2 * blockDim.x) {
                float4 a[2], b[2], c[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int k = v0 + q * blockDim.x;
                    if (k < nv) {
                        a[q] = __ldg(h4 + k);
                        b[q] = __ldg(u4 + k);
                        c[q] = __ldg(v4 + k);
                    }
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (v0 + q * (int)blockDim.x < nv) {
                        f(a[q].x, b[q].x, c[q].x);
                        f(a[q].y, b[q].y, c[q].y);
                        f(a[q].z, b[q].z, c[q].z);
                        f(a[q].w, b[q].w, c[q].w);
                    }
                }
            }
            if (sc == S - 1)
                for (int i = nv_all * 4 + threadIdx.x; i < G.nx; i += blockDim.x) f(H[ro + i], U[ro + i], V[ro + i]);
        } else {
            const int cw = (G.nx + S - 1) / S;
            const int i1 = min(G.nx, (sc + 1) * cw);
            for (int i = sc * cw + threadIdx.x; i < i1; i += blockDim.x) f(H[ro + i], U[ro + i], V[ro + i]);
        }
    }
}

template <typename T, bool VEC, bool MANY>
__global__ void __launch_bounds__(kRedThreads) cfl_pass1_kernel(RedGrid one, const RedGrid *__restrict__ many,
                                                                float g32, double *scratch)
{
    const RedGrid G = red_grid<MANY>(one, many);
    const size_t P = (size_t)gridDim.x * gridDim.y;
    float ax = 0.0f, ay = 0.0f;
    double bad = 0.0;
    auto cell = [&](T h, T u, T v) {
        if (cell_bad<T>(h, u, v)) {
            bad += 1.0;
            return;
        }
        float ex, ey;
        cfl_estimate((float)h, (float)u, (float)v, g32, ex, ey);
        ax = fmaxf(ax, ex);
        ay = fmaxf(ay, ey);
    };
    if constexpr (VEC && sizeof(T) == 4) {
        const float *planes[3] = {static_cast<const float *>(G.h), static_cast<const float *>(G.u),
                                  static_cast<const float *>(G.v)};
        stream_rows4<3, 2>(planes, G.pitch, G.nx, G.ny, blockIdx.x, gridDim.x,
                           [&](const float4 &h, const float4 &u, const float4 &v) {
                               cell(h.x, u.x, v.x);
                               cell(h.y, u.y, v.y);
                               cell(h.z, u.z, v.z);
                               cell(h.w, u.w, v.w);
                           });
        const T *H = static_cast<const T *>(G.h), *U = static_cast<const T *>(G.u), *V = static_cast<const T *>(G.v);
        for (int j = blockIdx.x; j < G.ny; j += gridDim.x) {
            const size_t ro = (size_t)j * (size_t)G.pitch;
            for (int i = (G.nx / 4) * 4 + threadIdx.x; i < G.nx; i += blockDim.x) cell(H[ro + i], U[ro + i], V[ro + i]);
        }
    } else {
        for_cells<T, VEC>(G, cell);
    }
    ax = (float)block_reduce<false, true>((double)ax);
    ay = (float)block_reduce<false, true>((double)ay);
    bad = block_reduce<false, false>(bad);
    if (threadIdx.x == 0) {
        const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        scratch[b] = ax;
        scratch[P + b] = ay;
        scratch[2 * P + b] = bad;
    }
}

// One block per grid: the pass-2 thresholds of grid blockIdx.x.
__global__ void __launch_bounds__(1024) cfl_pass1_final_kernel(double *scratch, int n, int B)
{
    const size_t P = (size_t)n * B;
    const size_t o = (size_t)blockIdx.x * B;
    double ax = 0.0, ay = 0.0, bad = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        ax = fmax(ax, scratch[o + i]);
        ay = fmax(ay, scratch[P + o + i]);
        bad += scratch[2 * P + o + i];
    }
    ax = block_reduce<false, true>(ax);
    ay = block_reduce<false, true>(ay);
    bad = block_reduce<false, false>(bad);
    if (threadIdx.x == 0) {
        // a non-finite or tiny estimate disables the screen (every cell exact)
        double *th = scratch + 3 * P + 3 * (size_t)blockIdx.x;
        th[0] = (isfinite(ax) && ax > 1e-30) ? ax * (1.0 - (double)kCflSlack) : -1.0;
        th[1] = (isfinite(ay) && ay > 1e-30) ? ay * (1.0 - (double)kCflSlack) : -1.0;
        th[2] = bad;
        double *ex = scratch + 3 * P + 3 * (size_t)n + 2 * (size_t)blockIdx.x;
        ex[0] = 0.0;
        ex[1] = 0.0;
    }
    // the candidate list, with pass 2's screen: a block whose maxima lie
    // below both FP32 thresholds holds no candidate
    __shared__ int count;
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    const double *th = scratch + 3 * P + 3 * (size_t)blockIdx.x;
    const float thx = __double2float_rd(th[0]), thy = __double2float_rd(th[1]);
    double *list = scratch + 3 * P + 5 * (size_t)n + o;
    for (int i = threadIdx.x; i < B; i += blockDim.x)
        if (!((float)scratch[o + i] < thx && (float)scratch[P + o + i] < thy)) list[atomicAdd(&count, 1)] = (double)i;
    __syncthreads();
    if (threadIdx.x == 0) scratch[4 * P + 5 * (size_t)n + blockIdx.x] = (double)count;
}

// Exact FP64 sx or sy of one cell, every operation correctly rounded.
__device__ __forceinline__ double exact_speed(double g, double h, double m)
{
    return __dadd_rn(__dsqrt_rn(__dmul_rn(g, h)), fabs(__ddiv_rn(m, h)));
}

// Pass 2: the CTAs of grid blockIdx.y stride over the items (candidate
// block, column chunk) of that grid's list: item i is chunk i % S of the
// rows of listed block list[i / S].  Blocks not listed hold no candidate.
template <typename T, bool VEC, bool MANY>
__global__ void __launch_bounds__(kRedThreads) cfl_pass2_kernel(RedGrid one, const RedGrid *__restrict__ many,
                                                                float g32, double g, double *scratch, int B, int S)
{
    const RedGrid G = red_grid<MANY>(one, many);
    const size_t n = gridDim.y;
    const size_t P = (size_t)B * n;
    const double *th = scratch + 3 * P + 3 * (size_t)blockIdx.y;
    const double *list = scratch + 3 * P + 5 * n + (size_t)blockIdx.y * B;
    const int items = (int)scratch[4 * P + 5 * n + blockIdx.y] * S;
    // thresholds as floats rounded toward -inf: the screen keeps every
    // candidate the FP64 threshold keeps, and compares in FP32
    const float thx = __double2float_rd(th[0]), thy = __double2float_rd(th[1]);
    double sx = 0.0, sy = 0.0;
    if ((int)blockIdx.x >= items) return;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int rb = (int)list[it / S], sc = it % S;
        T lhx = T(-1), lux = T(0), lhy = T(-1), lvy = T(0);  // last exactly evaluated inputs
        double lsx = 0.0, lsy = 0.0;
        for_cells<T, VEC>(G, [&](T h, T u, T v) {
            if (cell_bad<T>(h, u, v)) return;
            float ex, ey;
            cfl_estimate((float)h, (float)u, (float)v, g32, ex, ey);
            if (ex >= thx) {
                if (!(h == lhx && u == lux)) {
                    lhx = h;
                    lux = u;
                    lsx = exact_speed(g, (double)h, (double)u);
                }
                sx = fmax(sx, lsx);
            }
            if (ey >= thy) {
                if (!(h == lhy && v == lvy)) {
                    lhy = h;
                    lvy = v;
                    lsy = exact_speed(g, (double)h, (double)v);
                }
                sy = fmax(sy, lsy);
            }
        }, rb, B, sc, S);
    }
    sx = block_reduce<false, true>(sx);
    sy = block_reduce<false, true>(sy);
    if (threadIdx.x == 0) {
        unsigned long long *ex = reinterpret_cast<unsigned long long *>(scratch + 3 * P + 3 * n + 2 * (size_t)blockIdx.y);
        atomicMax(ex, (unsigned long long)__double_as_longlong(sx));
        atomicMax(ex + 1, (unsigned long long)__double_as_longlong(sy));
    }
}

// One block per grid: out[2g] = dt of grid g, out[2g+1] = its bad-cell count.
template <bool MANY>
__global__ void __launch_bounds__(1024) cfl_final_kernel(RedGrid one, const RedGrid *__restrict__ many,
                                                         const double *scratch, int n, int B, double cfl,
                                                         double *out)
{
    const RedGrid G = MANY ? many[blockIdx.x] : one;
    const size_t P = (size_t)n * B;
    if (threadIdx.x == 0) {
        const double sx = scratch[3 * P + 3 * (size_t)n + 2 * (size_t)blockIdx.x];
        const double sy = scratch[3 * P + 3 * (size_t)n + 2 * (size_t)blockIdx.x + 1];
        const double tx = __ddiv_rn(G.dx, sx), ty = __ddiv_rn(G.dy, sy);
        out[2 * (size_t)blockIdx.x] = __dmul_rn(cfl, fmin(tx, ty));
        out[2 * (size_t)blockIdx.x + 1] = scratch[3 * P + 3 * (size_t)blockIdx.x + 2];
    }
}

static int red_blocks(int ny) { return ny < kRedBlocks ? ny : kRedBlocks; }

// Blocks of a single-grid reduction: one resident wave of ``kern`` (SMs x
// CTAs per SM at kRedThreads threads), at most kRedBlocks and one per row.
// A ragged second wave measured slower than a single wave with more rows per
// block.  The results do not depend on the count: the CFL maxima are order
// free and the mass partials are exact sums.
template <typename K>
static int one_wave(K kern, int ny)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 0;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRedThreads, 0) != cudaSuccess || occ < 1 ||
        sms < 1)
        return red_blocks(ny);
    return std::min(red_blocks(ny), sms * occ);
}

static bool plane_vec_ok(const void *H, long long pitch, size_t es)
{
    return ((uintptr_t)H % 16 == 0) && (((size_t)pitch * es) % 16 == 0);
}

template <typename T, bool MANY>
static void mass_launch(const RedGrid &one, const RedGrid *many, int n, int B, bool vec, double *scratch,
                        double *out, cudaStream_t s)
{
    const dim3 grid(B, n);
    if (vec)
        mass_partial_kernel<T, true, MANY><<<grid, kRedThreads, 0, s>>>(one, many, scratch);
    else
        mass_partial_kernel<T, false, MANY><<<grid, kRedThreads, 0, s>>>(one, many, scratch);
    sum_final_kernel<MANY><<<n, 1024, 0, s>>>(one, many, scratch, B, out);
}

cudaError_t launch_mass(int dtype, const void *H, int nx, int ny, long long pitch, double dxdy, double *scratch,
                        double *out_dev, cudaStream_t s)
{
    RedGrid one{H, nullptr, nullptr, pitch, nx, ny, dxdy, 1.0};
    const size_t es = dtype == SWE_F64 ? 8 : 4;
    const bool vec = plane_vec_ok(H, pitch, es);
    if (dtype == SWE_F64)
        mass_launch<double, false>(one, nullptr, 1, one_wave(mass_partial_kernel<double, true, false>, ny), vec,
                                   scratch, out_dev, s);
    else
        mass_launch<float, false>(one, nullptr, 1, one_wave(mass_partial_kernel<float, true, false>, ny), vec,
                                  scratch, out_dev, s);
    return cudaGetLastError();
}

cudaError_t launch_mass_many(const RedGrid *grids_dev, int n, int B, double *scratch, double *out_dev,
                             cudaStream_t s)
{
    // batched planes are FP32 with 128-byte aligned rows
    RedGrid none{};
    mass_launch<float, true>(none, grids_dev, n, B, true, scratch, out_dev, s);
    return cudaGetLastError();
}

template <typename T, bool VEC, bool MANY>
static void cfl_launch(const RedGrid &one, const RedGrid *many, int n, int B, double g, double cfl, double *scratch,
                       double *out, cudaStream_t s)
{
    const dim3 grid(B, n);
    const float g32 = (float)g;
    cfl_pass1_kernel<T, VEC, MANY><<<grid, kRedThreads, 0, s>>>(one, many, g32, scratch);
    cfl_pass1_final_kernel<<<n, 1024, 0, s>>>(scratch, n, B);
    // column chunks of about 1024 cells (at most 8) for a single grid; a
    // fixed grid of CTAs per reduced grid strides over the candidate items
    const int S = MANY ? 1 : std::max(1, std::min(8, one.nx / 1024));
    const int ctas = MANY ? 8 : 256;
    cfl_pass2_kernel<T, VEC, MANY><<<dim3(ctas, n), kRedThreads, 0, s>>>(one, many, g32, g, scratch, B, S);
    cfl_final_kernel<MANY><<<n, 32, 0, s>>>(one, many, scratch, n, B, cfl, out);
}

cudaError_t launch_cfl(int dtype, const void *H, const void *U, const void *V, int nx, int ny, long long pitch,
                       double dx, double dy, double g, double cfl, double *scratch, double *out_dev, cudaStream_t s)
{
    RedGrid one{H, U, V, pitch, nx, ny, dx, dy};
    if (dtype == SWE_F64)
        cfl_launch<double, false, false>(one, nullptr, 1, one_wave(cfl_pass1_kernel<double, false, false>, ny), g,
                                         cfl, scratch, out_dev, s);
    else if (plane_vec_ok(H, pitch, 4) && plane_vec_ok(U, pitch, 4) && plane_vec_ok(V, pitch, 4))
        cfl_launch<float, true, false>(one, nullptr, 1, one_wave(cfl_pass1_kernel<float, true, false>, ny), g, cfl,
                                       scratch, out_dev, s);
    else
        cfl_launch<float, false, false>(one, nullptr, 1, one_wave(cfl_pass1_kernel<float, false, false>, ny), g,
                                        cfl, scratch, out_dev, s);
    return cudaGetLastError();
}

cudaError_t launch_cfl_many(const RedGrid *grids_dev, int n, int B, double g, double cfl, double *scratch,
                            double *out_dev, cudaStream_t s)
{
    // batched planes are FP32 with 128-byte aligned rows
    RedGrid none{};
    cfl_launch<float, true, true>(none, grids_dev, n, B, g, cfl, scratch, out_dev, s);
    return cudaGetLastError();
}

// Step coefficients on the device from a CFL result res = (dt, bad-cell
// count) (swe_run): make_coef<T> in the host's FP64 operations, so the bits
// are those the host would pass; skip is set when a cell was bad.
template <typename T>
__global__ void coef_from_cfl_kernel(const double *res, double dx, double dy, double g, DevCoef<T> *kd)
{
    kd->k = make_coef<T>(dx, dy, res[0], g);
    kd->skip = res[1] != 0.0 ? 1 : 0;
}

cudaError_t launch_coef_from_cfl(int dtype, const double *res_dev, double dx, double dy, double g, void *kd,
                                 cudaStream_t s)
{
    if (dtype == SWE_F64)
        coef_from_cfl_kernel<double><<<1, 1, 0, s>>>(res_dev, dx, dy, g, static_cast<DevCoef<double> *>(kd));
    else
        coef_from_cfl_kernel<float><<<1, 1, 0, s>>>(res_dev, dx, dy, g, static_cast<DevCoef<float> *>(kd));
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
