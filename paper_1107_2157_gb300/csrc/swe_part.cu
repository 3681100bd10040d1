// swe_part.cu -- one grid split into px x py partitions: the 2D domain
// decomposition a multi-GPU run would use (Sec. 4.1 and Fig. 1 lay out MPI
// partitions of the global array with their halos), all held on the current
// device.  Each partition stores its cells with a one-cell ghost ring.  A
// step is two launches over all partitions:
//   1. halo: every ghost cell next to another partition copies that
//      partition's edge cell; a ghost cell on the global boundary is the
//      reflective mirror of its own edge cell (h and the tangential momentum
//      copied, the normal momentum negated); corners are never read;
//   2. step: the Lax-Wendroff step of Sec. 3 on every interior cell: the
//      single-grid kernel's TMA tile + halo staging and strip routine
//      (swe_tile.cuh), in its ghosted mode -- the box's halo is the ghost
//      ring, so no wall is formed inside the kernel.
// Plane layout: (ny + 2) rows; the interior starts at column 4 (16-byte
// aligned, as TMA needs), column 3 is the left ghost, column nx + 4 the
// right ghost; rows 0 and ny + 1 are the bottom and top ghosts.
// A mirrored ghost fed through make_cell gives exactly the mirrored cell the
// single-grid kernels form in registers ((-u)(-u/h) = u(u/h) and
// (-u)(v/h) = -(u v/h) are exact), so the partitioned run gives the
// single-grid bits for every split.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include <mutex>

#include "swe_tile.cuh"

namespace swe {

enum { SIDE_L = 0, SIDE_R = 1, SIDE_B = 2, SIDE_T = 3 };

struct PartDev {
    float *buf[2];    // three ghosted planes each: (ny + 2) rows of pitch floats
    long long pitch;  // >= nx + 8, a multiple of 32 floats
    long long plane;  // pitch * (ny + 2)
    int nx, ny;       // interior cells
    int nbr[4];       // neighbouring partition on each side, -1 = global wall,
                      // -2 = another rank's partition (ghosts written by the caller)
};

// Cell (i, j) of partition P in ghosted coordinates: i = 0 and i = nx + 1
// are the left and right ghosts, j = 0 and j = ny + 1 the bottom and top.
__device__ __forceinline__ float *cellp(const PartDev &P, int b, int f, int i, int j)
{
    return P.buf[b] + f * P.plane + (long long)j * P.pitch + i + 3;
}

// One thread per ghost cell of one partition (sides L, R: ny cells each;
// B, T: nx cells each), grid-stride over all partitions.
__global__ void part_halo_kernel(const PartDev *__restrict__ parts, int n_parts, const long long *__restrict__ first,
                                 long long total, int b)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        // partition p owns ghost indices [first[p], first[p+1])
        int lo = 0, hi = n_parts - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const PartDev &P = parts[lo];
        int k = (int)(e - first[lo]);
        int side;
        if (k < P.ny) side = SIDE_L;
        else if ((k -= P.ny) < P.ny) side = SIDE_R;
        else if ((k -= P.ny) < P.nx) side = SIDE_B;
        else { k -= P.nx; side = SIDE_T; }
        int gi, gj, si, sj;  // ghost cell and the cell it copies (in the source partition)
        if (side == SIDE_L) { gi = 0; gj = k + 1; }
        else if (side == SIDE_R) { gi = P.nx + 1; gj = k + 1; }
        else if (side == SIDE_B) { gi = k + 1; gj = 0; }
        else { gi = k + 1; gj = P.ny + 1; }
        const int nb = P.nbr[side];
        if (nb == -2) continue;  // filled by the caller from the neighbouring rank
        float h, u, v;
        if (nb >= 0) {
            const PartDev &Q = parts[nb];
            if (side == SIDE_L) { si = Q.nx; sj = k + 1; }
            else if (side == SIDE_R) { si = 1; sj = k + 1; }
            else if (side == SIDE_B) { si = k + 1; sj = Q.ny; }
            else { si = k + 1; sj = 1; }
            h = *cellp(Q, b, 0, si, sj);
            u = *cellp(Q, b, 1, si, sj);
            v = *cellp(Q, b, 2, si, sj);
        } else {
            si = side == SIDE_L ? 1 : (side == SIDE_R ? P.nx : gi);
            sj = side == SIDE_B ? 1 : (side == SIDE_T ? P.ny : gj);
            h = *cellp(P, b, 0, si, sj);
            u = *cellp(P, b, 1, si, sj);
            v = *cellp(P, b, 2, si, sj);
            if (side == SIDE_L || side == SIDE_R) u = -u; else v = -v;
        }
        *cellp(P, b, 0, gi, gj) = h;
        *cellp(P, b, 1, gi, gj) = u;
        *cellp(P, b, 2, gi, gj) = v;
    }
}

// Edge strips of a single partition (a rank's), packed side by side:
// [left: h, hu, hv over ny rows][right: same][bottom: h, hu, hv over nx
// columns][top: same].  Offsets of a side's strip in that layout:
__host__ __device__ __forceinline__ long long strip_offset(int side, int nx, int ny)
{
    return side <= SIDE_R ? (long long)side * 3 * ny : 6LL * ny + (long long)(side - SIDE_B) * 3 * nx;
}

// edges[] <- the partition's interior cells along each side (to_ghosts =
// false), or the ghost ring of the sides in ``sides`` <- ghosts[] (true).
__global__ void part_strips_kernel(PartDev P, int b, float *__restrict__ strips, int sides, bool to_ghosts)
{
    const long long total = 6LL * P.ny + 6LL * P.nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int side = e < 6LL * P.ny ? (int)(e / (3LL * P.ny)) : SIDE_B + (int)((e - 6LL * P.ny) / (3LL * P.nx));
        const int len = side <= SIDE_R ? P.ny : P.nx;
        const long long r = e - strip_offset(side, P.nx, P.ny);
        const int f = (int)(r / len), k = (int)(r % len);
        int ei, ej, gi, gj;  // edge cell and ghost cell
        if (side == SIDE_L) { ei = 1; gi = 0; ej = gj = k + 1; }
        else if (side == SIDE_R) { ei = P.nx; gi = P.nx + 1; ej = gj = k + 1; }
        else if (side == SIDE_B) { ej = 1; gj = 0; ei = gi = k + 1; }
        else { ej = P.ny; gj = P.ny + 1; ei = gi = k + 1; }
        if (to_ghosts) {
            if (sides & (1 << side)) *cellp(P, b, f, gi, gj) = strips[e];
        } else {
            strips[e] = *cellp(P, b, f, ei, ej);
        }
    }
}

using PartCfg = TiledCfg<float, 4, 8>;  // 128 x 32 cells per CTA, as the single-grid kernel

// One CTA per tile of one partition (blockIdx.z); tiles past the
// partition's size exit.  maps: three per buffer per partition, over the
// ghosted planes (nx + 5 columns, ny + 2 rows).
__global__ void __launch_bounds__(128) part_tiled_kernel(const PartDev *__restrict__ parts,
                                                         const CUtensorMap *__restrict__ maps, int b, Coef<float> k,
                                                         int *err)
{
    using C = PartCfg;
    const PartDev &P = parts[blockIdx.z];
    const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
    if (x0 >= P.nx || y0 >= P.ny) return;
    extern __shared__ __align__(128) unsigned char smem[];
    float *sH = reinterpret_cast<float *>(smem);
    float *sU = reinterpret_cast<float *>(smem + C::BOX_STRIDE);
    float *sV = reinterpret_cast<float *>(smem + 2 * C::BOX_STRIDE);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 3 * C::BOX_STRIDE);
    if (threadIdx.x == 0) {
        const CUtensorMap *m = maps + ((size_t)blockIdx.z * 2 + b) * 3;
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(bar, (uint32_t)(3 * C::BOX_BYTES));
        // interior (x0, y0) is ghosted column x0 + 4, row y0 + 1: the box
        // origin (x0 - AX, y0 - 1) of the single-grid kernel is (x0, y0) here
        tma_load_2d(sH, m + 0, bar, x0, y0);
        tma_load_2d(sU, m + 1, bar, x0, y0);
        tma_load_2d(sV, m + 2, bar, x0, y0);
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait_bounded(bar, 0, err))) return;
    float *o = P.buf[b ^ 1] + P.pitch + 4;  // interior origin of the output
    tiled_compute<float, 4, 8, false, 1, true>(sH, sU, sV, o, o + P.plane, o + 2 * P.plane, P.nx, P.ny, P.pitch, x0,
                                               y0, k);
}

}  // namespace swe

using namespace swe;

struct swe_part {
    int nx = 0, ny = 0, px = 0, py = 0;
    Coef<float> k{};
    std::vector<int> xs, ys;  // partition bounds: x in [xs[a], xs[a+1]), y in [ys[b], ys[b+1])
    std::vector<PartDev> h_parts;
    PartDev *d_parts = nullptr;
    long long *d_first = nullptr;
    long long ghosts = 0;
    int max_nx = 0, max_ny = 0;
    float *pool = nullptr;
    CUtensorMap *d_maps = nullptr;
    int *d_err = nullptr;
    int cur = 0;
    long long launches = 0;
};

static swe_status pst(cudaError_t e)
{
    if (e == cudaSuccess) return SWE_OK;
    return e == cudaErrorMemoryAllocation ? SWE_ENOMEM : SWE_ECUDA;
}

extern "C" {

void swe_part_destroy(swe_part *p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    cudaFree(p->pool);
    cudaFree(p->d_maps);
    cudaFree(p->d_err);
    cudaFree(p->d_parts);
    cudaFree(p->d_first);
    delete p;
}

swe_status swe_part_create(int nx, int ny, int px, int py, double dx, double dy, double dt, double g, swe_part **out)
{
    if (!out) return SWE_EINVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || px < 1 || py < 1 || px > nx || py > ny || px * py > 4096)
        return SWE_EINVAL;
    for (double v : {dx, dy, dt, g})
        if (!(v > 0.0) || !std::isfinite(v)) return SWE_EINVAL;
    swe_part *p = new (std::nothrow) swe_part();
    if (!p) return SWE_ENOMEM;
    auto fail = [&](swe_status s) {
        swe_part_destroy(p);
        return s;
    };
    p->nx = nx;
    p->ny = ny;
    p->px = px;
    p->py = py;
    p->k = make_coef<float>(dx, dy, dt, g);
    for (int a = 0; a <= px; ++a) p->xs.push_back((int)((long long)a * nx / px));
    for (int b = 0; b <= py; ++b) p->ys.push_back((int)((long long)b * ny / py));
    const int n = px * py;
    std::vector<long long> offs;
    long long at = 0;
    for (int b = 0; b < py; ++b)
        for (int a = 0; a < px; ++a) {
            PartDev d{};
            d.nx = p->xs[a + 1] - p->xs[a];
            d.ny = p->ys[b + 1] - p->ys[b];
            d.pitch = ((long long)d.nx + 8 + 31) / 32 * 32;
            d.plane = d.pitch * (d.ny + 2);
            d.nbr[SIDE_L] = a > 0 ? b * px + a - 1 : -1;
            d.nbr[SIDE_R] = a + 1 < px ? b * px + a + 1 : -1;
            d.nbr[SIDE_B] = b > 0 ? (b - 1) * px + a : -1;
            d.nbr[SIDE_T] = b + 1 < py ? (b + 1) * px + a : -1;
            p->max_nx = std::max(p->max_nx, d.nx);
            p->max_ny = std::max(p->max_ny, d.ny);
            offs.push_back(at);
            at += 6 * d.plane;  // two buffers x three planes
            at = (at + 63) / 64 * 64;
            p->h_parts.push_back(d);
        }
    swe_status s;
    if ((s = pst(cudaMalloc(&p->pool, (size_t)at * sizeof(float)))) != SWE_OK) return fail(s);
    if ((s = pst(cudaMemset(p->pool, 0, (size_t)at * sizeof(float)))) != SWE_OK) return fail(s);
    std::vector<long long> first;
    for (int i = 0; i < n; ++i) {
        PartDev &d = p->h_parts[i];
        d.buf[0] = p->pool + offs[i];
        d.buf[1] = d.buf[0] + 3 * d.plane;
        first.push_back(p->ghosts);
        p->ghosts += 2LL * d.nx + 2LL * d.ny;
    }
    first.push_back(p->ghosts);
    {
        int bw, bh;
        tiled_box(SWE_F32, &bw, &bh);
        std::vector<CUtensorMap> maps((size_t)n * 6);
        for (int i = 0; i < n; ++i)
            for (int b = 0; b < 2; ++b)
                for (int f = 0; f < 3; ++f) {
                    const PartDev &d = p->h_parts[i];
                    if (!encode_plane_map(&maps[((size_t)i * 2 + b) * 3 + f], SWE_F32, d.buf[b] + f * d.plane,
                                          d.nx + 5, d.ny + 2, d.pitch, bw, bh))
                        return fail(SWE_ECUDA);
                }
        if ((s = pst(cudaMalloc(&p->d_maps, maps.size() * sizeof(CUtensorMap)))) != SWE_OK) return fail(s);
        if ((s = pst(cudaMemcpy(p->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice))) !=
            SWE_OK)
            return fail(s);
        if ((s = pst(cudaMalloc(&p->d_err, sizeof(int)))) != SWE_OK) return fail(s);
        if ((s = pst(cudaMemset(p->d_err, 0, sizeof(int)))) != SWE_OK) return fail(s);
    }
    if ((s = pst(cudaMalloc(&p->d_parts, n * sizeof(PartDev)))) != SWE_OK) return fail(s);
    if ((s = pst(cudaMemcpy(p->d_parts, p->h_parts.data(), n * sizeof(PartDev), cudaMemcpyHostToDevice))) != SWE_OK)
        return fail(s);
    if ((s = pst(cudaMalloc(&p->d_first, first.size() * sizeof(long long)))) != SWE_OK) return fail(s);
    if ((s = pst(cudaMemcpy(p->d_first, first.data(), first.size() * sizeof(long long), cudaMemcpyHostToDevice))) !=
        SWE_OK)
        return fail(s);
    *out = p;
    return SWE_OK;
}

static swe_status part_copy(swe_part *p, void *const *user, long long ld, bool to_dev, cudaStream_t s)
{
    if (!p || ld < p->nx) return SWE_EINVAL;
    for (int f = 0; f < 3; ++f)
        if (!user[f]) return SWE_EINVAL;
    for (int b = 0; b < p->py; ++b)
        for (int a = 0; a < p->px; ++a) {
            const PartDev &d = p->h_parts[b * p->px + a];
            for (int f = 0; f < 3; ++f) {
                float *dev = d.buf[p->cur] + f * d.plane + d.pitch + 4;  // the first interior cell
                float *usr = static_cast<float *>(user[f]) + (long long)p->ys[b] * ld + p->xs[a];
                const size_t w = (size_t)d.nx * sizeof(float);
                const cudaError_t e =
                    to_dev ? cudaMemcpy2DAsync(dev, d.pitch * sizeof(float), usr, ld * sizeof(float), w, d.ny,
                                               cudaMemcpyDefault, s)
                           : cudaMemcpy2DAsync(usr, ld * sizeof(float), dev, d.pitch * sizeof(float), w, d.ny,
                                               cudaMemcpyDefault, s);
                if (e != cudaSuccess) return pst(e);
            }
        }
    return SWE_OK;
}

swe_status swe_part_set_state(swe_part *p, const float *h, const float *hu, const float *hv, long long ld,
                              void *stream)
{
    void *u[3] = {const_cast<float *>(h), const_cast<float *>(hu), const_cast<float *>(hv)};
    return part_copy(p, u, ld, true, static_cast<cudaStream_t>(stream));
}

swe_status swe_part_get_state(swe_part *p, float *h, float *hu, float *hv, long long ld, void *stream)
{
    void *u[3] = {h, hu, hv};
    return part_copy(p, u, ld, false, static_cast<cudaStream_t>(stream));
}

swe_status swe_part_step(swe_part *p, int n_steps, void *stream)
{
    if (!p || n_steps < 0) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = p->px * p->py;
    const dim3 sgrid((p->max_nx + PartCfg::TX - 1) / PartCfg::TX, (p->max_ny + PartCfg::TY - 1) / PartCfg::TY, n);
    const int hblocks = (int)std::min<long long>((p->ghosts + 255) / 256, 4096);
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(part_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PartCfg::SMEM);
    });
    if (attr != cudaSuccess) return pst(attr);
    for (int i = 0; i < n_steps; ++i) {
        part_halo_kernel<<<hblocks, 256, 0, s>>>(p->d_parts, n, p->d_first, p->ghosts, p->cur);
        part_tiled_kernel<<<sgrid, 128, PartCfg::SMEM, s>>>(p->d_parts, p->d_maps, p->cur, p->k, p->d_err);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return pst(e);
        p->cur ^= 1;
        p->launches += 2;
    }
    return SWE_OK;
}

swe_status swe_part_create_rank(int nx, int ny, int walls, double dx, double dy, double dt, double g,
                                swe_part **out)
{
    if (!out) return SWE_EINVAL;
    *out = nullptr;
    if (walls < 0 || walls > 15) return SWE_EINVAL;
    swe_part *p = nullptr;
    swe_status s = swe_part_create(nx, ny, 1, 1, dx, dy, dt, g, &p);
    if (s != SWE_OK) return s;
    PartDev &d = p->h_parts[0];
    for (int side = 0; side < 4; ++side) d.nbr[side] = (walls & (1 << side)) ? -1 : -2;
    if ((s = pst(cudaMemcpy(p->d_parts, p->h_parts.data(), sizeof(PartDev), cudaMemcpyHostToDevice))) != SWE_OK) {
        swe_part_destroy(p);
        return s;
    }
    *out = p;
    return SWE_OK;
}

static swe_status part_strips(swe_part *p, float *strips, int sides, bool to_ghosts, cudaStream_t s)
{
    if (!p || !strips || p->px * p->py != 1 || sides < 0 || sides > 15) return SWE_EINVAL;
    const PartDev &d = p->h_parts[0];
    const long long total = 6LL * d.ny + 6LL * d.nx;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 1024);
    part_strips_kernel<<<blocks, 256, 0, s>>>(d, p->cur, strips, sides, to_ghosts);
    return pst(cudaGetLastError());
}

swe_status swe_part_edges(swe_part *p, float *edges, void *stream)
{
    return part_strips(p, edges, 15, false, static_cast<cudaStream_t>(stream));
}

swe_status swe_part_set_ghosts(swe_part *p, const float *ghosts, int sides, void *stream)
{
    return part_strips(p, const_cast<float *>(ghosts), sides, true, static_cast<cudaStream_t>(stream));
}

swe_status swe_part_query(swe_part *p, int key, long long *value)
{
    if (!p || !value) return SWE_EINVAL;
    switch (key) {
        case SWE_PQ_PARTS: *value = (long long)p->px * p->py; break;
        case SWE_PQ_HALO_CELLS: *value = p->ghosts; break;
        case SWE_PQ_LAUNCHES: *value = p->launches; break;
        case SWE_PQ_ERROR: {
            int word = 0;
            if (cudaMemcpy(&word, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SWE_ECUDA;
            *value = word;
            break;
        }
        default: return SWE_EINVAL;
    }
    return SWE_OK;
}

}  // extern "C"
