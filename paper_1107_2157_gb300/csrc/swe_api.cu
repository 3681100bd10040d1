// swe_api.cu -- the C ABI of include/swe.h for single grids: context
// lifetime, state transfer, the step loop, the FP64 reductions.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "swe_device.cuh"
#include "swe_internal.h"

struct swe_ctx {
    int device = 0;
    int nx = 0, ny = 0;
    double dx = 1, dy = 1, dt = 0, g = 9.8;
    int dtype = SWE_F32;
    size_t esize = 4;
    long long pitch = 0;    // elements per row of a device plane
    size_t plane = 0;       // elements per plane (pitch * ny)
    unsigned char *state[2] = {nullptr, nullptr};  // three planes each
    int cur = 0;            // buffer holding the current state
    int kernel = SWE_KERNEL_AUTO;
    int depth = 1;
    int tb_variant = 0;         // two-step kernel shape
    CUtensorMap maps[2][3];     // TMA maps of both buffers, one-step box
    CUtensorMap maps_tb[2][3];  // TMA maps of both buffers, two-step box
    // SWE_KERNEL_PACKED: the state lives in packed[cur] ((h, hu, hv, 0) cells,
    // ppitch per row); the planes are a staging copy, stale after steps until
    // a transfer or a reduction unpacks them.
    void *packed[2] = {nullptr, nullptr};
    long long ppitch = 0;
    CUtensorMap maps_pk[2];
    bool planes_stale = false;
    double *scratch = nullptr;  // reduction partials (device)
    double *result = nullptr;   // reduction results (device, 4 doubles)
    double *host_result = nullptr;  // pinned copy of result
    int *err = nullptr;          // device error word
    void *kdev = nullptr;        // device DevCoef<T> (swe_run's step coefficients)
    long long launches = 0;
};

namespace swe {

static std::once_flag g_encode_once;
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool encode_plane_map(CUtensorMap *map, int dtype, const void *base, int nx, int ny, long long pitch, int box_x,
                      int box_y)
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return false;
    const size_t es = dtype == SWE_F64 ? 8 : 4;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * es};
    const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(map, dtype == SWE_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_packed_map(CUtensorMap *map, const void *base, int nx, int ny, long long ppitch, int box_x, int box_y)
{
    if (!g_encode) {
        CUtensorMap dummy;
        float one = 0.0f;
        (void)encode_plane_map(&dummy, SWE_F32, &one, 1, 1, 32, 4, 1);  // resolves the entry point
    }
    if (!g_encode) return false;
    const cuuint64_t dims[3] = {4, (cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[2] = {16, (cuuint64_t)ppitch * 16};
    const cuuint32_t box[3] = {4, (cuuint32_t)box_x, (cuuint32_t)box_y};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 5D map over a row-chunked bf16 activation tensor [N][H][CH][W][8]:
// dims {8, W, CH, H, N}; box {8, 130, CH, box_rows, 1}.
bool encode_act_map(CUtensorMap *map, const void *base, int W, int H, int CH, int N, int box_rows)
{
    if (!g_encode) {
        CUtensorMap dummy;
        float one = 0.0f;
        (void)encode_plane_map(&dummy, SWE_F32, &one, 1, 1, 32, 4, 1);  // resolves the entry point
    }
    if (!g_encode) return false;
    const cuuint64_t dims[5] = {8, (cuuint64_t)W, (cuuint64_t)CH, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[4] = {16, (cuuint64_t)W * 16, (cuuint64_t)CH * W * 16, (cuuint64_t)H * CH * W * 16};
    const cuuint32_t box[5] = {8, 130, (cuuint32_t)CH, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace swe

using namespace swe;

static swe_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return SWE_OK;
    if (e == cudaErrorMemoryAllocation) return SWE_ENOMEM;
    return SWE_ECUDA;
}

#define SWE_TRY(expr)                                  \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

static void *plane_ptr(swe_ctx *c, int buf, int k)
{
    return c->state[buf] + (size_t)k * c->plane * c->esize;
}

extern "C" {

void swe_options_init(swe_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->dtype = SWE_F32;
    opt->kernel = SWE_KERNEL_AUTO;
}

const char *swe_strerror(swe_status s)
{
    switch (s) {
        case SWE_OK: return "ok";
        case SWE_EINVAL: return "invalid argument";
        case SWE_ENOMEM: return "out of memory";
        case SWE_ECUDA: return "CUDA runtime error";
        case SWE_ETIMEOUT: return "device wait timed out";
        case SWE_ECHECK: return "mass or positivity check failed";
        case SWE_EUNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

void swe_destroy(swe_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    cudaFree(c->state[0]);
    cudaFree(c->state[1]);
    cudaFree(c->packed[0]);
    cudaFree(c->packed[1]);
    cudaFree(c->scratch);
    cudaFree(c->result);
    cudaFree(c->err);
    cudaFree(c->kdev);
    cudaFreeHost(c->host_result);
    delete c;
}

swe_status swe_create_ex(int nx, int ny, double dx, double dy, double dt, double g, const swe_options *opt,
                         swe_ctx **out)
{
    if (!out) return SWE_EINVAL;
    *out = nullptr;
    swe_options o;
    swe_options_init(&o);
    if (opt) o = *opt;
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536) return SWE_EINVAL;
    if (!finite_pos(dx) || !finite_pos(dy) || !finite_pos(dt) || !finite_pos(g)) return SWE_EINVAL;
    if (o.dtype != SWE_F32 && o.dtype != SWE_F64) return SWE_EINVAL;
    if (o.kernel < SWE_KERNEL_AUTO || o.kernel > SWE_KERNEL_PACKED) return SWE_EINVAL;
    if (o.kernel == SWE_KERNEL_PACKED && o.dtype != SWE_F32) return SWE_EUNSUPPORTED;
    if (o.depth < 0 || o.depth > 2) return SWE_EUNSUPPORTED;
    if (o.reserved[0] >= 8 && o.reserved[0] <= 9 && o.dtype != SWE_F32)
        return SWE_EUNSUPPORTED;  // streaming shapes 7 and 8 are FP32 only

    swe_ctx *c = new (std::nothrow) swe_ctx();
    if (!c) return SWE_ENOMEM;
    cudaGetDevice(&c->device);
    c->nx = nx;
    c->ny = ny;
    c->dx = dx;
    c->dy = dy;
    c->dt = dt;
    c->g = g;
    c->dtype = o.dtype;
    c->esize = o.dtype == SWE_F64 ? 8 : 4;
    c->pitch = plane_pitch(nx, c->esize);
    c->plane = (size_t)c->pitch * (size_t)ny;
    // AUTO: the fastest measured on GB300 at 8192^2: the streaming two-step
    // kernel for both.  FP32: 0.148 ms/step against 0.236 for the HBM-bound
    // one-step kernel; FP64 (bound by GB300's FP64 rate, so the gain is the
    // arithmetic the streaming layout does not repeat): 8.14 ms/step against
    // 11.06.
    c->kernel = o.kernel != SWE_KERNEL_AUTO ? o.kernel : SWE_KERNEL_TEMPORAL;
    c->depth = c->kernel == SWE_KERNEL_TEMPORAL ? 2 : 1;
    // two-step shape: streaming warps, 5 for FP32, 6 for FP64 (capped for 3
    // CTAs per SM: 8.14 ms/step against 8.80 uncapped at 2)
    c->tb_variant = (o.reserved[0] > 0 && o.reserved[0] <= 9) ? o.reserved[0] - 1 : (o.dtype == SWE_F32 ? 5 : 6);

    const size_t bytes = 3 * c->plane * c->esize;
    swe_status st = SWE_OK;
    auto fail = [&](swe_status s) {
        swe_destroy(c);
        return s;
    };
    if ((st = cuda_status(cudaMalloc(&c->state[0], bytes))) != SWE_OK) return fail(st);
    if ((st = cuda_status(cudaMalloc(&c->state[1], bytes))) != SWE_OK) return fail(st);
    // padding columns are never read as cells; zero them once for tidiness
    if ((st = cuda_status(cudaMemset(c->state[0], 0, bytes))) != SWE_OK) return fail(st);
    if ((st = cuda_status(cudaMemset(c->state[1], 0, bytes))) != SWE_OK) return fail(st);
    if ((st = cuda_status(cudaMalloc(&c->scratch, reduce_scratch_doubles() * sizeof(double)))) != SWE_OK)
        return fail(st);
    if ((st = cuda_status(cudaMalloc(&c->result, 4 * sizeof(double)))) != SWE_OK) return fail(st);
    if ((st = cuda_status(cudaMalloc(&c->err, sizeof(int)))) != SWE_OK) return fail(st);
    if ((st = cuda_status(cudaMalloc(&c->kdev, sizeof(swe::DevCoef<double>)))) != SWE_OK) return fail(st);
    if ((st = cuda_status(cudaMemset(c->err, 0, sizeof(int)))) != SWE_OK) return fail(st);
    if ((st = cuda_status(cudaMallocHost(&c->host_result, 4 * sizeof(double)))) != SWE_OK) return fail(st);

    if (c->kernel == SWE_KERNEL_PACKED) {
        c->ppitch = ((long long)nx + 7) / 8 * 8;  // 128-byte rows
        const size_t pbytes = (size_t)c->ppitch * ny * 16;
        int bw, bh;
        packed_box(&bw, &bh);
        for (int b = 0; b < 2; ++b) {
            if ((st = cuda_status(cudaMalloc(&c->packed[b], pbytes))) != SWE_OK) return fail(st);
            if ((st = cuda_status(cudaMemset(c->packed[b], 0, pbytes))) != SWE_OK) return fail(st);
            if (!encode_packed_map(&c->maps_pk[b], c->packed[b], nx, ny, c->ppitch, bw, bh)) return fail(SWE_ECUDA);
        }
    }
    if (c->kernel == SWE_KERNEL_TILED || c->kernel == SWE_KERNEL_TEMPORAL) {
        int bw, bh, tw, th;
        tiled_box(c->dtype, &bw, &bh);
        tb2_box(c->dtype, c->tb_variant, &tw, &th);
        for (int b = 0; b < 2; ++b)
            for (int k = 0; k < 3; ++k) {
                if (!encode_plane_map(&c->maps[b][k], c->dtype, plane_ptr(c, b, k), nx, ny, c->pitch, bw, bh))
                    return fail(SWE_ECUDA);
                if (!encode_plane_map(&c->maps_tb[b][k], c->dtype, plane_ptr(c, b, k), nx, ny, c->pitch, tw, th))
                    return fail(SWE_ECUDA);
            }
    }
    *out = c;
    return SWE_OK;
}

swe_status swe_create(int nx, int ny, double dx, double dy, double dt, double g, swe_ctx **out)
{
    return swe_create_ex(nx, ny, dx, dy, dt, g, nullptr, out);
}

swe_status swe_set_dt(swe_ctx *c, double dt)
{
    if (!c || !finite_pos(dt)) return SWE_EINVAL;
    c->dt = dt;
    return SWE_OK;
}

// Packed contexts: brings the plane copy of the current state up to date.
static cudaError_t sync_planes(swe_ctx *c, cudaStream_t s)
{
    if (c->kernel != SWE_KERNEL_PACKED || !c->planes_stale) return cudaSuccess;
    const cudaError_t e = launch_pack(plane_ptr(c, c->cur, 0), plane_ptr(c, c->cur, 1), plane_ptr(c, c->cur, 2),
                                      c->pitch, c->packed[c->cur], c->ppitch, c->nx, c->ny, true, s);
    if (e == cudaSuccess) c->planes_stale = false;
    return e;
}

static swe_status copy_planes(swe_ctx *c, void *const *user, long long ld, bool to_device, cudaStream_t s)
{
    if (ld < c->nx) return SWE_EINVAL;
    if (!to_device) SWE_TRY(sync_planes(c, s));
    for (int k = 0; k < 3; ++k)
        if (!user[k]) return SWE_EINVAL;
    for (int k = 0; k < 3; ++k) {
        void *dev = plane_ptr(c, c->cur, k);
        const size_t w = (size_t)c->nx * c->esize;
        if (to_device)
            SWE_TRY(cudaMemcpy2DAsync(dev, (size_t)c->pitch * c->esize, user[k], (size_t)ld * c->esize, w, c->ny,
                                      cudaMemcpyDefault, s));
        else
            SWE_TRY(cudaMemcpy2DAsync(user[k], (size_t)ld * c->esize, dev, (size_t)c->pitch * c->esize, w, c->ny,
                                      cudaMemcpyDefault, s));
    }
    if (to_device && c->kernel == SWE_KERNEL_PACKED) {
        SWE_TRY(launch_pack(plane_ptr(c, c->cur, 0), plane_ptr(c, c->cur, 1), plane_ptr(c, c->cur, 2), c->pitch,
                            c->packed[c->cur], c->ppitch, c->nx, c->ny, false, s));
        c->planes_stale = false;
    }
    return SWE_OK;
}

swe_status swe_set_state(swe_ctx *c, const void *h, const void *hu, const void *hv, long long ld, int on_device,
                         void *stream)
{
    (void)on_device;  // cudaMemcpyDefault resolves host vs device pointers
    if (!c) return SWE_EINVAL;
    void *p[3] = {const_cast<void *>(h), const_cast<void *>(hu), const_cast<void *>(hv)};
    return copy_planes(c, p, ld, true, static_cast<cudaStream_t>(stream));
}

swe_status swe_get_state(swe_ctx *c, void *h, void *hu, void *hv, long long ld, int on_device, void *stream)
{
    (void)on_device;
    if (!c) return SWE_EINVAL;
    void *p[3] = {h, hu, hv};
    return copy_planes(c, p, ld, false, static_cast<cudaStream_t>(stream));
}

// n_steps steps of the context's kernel on stream s; kd (optional) is the
// device DevCoef the kernels take their coefficients from instead of c->dt.
static swe_status step_launches(swe_ctx *c, int n_steps, cudaStream_t s, const void *kd)
{
    int n = 0;
    if (c->kernel == SWE_KERNEL_TEMPORAL) {
        for (; n + 2 <= n_steps; n += 2) {
            const int in = c->cur, outb = c->cur ^ 1;
            cudaError_t e = launch_tb2(c->dtype, c->tb_variant, c->maps_tb[in], c->state[outb], c->plane, c->nx,
                                       c->ny, c->pitch, c->dx, c->dy, c->dt, c->g, c->err, s, kd);
            if (e != cudaSuccess) return cuda_status(e);
            c->cur = outb;
            c->launches += 1;
        }
    }
    for (; n < n_steps; ++n) {
        const int in = c->cur, outb = c->cur ^ 1;
        cudaError_t e;
        if (c->kernel == SWE_KERNEL_PACKED) {
            e = launch_packed(&c->maps_pk[in], c->packed[outb], c->nx, c->ny, c->ppitch, c->dx, c->dy, c->dt, c->g,
                              c->err, s, kd);
            c->planes_stale = true;
        } else if (c->kernel == SWE_KERNEL_NAIVE)
            e = launch_naive(c->dtype, c->state[in], c->state[outb], c->plane, c->nx, c->ny, c->pitch, c->dx, c->dy,
                             c->dt, c->g, s, kd);
        else
            e = launch_tiled(c->dtype, c->maps[in], c->state[outb], c->plane, c->nx, c->ny, c->pitch, c->dx, c->dy,
                             c->dt, c->g, c->err, s, kd);
        if (e != cudaSuccess) return cuda_status(e);
        c->cur = outb;
        c->launches += 1;
    }
    return SWE_OK;
}

swe_status swe_step(swe_ctx *c, int n_steps, void *stream)
{
    if (!c || n_steps < 0) return SWE_EINVAL;
    return step_launches(c, n_steps, static_cast<cudaStream_t>(stream), nullptr);
}

swe_status swe_mass(swe_ctx *c, double *mass_out, void *stream)
{
    if (!c || !mass_out) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SWE_TRY(sync_planes(c, s));
    SWE_TRY(launch_mass(c->dtype, plane_ptr(c, c->cur, 0), c->nx, c->ny, c->pitch, c->dx * c->dy, c->scratch,
                        c->result, s));
    SWE_TRY(cudaMemcpyAsync(c->host_result, c->result, sizeof(double), cudaMemcpyDeviceToHost, s));
    SWE_TRY(cudaStreamSynchronize(s));
    *mass_out = c->host_result[0];
    return SWE_OK;
}

swe_status swe_cfl_dt(swe_ctx *c, double cfl, double *dt_out, void *stream)
{
    if (!c || !dt_out || !finite_pos(cfl)) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SWE_TRY(sync_planes(c, s));
    SWE_TRY(launch_cfl(c->dtype, plane_ptr(c, c->cur, 0), plane_ptr(c, c->cur, 1), plane_ptr(c, c->cur, 2), c->nx,
                       c->ny, c->pitch, c->dx, c->dy, c->g, cfl, c->scratch, c->result, s));
    SWE_TRY(cudaMemcpyAsync(c->host_result, c->result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SWE_TRY(cudaStreamSynchronize(s));
    if (c->host_result[1] != 0.0) {
        *dt_out = 0.0;
        return SWE_ECHECK;
    }
    *dt_out = c->host_result[0];
    return SWE_OK;
}

swe_status swe_run(swe_ctx *c, int n_steps, double cfl, double *dt_out, double *mass_out, void *const *events,
                   void *stream)
{
    if (!c || n_steps < 0 || !finite_pos(cfl)) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto mark = [&](int i) -> cudaError_t {
        return events && events[i] ? cudaEventRecord(static_cast<cudaEvent_t>(events[i]), s) : cudaSuccess;
    };
    SWE_TRY(mark(0));
    SWE_TRY(sync_planes(c, s));
    // result[0..1] = (dt, bad cells), result[2] = mass
    SWE_TRY(launch_cfl(c->dtype, plane_ptr(c, c->cur, 0), plane_ptr(c, c->cur, 1), plane_ptr(c, c->cur, 2), c->nx,
                       c->ny, c->pitch, c->dx, c->dy, c->g, cfl, c->scratch, c->result, s));
    SWE_TRY(launch_coef_from_cfl(c->dtype, c->result, c->dx, c->dy, c->g, c->kdev, s));
    const int cur0 = c->cur;
    const long long launches0 = c->launches;
    SWE_TRY(mark(1));
    const swe_status st = step_launches(c, n_steps, s, c->kdev);
    if (st != SWE_OK) return st;
    SWE_TRY(mark(2));
    SWE_TRY(sync_planes(c, s));
    SWE_TRY(launch_mass(c->dtype, plane_ptr(c, c->cur, 0), c->nx, c->ny, c->pitch, c->dx * c->dy, c->scratch,
                        c->result + 2, s));
    SWE_TRY(cudaMemcpyAsync(c->host_result, c->result, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SWE_TRY(mark(3));
    SWE_TRY(cudaStreamSynchronize(s));
    if (c->host_result[1] != 0.0) {
        // the step kernels skipped: the state is still in the first buffer
        c->cur = cur0;
        c->launches = launches0;
        c->planes_stale = false;
        if (dt_out) *dt_out = 0.0;
        return SWE_ECHECK;
    }
    c->dt = c->host_result[0];
    if (dt_out) *dt_out = c->dt;
    if (mass_out) *mass_out = c->host_result[2];
    return SWE_OK;
}

swe_status swe_check(swe_ctx *c, void *stream)
{
    if (!c) return SWE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int word = 0;
    SWE_TRY(cudaMemcpyAsync(&word, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SWE_TRY(cudaStreamSynchronize(s));
    if (word != 0) {
        SWE_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), s));
        SWE_TRY(cudaStreamSynchronize(s));
        return (swe_status)word;
    }
    return SWE_OK;
}

swe_status swe_query(swe_ctx *c, int key, long long *value)
{
    if (!c || !value) return SWE_EINVAL;
    switch (key) {
        case SWE_Q_KERNEL: *value = c->kernel; break;
        case SWE_Q_DEPTH: *value = c->depth; break;
        case SWE_Q_PITCH: *value = c->pitch; break;
        case SWE_Q_LAUNCHES: *value = c->launches; break;
        case SWE_Q_TILE_X: *value = c->kernel == SWE_KERNEL_NAIVE ? 64 : tiled_geom(c->dtype).tile_x; break;
        case SWE_Q_STEPS_PER_LAUNCH: *value = c->depth; break;
        case SWE_Q_SHAPE: *value = c->kernel == SWE_KERNEL_TEMPORAL ? c->tb_variant : -1; break;
        case SWE_Q_TILE_Y: *value = c->kernel == SWE_KERNEL_NAIVE ? 4 : tiled_geom(c->dtype).tile_y; break;
        case SWE_Q_STATE_PTR:
            // packed contexts: the packed state (h, hu, hv, 0 per cell)
            *value = (long long)(uintptr_t)(c->kernel == SWE_KERNEL_PACKED ? c->packed[c->cur] : plane_ptr(c, c->cur, 0));
            break;
        default: return SWE_EINVAL;
    }
    return SWE_OK;
}

}  // extern "C"
