/*
 * swe.h -- C ABI of the GB300 (sm_103a) shallow-water Lax-Wendroff library.
 *
 * The library advances the 2D shallow-water equations (Sec. 3: conservation
 * of mass and of x- and y-momentum for h, hu, hv under gravity g) with the
 * two-step (Richtmyer) Lax-Wendroff scheme of Sec. 3 and the statements of
 * Sec. 3.1: reflective-wall ghost cells, x- and y-face half steps, and a
 * dimensionally unsplit conservative full step.  The kernel procedure
 * wave_advance(dx, dy, dt, H, U, V, oH, oU, oV) of Sec. 3.1 is the model for
 * swe_step: the state is read-only during a step and the result goes to a
 * second buffer (double buffering, Sec. 2.5).
 *
 * Conventions for every call:
 *  - Grids are nx x ny interior cells, x fastest in memory: element (i, j),
 *    0 <= i < nx, 0 <= j < ny, of a caller buffer with row stride ``ld``
 *    elements sits at offset j*ld + i.  Fields are H = h (height), U = hu,
 *    V = hv (momenta), as the paper names them.
 *  - Ownership: the library owns every device buffer it allocates; the
 *    caller owns the pointers it passes and keeps them valid until the
 *    call's stream work has completed.
 *  - Streams: ``stream`` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Calls enqueue work and return; only the calls marked
 *    "synchronous" wait for it.
 *  - Errors are returned as swe_status codes; the library never aborts or
 *    traps.  Errors that kernels detect (a bounded wait that gave up) are
 *    recorded in a device error word and reported by swe_check.
 *  - A handle is not thread-safe; one host thread at a time per handle.
 *  - dt is the caller's: the paper uses a fixed time step (Sec. 3);
 *    swe_cfl_dt computes the CFL-limited value.
 */
#ifndef SWE_H
#define SWE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swe_ctx swe_ctx;

typedef enum {
    SWE_OK = 0,
    SWE_EINVAL = 1,       /* invalid argument (sizes, pointers, dtype ...) */
    SWE_ENOMEM = 2,       /* device or pinned host allocation failed */
    SWE_ECUDA = 3,        /* a CUDA runtime call failed */
    SWE_ETIMEOUT = 4,     /* a device-side bounded wait gave up */
    SWE_ECHECK = 5,       /* a mass/positivity check failed */
    SWE_EUNSUPPORTED = 6  /* valid request this build does not support */
} swe_status;

typedef enum { SWE_F32 = 0, SWE_F64 = 1 } swe_dtype;

/* Step kernel selection (swe_options.kernel). */
typedef enum {
    SWE_KERNEL_AUTO = 0,   /* the fastest variant for the dtype and size */
    SWE_KERNEL_NAIVE = 1,  /* one thread per cell, neighbours from global memory */
    SWE_KERNEL_TILED = 2,  /* TMA tile + halo in shared memory, one step per launch */
    SWE_KERNEL_TEMPORAL = 3 /* TMA tile + k-cell halo, k steps per launch */
} swe_kernel;

typedef struct {
    int dtype;   /* swe_dtype; default SWE_F32 */
    int kernel;  /* swe_kernel; default SWE_KERNEL_AUTO */
    int depth;   /* steps per launch for SWE_KERNEL_TEMPORAL; 0 = default */
    int reserved[5];
} swe_options;

/* Fills *opt with the defaults (FP32, automatic kernel choice). */
void swe_options_init(swe_options *opt);

/*
 * swe_create / swe_create_ex: allocate a grid of nx x ny interior cells
 * (1 <= nx, ny <= 65536) with spacing dx, dy > 0, time step dt > 0 and
 * gravity g > 0 on the current CUDA device.  Two device state buffers of
 * three planes each are allocated (the double buffer of Sec. 2.5); their
 * contents are undefined until swe_set_state.  swe_create uses FP32.
 * Returns SWE_EINVAL for bad sizes, SWE_ENOMEM if allocation fails.
 */
swe_status swe_create(int nx, int ny, double dx, double dy, double dt, double g, swe_ctx **out);
swe_status swe_create_ex(int nx, int ny, double dx, double dy, double dt, double g,
                         const swe_options *opt, swe_ctx **out);

/* Frees the handle and its device memory (waits for the device first).
 * NULL is ignored. */
void swe_destroy(swe_ctx *ctx);

/* Replaces the time step used by the following swe_step calls (dt > 0). */
swe_status swe_set_dt(swe_ctx *ctx, double dt);

/*
 * swe_set_state: copy the interior state (h, hu, hv) into the current
 * buffer.  Each pointer addresses nx x ny elements of the context dtype
 * (float for SWE_F32, double for SWE_F64) with row stride ld >= nx
 * elements; on_device = 1 if they are device pointers, 0 for host memory
 * (pinned host memory makes the copy asynchronous).  Stream-ordered.
 */
swe_status swe_set_state(swe_ctx *ctx, const void *h, const void *hu, const void *hv,
                         long long ld, int on_device, void *stream);

/* swe_get_state: the reverse copy of the current state, same layout rules. */
swe_status swe_get_state(swe_ctx *ctx, void *h, void *hu, void *hv,
                         long long ld, int on_device, void *stream);

/*
 * swe_step: advance n_steps >= 0 time steps of size dt (Sec. 3, the two
 * step equations), applying the reflective walls itself: the ghost value of
 * a wall cell mirrors the adjacent interior cell, with the wall-normal
 * momentum negated (U at x-walls, V at y-walls).  Enqueued on ``stream``.
 */
swe_status swe_step(swe_ctx *ctx, int n_steps, void *stream);

/*
 * swe_mass: FP64 mass sum(h) * dx * dy over the interior of the current
 * state (Sec. 3: h stands for the mass of a cell).  The sum runs in FP64 on
 * the device (a fixed-order tree, so repeated calls give identical bits).
 * Synchronous: waits for ``stream`` and writes *mass_out.
 */
swe_status swe_mass(swe_ctx *ctx, double *mass_out, void *stream);

/*
 * swe_cfl_dt: FP64 CFL time step of the current state,
 *   cfl * min over cells of min(dx / (sqrt(g h) + |hu/h|), dy / (sqrt(g h) + |hv/h|)),
 * the per-direction form of the bound dt <= dx / (sqrt(g h) + |u|) of Sec. 3.
 * Synchronous.  Returns SWE_ECHECK (and *dt_out = 0) if some h <= 0 or is
 * not finite.  Does not change the context's dt.
 */
swe_status swe_cfl_dt(swe_ctx *ctx, double cfl, double *dt_out, void *stream);

/* Synchronises ``stream`` and returns the device error word:
 * SWE_OK or SWE_ETIMEOUT (a kernel's bounded wait gave up); clears it. */
swe_status swe_check(swe_ctx *ctx, void *stream);

/* Introspection keys for swe_query. */
typedef enum {
    SWE_Q_KERNEL = 0,           /* swe_kernel actually used by swe_step */
    SWE_Q_DEPTH = 1,            /* steps per launch */
    SWE_Q_PITCH = 2,            /* row pitch of a device plane, elements */
    SWE_Q_LAUNCHES = 3,         /* step-kernel launches enqueued so far */
    SWE_Q_TILE_X = 4,           /* tile width in cells */
    SWE_Q_TILE_Y = 5,           /* tile height in cells */
    SWE_Q_STATE_PTR = 6         /* device address of the current H plane */
} swe_query_key;

/* Writes the value of ``key`` to *value. */
swe_status swe_query(swe_ctx *ctx, int key, long long *value);

/*
 * swe_mass_noalloc: the FP64 mass sum(h) * dx * dy of a caller-owned device
 * plane, computed without allocating anything.  The paper has no
 * counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: programs whose device memory is all owned by another
 * allocator (a framework's caching pool that has reserved the GPU, so an
 * extra cudaMalloc may fail or fragment it), and loops that cannot afford
 * the device-wide synchronisation cudaMalloc/cudaFree may cause.  Such a
 * caller has no swe_ctx (creating one allocates), only its own buffers.
 *
 * h: device pointer to nx x ny elements of ``dtype`` (SWE_F32 or SWE_F64),
 * row stride ld >= nx elements.  mass_dev: device pointer to one double that
 * receives the result.  Both stay owned by the caller.  Enqueued on
 * ``stream``; the result is the same FP64 fixed-order sum swe_mass computes
 * for the same data.
 *
 * Scratch: the partial sums live in a file-scope __device__ array of 1024
 * doubles (8 KB), which every GPU that loads the library holds until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, with the device current); make the first
 * call on each device before any stream capture.  All calls share the
 * array and each call overwrites every partial it reads, so nothing needs
 * clearing, but calls that overlap on the GPU (other streams, other host
 * threads) race on it: serialise them.
 *
 * Returns SWE_EINVAL for a bad dtype, a NULL pointer, ld < nx, dx or dy not
 * finite and positive, or nx or ny outside 1..SWE_NOALLOC_MAX_DIM; SWE_ECUDA
 * if the address lookup or the launch fails.  Allocates nothing: no
 * cudaMalloc, cudaFree or allocating library call.
 */
#define SWE_NOALLOC_MAX_DIM 65536
swe_status swe_mass_noalloc(int dtype, const void *h, int nx, int ny, long long ld, double dx, double dy,
                            double *mass_dev, void *stream);

/* Static description of a status code. */
const char *swe_strerror(swe_status s);

#ifdef __cplusplus
}
#endif

#endif /* SWE_H */
