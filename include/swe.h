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
    SWE_EUNSUPPORTED = 6  /* valid request that the library does not support */
} swe_status;

typedef enum { SWE_F32 = 0, SWE_F64 = 1 } swe_dtype;

/* Step kernel selection (swe_options.kernel). */
typedef enum {
    SWE_KERNEL_AUTO = 0,   /* TEMPORAL with the streaming shape (the fastest measured at 8192^2, FP32 and FP64) */
    SWE_KERNEL_NAIVE = 1,  /* one thread per cell, neighbours from global memory */
    SWE_KERNEL_TILED = 2,  /* TMA tile + halo in shared memory, one step per launch */
    SWE_KERNEL_TEMPORAL = 3, /* TMA tile + 2-cell halo, 2 steps per launch (an odd
                               last step uses the one-step kernel); same bits */
    SWE_KERNEL_PACKED = 4    /* FP32 only: the state packed as (h, hu, hv, 0) 16-byte
                               cells on the device (Sec. 5's packed vector type) instead
                               of three planes; TMA tile + halo, one step per launch;
                               32 B of HBM traffic per cell-update (planes: 24); same
                               bits as the plane kernels.  State transfers and the
                               reductions go through plane copies. */
} swe_kernel;

typedef struct {
    int dtype;   /* swe_dtype; default SWE_F32 */
    int kernel;  /* swe_kernel; default SWE_KERNEL_AUTO */
    int depth;   /* 0 = default; SWE_KERNEL_TEMPORAL runs 2 steps per launch */
    int reserved[5]; /* reserved[0]: two-step kernel shape + 1 (0 = the default: shape 5 for FP32, 6 for
                        FP64).  Shapes 0..3 take one CTA per tile (warps x rows: 4x8, 8x4, 4x4, 8x2),
                        shape 4 is 8x4 with persistent CTAs that prefetch their next tile.  Shapes 5..8
                        are warps that stream up column strips with the intermediate rows in registers
                        and x-neighbours from warp shuffles.  FP32: 5: 120-column strips, two 4-row TMA
                        chunks per warp; 6: three chunks; 7: 56-column strips; 8: four 2-row chunks.
                        FP64 (5 and 6 only; SWE_EUNSUPPORTED for 7, 8): 60-column strips, registers
                        uncapped (5) or capped for 3 CTAs per SM (6).  All shapes give the same bits.
                        Others 0 */
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

/*
 * swe_run: one job of the Sec. 3 time loop without a host round trip inside:
 * the FP64 CFL step of the current state (as swe_cfl_dt) is computed on the
 * device and stays there, the n_steps >= 0 steps (as swe_step) take their
 * coefficients from it, and the FP64 mass of the result (as swe_mass)
 * follows.  Bit for bit the same dt, state and mass as swe_cfl_dt,
 * swe_set_dt, swe_step and swe_mass in turn.  ``events`` (optional) is an
 * array of four cudaEvent_t (as void*, each may be NULL) recorded on
 * ``stream`` before the first kernel, before the first step launch, after
 * the last step launch and after the results' copy to the host, so that the
 * job's device time excludes host latency.  Synchronous: waits once, at the
 * end, then sets the context's dt and writes *dt_out and *mass_out (either
 * may be NULL).  Returns SWE_ECHECK (*dt_out = 0, the state left as it was)
 * if some h <= 0 or is not finite.
 */
swe_status swe_run(swe_ctx *ctx, int n_steps, double cfl, double *dt_out, double *mass_out, void *const *events,
                   void *stream);

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
    SWE_Q_STATE_PTR = 6,        /* device address of the current H plane (SWE_KERNEL_PACKED: of the packed state) */
    SWE_Q_STEPS_PER_LAUNCH = 7, /* steps a full step-kernel launch advances */
    SWE_Q_SHAPE = 8             /* two-step kernel shape (see swe_options), -1 for the other kernels */
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
 * address (cudaGetSymbolAddress, with the device current) and keeps it for
 * the life of the process; make the first call on each device before any
 * stream capture.  A device reset (cudaDeviceReset, or anything else that
 * destroys the device's primary context) invalidates that address: do not
 * call swe_mass_noalloc on that device afterwards.  All calls share the
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

/* ==========================================================================
 * Batched ensembles (no counterpart in the paper: many independent
 * instances of the Sec. 3 step, each with its own size, dx, dy and dt).
 * All instances are FP32, share g, and step together.
 * ========================================================================== */
typedef struct swe_batch swe_batch;

/* Per-instance flags reported by swe_batch_status. */
#define SWE_FLAG_NONPOSITIVE 1 /* a step produced h <= 0 (or NaN) in the instance */
#define SWE_FLAG_MASS 2        /* the instance failed a mass-drift check */
#define SWE_FLAG_TIMEOUT 4     /* a device-side bounded wait gave up (all instances) */
#define SWE_FLAG_FALLBACK 8    /* the instance was recomputed by the fallback solver */

/*
 * swe_batch_create: n >= 1 instances; instance i has nx[i] x ny[i] cells
 * (1..65536 each), spacing dx[i], dy[i] and time step dt[i] (all finite,
 * > 0); gravity g.  Allocates one device pool holding two FP32 state
 * buffers (three planes each) per instance, rows 128-byte aligned.
 * The arrays are copied; the caller keeps ownership.
 */
swe_status swe_batch_create(int n, const int *nx, const int *ny, const double *dx, const double *dy,
                            const double *dt, double g, swe_batch **out);
void swe_batch_destroy(swe_batch *b);

/* Copy instance i's interior state in / out (float, row stride ld >= nx[i];
 * host or device pointers as for swe_set_state).  Stream-ordered. */
swe_status swe_batch_set_state(swe_batch *b, int i, const void *h, const void *hu, const void *hv,
                               long long ld, int on_device, void *stream);
swe_status swe_batch_get_state(swe_batch *b, int i, void *h, void *hu, void *hv, long long ld,
                               int on_device, void *stream);

/* Replaces every instance's time step (dt[0..n-1], finite, > 0). */
swe_status swe_batch_set_dt(swe_batch *b, const double *dt, void *stream);

/*
 * swe_batch_step: advance every instance by n_steps steps of its own dt in
 * ONE persistent, cooperatively launched kernel (the Sec. 3 step per tile;
 * a grid-wide barrier with a bounded wait between steps).  The launch is
 * captured into a CUDA graph per (n_steps, buffer parity) and replayed on
 * ``stream``; where capture is unavailable it is launched directly.  A step
 * that makes h <= 0 sets SWE_FLAG_NONPOSITIVE for that instance.
 */
swe_status swe_batch_step(swe_batch *b, int n_steps, void *stream);

/* Synchronous: writes each instance's flags to flags_out[0..n-1], clears
 * them, and returns SWE_ETIMEOUT if a bounded wait gave up, else SWE_OK. */
swe_status swe_batch_status(swe_batch *b, int *flags_out, void *stream);

/* Synchronous FP64 reductions per instance (as swe_mass / swe_cfl_dt):
 * mass_out[i] = sum(h) dx dy; dt_out[i] = CFL step (0 and SWE_ECHECK if
 * some h <= 0 or a value is not finite). */
swe_status swe_batch_mass(swe_batch *b, double *mass_out, void *stream);
swe_status swe_batch_cfl_dt(swe_batch *b, double cfl, double *dt_out, void *stream);

/*
 * swe_batch_tune: autotuner.  Times every kernel variant (tile shape,
 * staging depth) at every feasible CTA count per SM on this batch, keeps the
 * fastest, and appends it to the JSON-lines cache ``cache_path`` (or
 * $SWE_TUNE_CACHE; NULL and no variable = no cache), keyed by GPU name and
 * instance sizes.  A cached entry is reused without timing.  The current
 * state is saved and restored around the trials.  Synchronous.
 */
swe_status swe_batch_tune(swe_batch *b, const char *cache_path, void *stream);

/*
 * swe_selftest_wait: exercises the library's bounded device waits.  which =
 * 0 waits on an mbarrier that nothing completes; which = 1 on a grid barrier
 * that expects one CTA more than are launched.  Each wait gives up after
 * limit_ms (0 < limit_ms <= 5000) and the kernel returns.  Synchronous;
 * returns SWE_ETIMEOUT when the wait ran out as designed.
 */
swe_status swe_selftest_wait(int which, double limit_ms, void *stream);

/*
 * swe_probe_rate (no counterpart in the paper): measures the current
 * device's arithmetic throughput, the peak against which the ALU-bound
 * kernels' fractions are stated.  kind 0: scalar FP32 FMA, 1: packed f32x2
 * FMA (two lanes per instruction), 2: FP64 FMA.  Runs independent FMA
 * chains in 8 CTAs of 256 threads per SM for a few milliseconds on a
 * private stream, times the last of three launches with CUDA events and
 * writes FMAs per second (lane operations; an FMA is two flops) to
 * *rate_out.  Synchronous; changes no device setting.  SWE_EINVAL for an
 * unknown kind or a null pointer, SWE_ECUDA on a CUDA error.
 */
swe_status swe_probe_rate(int kind, double *rate_out);

/* Device address of instance i's h plane in the current buffer, and the
 * plane stride and row pitch in floats (hu, hv follow at +1, +2 planes). */
swe_status swe_batch_state_ptr(swe_batch *b, int i, float **h, long long *plane_stride, long long *pitch);

/* Copies every instance's current state, in order, to a contiguous device
 * buffer: instance i's h, hu, hv planes of ny[i] x nx[i] floats each. */
swe_status swe_batch_copy_states(swe_batch *b, float *dst, void *stream);

/* Selects a kernel variant (0 .. the count swe_batch_query reports for
 * SWE_BQ_VARIANT_COUNT, minus 1) and CTAs per SM explicitly (tests, tuning,
 * profiling); a CTA count above what fits is
 * lowered to it.  Variants: 0..4 one step per pass over tiles (128 x 16..64,
 * 4 or 8 warps, one or two TMA stages); 5..7 two steps per pass over tiles;
 * 8, 9 two steps per pass by warps streaming up 120-column strips (3 and 2
 * CTAs per SM).  Synchronous; call it with no step of this batch in
 * flight, since it rewrites the tile list the kernel reads.  SWE_EINVAL for
 * a variant out of range or ctas_per_sm < 1, SWE_EUNSUPPORTED if the
 * variant cannot run on this device. */
swe_status swe_batch_configure(swe_batch *b, int variant, int ctas_per_sm);

typedef enum {
    SWE_BQ_VARIANT = 0, SWE_BQ_CTAS_PER_SM = 1, SWE_BQ_BLOCKS = 2, SWE_BQ_TILES = 3,
    SWE_BQ_TILE_X = 4, SWE_BQ_TILE_Y = 5, SWE_BQ_STAGES = 6, SWE_BQ_DEPTH = 7,
    SWE_BQ_GRAPH = 8,        /* 1 if steps replay a captured CUDA graph */
    SWE_BQ_LAUNCHES = 9,     /* persistent launches enqueued so far */
    SWE_BQ_TUNED = 10,       /* 0 default, 1 tuned by timing, 2 from cache */
    SWE_BQ_CELLS = 11,       /* total cells over all instances */
    SWE_BQ_VARIANT_COUNT = 12,
    SWE_BQ_KIND = 13         /* the variant's kernel: 0 tiles (batch_lw / batch_tb2), 1 streaming warps */
} swe_batch_query_key;
swe_status swe_batch_query(swe_batch *b, int key, long long *value);

/* ==========================================================================
 * Domain decomposition.  One grid split into px x py partitions, each with a
 * one-cell ghost ring, all on the current device: the layout a multi-GPU run
 * would give each GPU (Sec. 4.1 and Fig. 1: MPI partitions of the global
 * array with their halos, named there as future work), with the halo
 * exchange done by a kernel.  Partition (a, b) holds columns
 * [a nx / px, (a+1) nx / px) and rows [b ny / py, (b+1) ny / py) (integer
 * division).  A step is a halo launch (ghosts next to another partition
 * copy its edge cells; ghosts on the grid boundary are the reflective
 * mirror of their own edge cell) and a step launch over all partitions
 * (the single-grid kernel's TMA tiles, reading the ghost ring); the result
 * equals swe_step on the whole grid bit for bit.  FP32.
 * ========================================================================== */
typedef struct swe_part swe_part;

/* 1 <= px <= nx, 1 <= py <= ny, px * py <= 4096; spacing, dt, g > 0. */
swe_status swe_part_create(int nx, int ny, int px, int py, double dx, double dy, double dt, double g,
                           swe_part **out);
void swe_part_destroy(swe_part *part);
/* The whole nx x ny interior in or out (row stride ld >= nx floats, host or
 * device pointers), scattered to / gathered from the partitions;
 * stream-ordered. */
swe_status swe_part_set_state(swe_part *part, const float *h, const float *hu, const float *hv, long long ld,
                              void *stream);
swe_status swe_part_get_state(swe_part *part, float *h, float *hu, float *hv, long long ld, void *stream);
/* n_steps steps of every partition (two launches per step); stream-ordered. */
swe_status swe_part_step(swe_part *part, int n_steps, void *stream);
typedef enum {
    SWE_PQ_PARTS = 0,      /* px * py */
    SWE_PQ_HALO_CELLS = 1, /* ghost cells exchanged or mirrored per step (per field) */
    SWE_PQ_LAUNCHES = 2,   /* launches enqueued so far */
    SWE_PQ_ERROR = 3       /* the device error word (synchronous): 0 or SWE_ETIMEOUT */
} swe_part_query_key;
swe_status swe_part_query(swe_part *part, int key, long long *value);

/*
 * One rank's partition of a grid decomposed across processes (Sec. 4.1 and
 * Fig. 1: each MPI rank holds its part of the global array with a halo).
 * swe_part_create_rank makes a single nx x ny partition whose sides in the
 * bitmask ``walls`` (1 left, 2 right, 4 bottom, 8 top) lie on the global
 * boundary: their ghosts are filled by swe_part_step as reflective walls.
 * The ghosts of the other sides face another rank's partition; before each
 * swe_part_step the caller writes them with swe_part_set_ghosts from that
 * rank's edge cells, which swe_part_edges reads.  Both use one device
 * buffer of 6 (nx + ny) floats, the four sides' strips one after another:
 * left (h, hu, hv over the ny rows), right (the same), bottom (h, hu, hv
 * over the nx columns), top (the same), each strip in increasing row or
 * column order.  swe_part_edges writes all four edge strips of the current
 * state; swe_part_set_ghosts reads the strips of the sides in the bitmask
 * ``sides`` and leaves the rest of the buffer unread.  Stream-ordered; the
 * buffer is the caller's.  With every rank's ghosts so exchanged, each
 * step gives the single-grid result bit for bit.  SWE_EINVAL for walls or
 * sides outside 0..15, a null buffer, or a context from swe_part_create
 * with more than one partition.  swe_part_set_state / get_state / step /
 * query / destroy apply as above (px = py = 1).
 */
swe_status swe_part_create_rank(int nx, int ny, int walls, double dx, double dy, double dt, double g,
                                swe_part **out);
swe_status swe_part_edges(swe_part *part, float *edges, void *stream);
swe_status swe_part_set_ghosts(swe_part *part, const float *ghosts, int sides, void *stream);

/* ==========================================================================
 * Region front end (Sec. 2.3 region functions; Sec. 3.1 statements; Sec.
 * 4.2.1 lowering).  The step and the wall fill written as array statements
 * over halo regions (region_cpy / region_ptr with halo [left, right, down,
 * up]) in a C++ expression-template header, each statement lowered to a
 * loop of a CTA's threads over the statement's region, with the inputs
 * staged in shared memory by TMA.  Every operation of a statement is one
 * IEEE round-to-nearest operation in the stated order (no FMA contraction,
 * IEEE division), so an FP64 step equals the FP64 oracle bit for bit.
 *
 * Arrays are device planes of (nx + 2) x (ny + 2) elements with the ghost
 * ring, row stride ``pitch`` elements (pitch >= nx + 2, pitch * element size
 * a multiple of 16 bytes, planes 16-byte aligned), interior cell (i, j),
 * 1 <= i <= nx, 1 <= j <= ny, at j * pitch + i.  The caller owns them.
 * As in Sec. 2.3 the step leaves boundary conditions to the caller: it reads
 * the ghosts as they are, and swe_region_walls fills them.
 * ========================================================================== */
typedef struct swe_region swe_region;

/* dtype SWE_F32 or SWE_F64; 1 <= nx, ny <= 65536; variant 0 (default: FP32
 * 3, FP64 2) or a tile shape, cells per CTA / threads: FP32 1..5 =
 * 64x16/256, 128x8/256, 32x32/256, 64x16/128, 32x16/128; FP64 1..3 =
 * 64x8/256, 32x16/256, 32x8/128.  SWE_EINVAL for anything else. */
swe_status swe_region_create(int dtype, int nx, int ny, long long pitch, int variant, swe_region **out);
void swe_region_destroy(swe_region *r);
/* One step: in[0..2] = H, U, V with ghosts filled, out[0..2] receive the
 * interior (their ghosts are not written; out must not alias in).
 * Stream-ordered; SWE_EINVAL for NULL or misaligned planes or a
 * non-positive dx, dy, dt or g. */
swe_status swe_region_step(swe_region *r, const void *const in[3], void *const out[3], double dx, double dy,
                           double dt, double g, void *stream);
/* One step over a bottom topography (no counterpart in the paper, whose
 * bed is flat): ``bed`` is the bed elevation B, a plane like the state's
 * with its ghost ring filled (for walls and open sides alike the ghost
 * copies the edge cell), H the water depth and H + B the free surface.  The
 * momentum rows gain the bed-slope source -g H B_x, -g H B_y, taken at the
 * points of the pressure-flux difference it balances with the depth
 * averaged over the same two points (step 1: + dt/2dx g (H_a + H_b)/2
 * (B_a - B_b) on the face between cells a, b; step 2: + dt/dx g (Hx_L +
 * Hx_R)/2 (Bx_L - Bx_R) with Bx the mean of the two cells beside a face;
 * likewise in y), so a lake at rest (H + B constant, no flow) stays at
 * rest.  Otherwise as swe_region_step. */
swe_status swe_region_step_bed(swe_region *r, const void *const in[3], const void *bed, void *const out[3], double dx,
                               double dy, double dt, double g, void *stream);
/* Reflective ghost fill of the sides in ``walls`` (1 left, 2 right,
 * 4 bottom, 8 top): ghost = the adjacent interior cell, wall-normal
 * momentum negated; corner ghosts untouched.  Stream-ordered. */
swe_status swe_region_walls(swe_region *r, void *const state[3], int walls, void *stream);
/* Ghost fill with a kind per side (kinds[0..3] = left, right, bottom, top):
 * 0 leaves the side alone, 1 reflective wall (as swe_region_walls), 2 open
 * (zero-gradient: the ghost copies the adjacent interior cell, all three
 * components, so waves leave the domain).  SWE_EINVAL for another kind. */
swe_status swe_region_boundary(swe_region *r, void *const state[3], const int kinds[4], void *stream);
/* n_steps of (walls, step), alternating between a and b starting from a;
 * *result_in_b (if not NULL) is 1 when the final state is in b. */
swe_status swe_region_run(swe_region *r, void *const a[3], void *const b[3], int n_steps, int walls, double dx,
                          double dy, double dt, double g, void *stream, int *result_in_b);
/* As swe_region_run with per-side boundary kinds (swe_region_boundary) and,
 * if ``bed`` is not NULL, the step over that bed (swe_region_step_bed). */
swe_status swe_region_run_bc(swe_region *r, void *const a[3], void *const b[3], const void *bed, int n_steps,
                             const int kinds[4], double dx, double dy, double dt, double g, void *stream,
                             int *result_in_b);
typedef enum {
    SWE_RQ_LAUNCHES = 0, /* launches enqueued so far */
    SWE_RQ_TILE_X = 1,   /* interior cells per CTA in x */
    SWE_RQ_TILE_Y = 2,   /* ... in y */
    SWE_RQ_SMEM = 3,     /* dynamic shared memory per CTA, bytes */
    SWE_RQ_ERROR = 4     /* the device error word (synchronous): 0, SWE_EINVAL (a
                            statement whose regions do not conform) or SWE_ETIMEOUT */
} swe_region_query_key;
swe_status swe_region_query(swe_region *r, int key, long long *value);
/* Host only, evaluates nothing: the extents (x, y) the statement groups of
 * the step and the wall fill take on nx x ny interior cells, in order:
 * cell fluxes, x-faces, y-faces, update, then the left, right, bottom and top ghost
 * strips.  ext receives 2 * min(*n_groups, max_groups) ints; an extent of a
 * group whose regions do not conform is negative.  1 <= nx, ny <= 65536. */
swe_status swe_region_shapes(int nx, int ny, int *ext, int max_groups, int *n_groups);
/* Self-test of the FP32 division of the region statements: out[i] =
 * a[i] / b[i] correctly rounded, by the statements' FMA division (which = 0),
 * by the same division on element pairs (2m, 2m + 1) as the paired FP32
 * evaluation takes it (2; n even), or by CUDA's __fdiv_rn (1); which = 3
 * gives the reciprocal step of the statements' division alone, out[i] =
 * 1 / b[i] correctly rounded for 2^-20 <= b[i] < 2^20 whose significand is
 * not all ones (a is not read; other b give an undefined value); which = 4
 * gives the stencil kernels' approximate reciprocal of b[i] (rcp.approx,
 * flushing subnormals; a is not read).  Device pointers, n >= 0;
 * stream-ordered. */
swe_status swe_selftest_div(const float *a, const float *b, float *out, int n, int which, void *stream);

/* ==========================================================================
 * Learned coarse-grid corrector (no counterpart in the paper).  A network
 * of zero-padded 3x3 convolutions, 3 -> 32 -> 32 -> 3 channels with GELU
 * (0.5 z (1 + erf(z / sqrt 2))), BF16 weights and activations with FP32
 * accumulation on the tcgen05 tensor cores, predicts the residual that
 * carries a coarse Lax-Wendroff step (Sec. 3) toward the 4x4 block
 * average of the fine solution.  Images are H x W coarse grids.
 *
 * Parameters (FP32 master copy, swe_net_param_count() floats, in order):
 * W1[3][3][3][32], b1[32], W2[3][3][32][32], b2[32], W3[3][3][32][3], b3[3],
 * with W[ky][kx][c_in][c_out] applied as y[o](i,j) = b[o] +
 * sum W[ky][kx][c][o] x[c](i+ky-1, j+kx-1).
 * Normalisation (swe_net_set_norm, 5 floats): h0, sh, su (network input
 * ((h - h0)/sh, hu/su, hv/su)) and oh, ou (output scale of the h and
 * momentum residuals).  State arguments are FP32 device pointers to image
 * 0's h plane; image i's field f row y starts at
 * state + i*img_stride + f*plane_stride + y*pitch (all in floats).
 * ========================================================================== */
typedef struct swe_net swe_net;

size_t swe_net_param_count(void);
/* Allocates activations for up to max_images images of H x W (<= 8192). */
swe_status swe_net_create(int max_images, int H, int W, swe_net **out);
void swe_net_destroy(swe_net *net);
/* Host FP32 parameters in / out; setting them resets the optimiser state. */
swe_status swe_net_set_params(swe_net *net, const float *params);
swe_status swe_net_get_params(swe_net *net, float *params);
swe_status swe_net_set_norm(swe_net *net, const float *norm5);
/* Builds the network input of n images from a state (stream-ordered):
 * ((h - h0)/sh, hu/su, hv/su), or, with a second state ``base`` (same
 * strides, may be NULL), the FP32 difference (state - base) scaled by
 * (1/sh, 1/su, 1/su).  The corrector uses the latter with state = the coarse
 * Lax-Wendroff result and base = the state it started from, so the network
 * sees the step's increment at FP32 resolution before the BF16 rounding. */
swe_status swe_net_prep_input(swe_net *net, int n, const float *state, const float *base, long long img_stride,
                              long long plane_stride, long long pitch, void *stream);
/* Inference on the prepared input: residual in physical units, FP32
 * [n][3][H][W] into resid (device; NULL = the net's own buffer). */
swe_status swe_net_infer(swe_net *net, int n, float *resid, void *stream);
/* state += residual (the net's own buffer, from swe_net_infer(.., NULL, ..));
 * with project_mass the h residual's mean is removed per image first, so
 * the corrected step keeps the Lax-Wendroff step's mass. */
swe_status swe_net_apply(swe_net *net, int n, float *state, long long img_stride, long long plane_stride,
                         long long pitch, int project_mass, void *stream);
/* The corrected step in one call on the prepared input: the network, with
 * its scaled residual added to ``state`` in the last layer's epilogue;
 * with project_mass the per-image mean of the h correction is then
 * subtracted (mass of the Lax-Wendroff step kept up to rounding). */
swe_status swe_net_correct(swe_net *net, int n, float *state, long long img_stride, long long plane_stride,
                           long long pitch, int project_mass, void *stream);
/* Training target (normalised): (next - lw) / (oh, ou, ou), clipped to
 * [-clip, clip] if clip > 0, FP32 [n][3][H][W]; next is FP32 [n][3][H][W]
 * contiguous, lw a state as above. */
swe_status swe_net_make_target(swe_net *net, int n, const float *next, const float *lw, long long img_stride,
                               long long plane_stride, long long pitch, float clip, float *target, void *stream);
/* One training step on the prepared input: forward, mean squared error
 * against target (weighted per image, see swe_net_set_loss_weighting), backward (tcgen05 input gradients, CUDA-core weight
 * gradients), and with update = 1 an AdamW step (lr, weight decay wd,
 * global-norm clip if clip > 0).  Synchronous.  Optional outputs: the loss,
 * the gradients (host, param_count floats), the raw network output r
 * (device FP32 [n][3][H][W]). */
swe_status swe_net_train_step(swe_net *net, int n, const float *target, float lr, float wd, float clip, int update,
                              double *loss_out, float *grads_out, float *resid_out, void *stream);
/* Per-image weighting of the training loss: image i's squared error is
 * multiplied by w_i = max(ms_i, floor)^(-power/2), ms_i the mean square of
 * its target over the three channels (computed on the device each step).
 * power = 0 (the default) is the plain mean squared error; power = 1 weighs
 * an image by the inverse of its target's RMS, power = 2 makes every
 * image's relative error count alike.  0 <= power <= 4, floor > 0. */
swe_status swe_net_set_loss_weighting(swe_net *net, float power, float floor);
/* Synchronises and returns the device error word of the net's kernels. */
swe_status swe_net_check(swe_net *net, void *stream);
/* The learned coarse step of every instance of batch b, n_steps times, in
 * ONE persistent launch (stream-ordered): each step is the coarse
 * Lax-Wendroff step (Sec. 3), the network on its normalised FP32 increment
 * (as swe_net_prep_input with base = the state the step started from) and
 * the scaled residual added to the Lax-Wendroff result; with project_mass
 * the per-image mean of the h correction is removed (the step keeps the
 * Lax-Wendroff mass up to rounding).  Same arithmetic as swe_batch_step(1)
 * + swe_net_prep_input + swe_net_correct per step, but the activations
 * never leave the SM: one CTA sweeps one instance at a time, row by row.
 * Uses the net's current weights and normalisation; the net's image size is
 * not used.  Every instance must be at most 256 cells wide
 * (SWE_EUNSUPPORTED otherwise); instances may differ in size.  A step that
 * produces h <= 0 (or NaN) sets SWE_FLAG_NONPOSITIVE for the instance
 * (swe_batch_status); a device-side wait that gives up records
 * SWE_ETIMEOUT there too.  The batch's current buffer advances as with
 * swe_batch_step. */
swe_status swe_batch_learned_step(swe_batch *b, swe_net *net, int n_steps, int project_mass, void *stream);
/* Self-test of the network's activation on the device: out[i] = erf(z[i])
 * (which = 0; Abramowitz & Stegun 7.1.26, |error| <= 1.5e-7), gelu(z[i])
 * (1; the forward activation, erf from A&S 7.1.27, |error| <= 6.9e-4) or
 * gelu'(z[i]) (2; with 7.1.26); device pointers. */
swe_status swe_selftest_gelu(const float *z, float *out, int n, int which, void *stream);
/* factor x factor block average (factor 1..4) of n images (3 planes each)
 * of (factor Hc) x (factor Wc) fine cells into Hc x Wc coarse cells; strides
 * in floats as above.  The restriction that turns a fine solution into the
 * coarse target.  Stream-ordered. */
swe_status swe_downsample(int factor, const float *fine, long long f_img, long long f_plane, long long f_pitch,
                          float *coarse, long long c_img, long long c_plane, long long c_pitch, int Wc, int Hc, int n,
                          void *stream);

/* Area-weighted average of n images (3 planes each) of Hs x Ws cells onto
 * Hd x Wd cells covering the same domain (Wd <= Ws, Hd <= Hs, any ratio):
 * destination cell (X, Y) is the mean of the source over
 * [X Ws/Wd, (X+1) Ws/Wd) x [Y Hs/Hd, (Y+1) Hs/Hd), each source cell weighted
 * by its overlap (FP64 sums).  Keeps the integral of every plane; an
 * integer ratio is the block average of swe_downsample.  The restriction
 * between grids of the learned-vs-plain protocol (no counterpart in the
 * paper).  Strides in floats as above; stream-ordered; SWE_EINVAL for
 * upsampling or bad strides. */
swe_status swe_resample(const float *src, long long s_img, long long s_plane, long long s_pitch, int Ws, int Hs,
                        float *dst, long long d_img, long long d_plane, long long d_pitch, int Wd, int Hd, int n,
                        void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SWE_H */
