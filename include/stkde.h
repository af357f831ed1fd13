/*
 * stkde.h -- C ABI of the GB300 space-time kernel density estimation library.
 *
 * The library computes the STKDE density of Section 2.1 (the density equation
 * with kernels k_s and k_t) on a voxel grid:
 *
 *   out[X][Y][T] = 1/(n hs^2 ht) * sum_i [d_i < hs] [|t - t_i| <= ht]
 *                  k_s((x - x_i)/hs, (y - y_i)/hs) * k_t((t - t_i)/ht)
 *
 * sampled at voxel centres x = x0 + (X + 1/2) sres, y = y0 + (Y + 1/2) sres,
 * t = t0 + (T + 1/2) tres, with k_s(u,v) = c_s (1-u^2)(1-v^2) and
 * k_t(w) = c_t (1-w^2).  The work is the point-based symmetric scatter PB-SYM
 * (Section 3.2, Algorithm 3): per event, a spatial invariant K_s[X][Y] and a
 * temporal invariant K_t[T] whose outer product is added over the event's
 * cylinder.  On the GPU the sum over events inside a voxel tile is evaluated as
 * a rank-k contraction C[xy][t] = sum_k K_s[xy][k] K_t[k][t].
 *
 * Conventions shared by every entry point:
 *  - Events are n rows of three doubles (x, y, t), row-major, in domain units.
 *    The pointer may be host memory (pageable or pinned) or device memory of
 *    the context's device; the library detects which.
 *  - The grid is row-major [gx][gy][gt] binary32, T fastest (the stkde[X][Y][T]
 *    array of Algorithms 1-3), gx*gy*gt floats.
 *  - Bandwidths hs, ht are in domain units (hs in the units of x and y, ht in
 *    the units of t), as in the density equation.
 *  - Every event counts in n, including events outside the grid; cylinder
 *    voxels outside the grid are dropped.  n = 0 yields an all-zero grid.
 *  - The caller owns the events and the output buffer; the context owns its
 *    workspace, which grows on demand and is freed by stkde_destroy.
 *  - Calls are ordered on the context's stream and return once the work is
 *    enqueued.  Argument errors are reported synchronously, before any launch.
 *    Errors found on the device (non-finite coordinates, a bounded wait that
 *    gave up) are latched and returned by stkde_synchronize, or by the next
 *    call that synchronizes.
 *  - A context is not thread-safe: use one per host thread.  Contexts share
 *    no device state, so several contexts on several streams run concurrently.
 *  - Stream capture (CUDA graphs): stkde_compute and stkde_compute_batch may be
 *    captured when their events and outputs are device memory and the
 *    workspace already fits (an earlier call of the same size, or
 *    stkde_reserve); a call that would have to grow a buffer, wait for the
 *    stream or copy host memory returns STKDE_ERR_UNSUPPORTED before enqueueing
 *    anything, and so do the synchronous and per-event-bandwidth entry points.
 */
#ifndef STKDE_H
#define STKDE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define STKDE_API __attribute__((visibility("default")))
#else
#define STKDE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stkde_ctx stkde_ctx;

typedef enum {
    STKDE_OK = 0,
    STKDE_ERR_INVALID_ARGUMENT = 1, /* bad pointer, size, bandwidth or resolution */
    STKDE_ERR_OOM = 2,              /* a device allocation failed; no work was enqueued */
    STKDE_ERR_CUDA = 3,             /* a CUDA runtime call failed */
    STKDE_ERR_TIMEOUT = 4,          /* a device-side bounded wait gave up */
    STKDE_ERR_UNSUPPORTED = 5,      /* e.g. no sm_103a device, or a form not built */
    STKDE_ERR_NONFINITE = 6,        /* an event coordinate was NaN or infinite */
    STKDE_ERR_INTERNAL = 7          /* a device-side consistency check refused an operation (an
                                       accumulator window outside its tile); the grid is not valid */
} stkde_status;

/* How the sum over events is evaluated.  Every form writes each voxel of the
 * grid exactly once, except STKDE_FORM_SCATTER. */
typedef enum {
    /* tcgen05 tensor cores: K_s and K_t split into bf16 hi + lo parts, three
     * products (hi*hi + hi*lo + lo*hi) accumulated in fp32 in tensor memory. */
    STKDE_FORM_TENSOR_BF16X3 = 0,
    /* the same with fp16 hi + lo parts (11-bit significands). */
    STKDE_FORM_TENSOR_FP16X3 = 1,
    /* fp32 CUDA cores, per-voxel accumulation in registers. */
    STKDE_FORM_FP32 = 2,
    /* plain port of Algorithm 3: one block per event, atomic adds into a
     * zeroed grid.  Baseline only: the summation order, and so the last bits,
     * vary from run to run. */
    STKDE_FORM_SCATTER = 3,
    /* tcgen05 tensor cores, kind::tf32: hi = the value with its low 13
     * significand bits cleared, lo = the remainder; three products (hi*hi +
     * hi*lo + lo*hi), fp32 accumulation in tensor memory.  Fixed bandwidths only. */
    STKDE_FORM_TENSOR_TF32X3 = 4,
    /* one tf32 product per term (hi*hi): about 2^-11 relative error per term,
     * for comparison only.  Fixed bandwidths only. */
    STKDE_FORM_TENSOR_TF32X1 = 5
} stkde_form;

/* Kernel constants (Section 2.1). */
typedef enum {
    STKDE_KERNEL_PRINTED = 0,   /* c_s = pi/2, c_t = 3/4, as printed */
    STKDE_KERNEL_UNIT_MASS = 1  /* c_s = 24/(13 pi), c_t = 3/4: the density integrates to 1 */
} stkde_kernel_constants;

typedef struct {
    int device;            /* CUDA device ordinal */
    void* stream;          /* cudaStream_t the work is ordered on; NULL = legacy default stream */
    int form;              /* stkde_form */
    int kernel_constants;  /* stkde_kernel_constants */
    int t_block;           /* reserved, must be 0 (tiles span 256 voxels of T in the tensor
                              forms and 64 in the fp32 form) */
    int slab;              /* T extent of an event bin: 0 = automatic (tensor forms: the
                              smallest power of two from 4 to 16 giving at least 3.5
                              events per bin on average, 1.8 for the tf32 forms; fp32
                              form: 64), else >= 1 */
    int profile;           /* 1: time each phase with CUDA events (see stkde_phase_times) */
} stkde_options;

typedef struct {
    double x0, y0, t0;     /* domain origin: the corner of voxel (0, 0, 0) */
    double sres, tres;     /* voxel size in space (x and y) and in time, > 0 */
    int64_t gx, gy, gt;    /* grid size in voxels, >= 1 each */
} stkde_grid;

/* Fills *opt with the defaults: device 0, legacy stream, tensor bf16x3 form,
 * printed constants, automatic tiling, no profiling. */
STKDE_API void stkde_default_options(stkde_options* opt);

/* Creates a context on opt->device (opt may be NULL for the defaults).
 * Returns STKDE_ERR_UNSUPPORTED if the device is not compute capability 10.3. */
STKDE_API stkde_status stkde_create(stkde_ctx** ctx, const stkde_options* opt);

/* Section 2.1 density of n events on `grid`, bandwidths hs and ht, written to
 * `out` (gx*gy*gt binary32, row-major [X][Y][T]).  `out` may be device memory
 * of the context's device or host memory; with host memory the result is
 * computed into a context-owned device buffer and copied back (pinned memory:
 * asynchronously; pageable memory: the call returns after the copy).  With the
 * tensor forms a host grid of at least 128 MB is computed in slabs along X and
 * each slab is copied on a second stream while the later slabs compute; the
 * context's stream waits for those copies.  `points` may be NULL only when
 * n == 0.
 * Errors: INVALID_ARGUMENT (NULL pointers, n < 0 or n >= 2^31, non-positive or
 * non-finite hs, ht, sres, tres, a grid dimension < 1 or >= 2^31, or an
 * origin that is not finite), OOM (workspace), CUDA. */
STKDE_API stkde_status stkde_compute(stkde_ctx* ctx, const double* points, int64_t n,
                           const stkde_grid* grid, double hs, double ht, float* out);

/* One problem of a batch. */
typedef struct {
    const double* points;  /* n x 3 doubles, host or device */
    int64_t n;
    stkde_grid grid;
    double hs, ht;
    float* out;            /* device memory, gx*gy*gt binary32 */
} stkde_problem;

/* Computes `count` independent problems in one batched call (the paper's
 * runs are one problem each; batching is this library's addition for many small
 * problems): one re-centre, one binning sort and one bin-bounds pass over the
 * concatenated events of all problems, then one tile-kernel launch over the
 * tiles of every problem (the tensor forms: a persistent kernel whose work
 * queue holds them heaviest first; the fp32 form: one block per tile).  The
 * problem table travels in kernel parameters, so the call keeps no pointer to
 * `problems` after it returns.
 * Each result is bit-identical to the problem computed alone by stkde_compute
 * with the same form.  Events may be host or device memory per problem; outputs
 * must be device memory of the context's device.  Errors: INVALID_ARGUMENT (any
 * problem fails stkde_compute's checks, or an output is not device memory;
 * nothing is enqueued), UNSUPPORTED (the scatter form, or a batch of 2^31 events,
 * 2^32 bins or 2^31 tiles or more), OOM, CUDA.  count = 0 is a no-op. */
STKDE_API stkde_status stkde_compute_batch(stkde_ctx* ctx, const stkde_problem* problems, int count);

/* The Section 2.1 density with one bandwidth pair per event, the bandwidth that
 * adapts to the local population density which Section 8 (Conclusion) names as
 * future work; the caller chooses the bandwidths.  Event i adds
 *     k_s((x - x_i)/hs[i], (y - y_i)/hs[i]) k_t((t - t_i)/ht[i]) / (n hs[i]^2 ht[i])
 * to every voxel inside its own cylinder (spatial test strict, temporal
 * inclusive), so hs[i] = hs, ht[i] = ht for all i gives stkde_compute's density.
 * hs, ht: n doubles each, domain units, host or device memory (each on its
 * own); points, grid and out as in stkde_compute.  Event binning and tile reach
 * use the largest bandwidths, so a few very large ones slow every tile.  The
 * call waits for the stream once, to read the bandwidth range (host arrays are
 * first copied into a context-owned device buffer).  Errors: INVALID_ARGUMENT (as stkde_compute; a NULL hs or ht with
 * n > 0; a bandwidth that is not finite and positive, or hs[i]/sres or
 * ht[i]/tres >= 1e6), UNSUPPORTED (the scatter form; the fp16x3 form when
 * (max hs / min hs)^2 (max ht / min ht) > 2^14, where its weighted operand
 * would leave the fp16 range), OOM, CUDA.  n = 0 writes zeros. */
STKDE_API stkde_status stkde_compute_adaptive(stkde_ctx* ctx, const double* points, int64_t n,
                                              const stkde_grid* grid, const double* hs,
                                              const double* ht, float* out);

/* Number of (event, in-grid voxel) pairs inside the bandwidth cylinder
 * (spatial test strict, temporal inclusive): the voxel-point updates of the
 * problem.  Synchronous; FP64 arithmetic on the re-centred binary32 events. */
STKDE_API stkde_status stkde_count_updates(stkde_ctx* ctx, const double* points, int64_t n,
                                 const stkde_grid* grid, double hs, double ht,
                                 uint64_t* count);

/* Per-event bandwidths that follow the population density, for
 * stkde_compute_adaptive: Abramson's square-root law on a pilot density.  The
 * pilot is the density with the fixed pair (hs, ht), computed as by
 * stkde_compute into `pilot` (device memory, gx*gy*gt binary32) or, when pilot is
 * NULL, into a context-owned buffer.  It is read at each event's voxel
 * (floor((x - x0)/sres) etc., clamped into the grid) and floored at 1e-6 of the
 * largest such value, f_i; with g the geometric mean of the f_i,
 *     lambda_i = clamp((f_i / g)^(-alpha), lam_min, lam_max),
 *     hs_out[i] = hs lambda_i,   ht_out[i] = ht lambda_i
 * (device memory, n doubles each).  alpha = 1/2 is Abramson's law, alpha = 0
 * gives the fixed pair.  Dense areas get narrower kernels.  Errors:
 * INVALID_ARGUMENT (as stkde_compute; alpha negative or not finite; lam_min not
 * in (0, 1]; lam_max not finite or below 1; outputs or pilot not device memory),
 * OOM, CUDA.  n = 0 leaves the outputs untouched (and zeroes a given pilot). */
STKDE_API stkde_status stkde_abramson_bandwidths(stkde_ctx* ctx, const double* points, int64_t n,
                                                 const stkde_grid* grid, double hs, double ht,
                                                 double alpha, double lam_min, double lam_max,
                                                 float* pilot, double* hs_out, double* ht_out);

/* stkde_count_updates with per-event bandwidths hs, ht (as in
 * stkde_compute_adaptive): the pairs inside each event's own cylinder.
 * Synchronous.  Errors as stkde_compute_adaptive's INVALID_ARGUMENT cases. */
STKDE_API stkde_status stkde_count_updates_adaptive(stkde_ctx* ctx, const double* points, int64_t n,
                                                    const stkde_grid* grid, const double* hs,
                                                    const double* ht, uint64_t* count);

/* Waits for the context's stream and returns the first latched device error,
 * clearing it. */
STKDE_API stkde_status stkde_synchronize(stkde_ctx* ctx);

/* With options.profile = 1: fills ms[0..k) with the durations of the phases of
 * the last stkde_compute (0 re-centre, 1 binning sort, 2 bin boundaries and
 * gather, 3 tile kernel) and returns k; waits for the stream.  Returns 0 when
 * profiling is off. */
STKDE_API int stkde_phase_times(stkde_ctx* ctx, float* ms, int cap);

/* Number of library kernels the last stkde_compute enqueued (0 for a NULL ctx). */
STKDE_API int stkde_last_launch_count(stkde_ctx* ctx);

/* Largest problem stkde_compute_static accepts: events, and bin boundaries
 * (number of event bins + 1; a bin is 16 x 8 voxels in the plane by a slab of
 * at least 4 voxels of T, so at most about gx*gy*gt/512 bins). */
#define STKDE_STATIC_MAX_EVENTS 262144
#define STKDE_STATIC_MAX_BINS 1048576

/* stkde_compute without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code where
 * another component owns every device allocation (a host application's or a
 * framework's memory pool, an arena reserved up front), or a loop that must not
 * take the device-wide synchronisation of cudaMalloc/cudaFree.  It needs no
 * context: `points` (n x 3 doubles) and `out` (gx*gy*gt binary32) must be
 * device memory of the current device, the work is ordered on `stream`
 * (cudaStream_t, NULL = legacy default stream), `form` and `kernel_constants`
 * are as in stkde_options.  All scratch lives in one fixed file-scope device
 * array of about 16 MB that every device loading the library keeps until the
 * process exits; its device address is looked up on every call made outside
 * stream capture, and a call made while `stream` is being captured uses the
 * address the last call on that device found, so make a first call on each
 * device before any capture (a captured call with no such predecessor, or with
 * sync != 0, returns STKDE_ERR_UNSUPPORTED).  All calls on a device share that
 * array: calls whose work overlaps on the GPU race and must be serialised by
 * the caller.
 * Returns STKDE_ERR_UNSUPPORTED, before any launch, when n exceeds
 * STKDE_STATIC_MAX_EVENTS or the grid needs more than STKDE_STATIC_MAX_BINS bin
 * boundaries; INVALID_ARGUMENT for host pointers or the argument errors of
 * stkde_compute.  With sync != 0 the call waits for the stream and returns
 * device-side errors (non-finite coordinates, timeouts); with sync == 0 it
 * returns after enqueueing and device-side errors are not reported. */
STKDE_API stkde_status stkde_compute_static(const double* points, int64_t n,
                                            const stkde_grid* grid, double hs, double ht,
                                            float* out, int form, int kernel_constants,
                                            void* stream, int sync);

/* Grows the context's workspace to at least `bytes` now (waiting for the stream
 * if it must grow), so that later calls whose workspace fits allocate nothing:
 * a serving loop then never takes the device-wide synchronisation of
 * cudaMalloc/cudaFree, and the calls can be captured into a CUDA graph.  A
 * problem of n events needs about 56 n bytes plus 4 bytes per 512 voxels of
 * grid (more with host events or per-event bandwidths).  The workspace never
 * shrinks before stkde_destroy.  Errors: INVALID_ARGUMENT (NULL ctx), OOM (the
 * workspace is then empty; the context stays usable), UNSUPPORTED (during
 * stream capture). */
STKDE_API stkde_status stkde_reserve(stkde_ctx* ctx, size_t bytes);

/* Frees the context and its workspace (waits for its stream first). */
STKDE_API void stkde_destroy(stkde_ctx* ctx);

/* Static description of a status code. */
STKDE_API const char* stkde_status_string(stkde_status s);

#ifdef __cplusplus
}
#endif

#endif /* STKDE_H */
