/*
 * dd_inpaint -- homogeneous diffusion inpainting by multilevel optimised
 * restricted additive Schwarz (ORAS) on one GB300 GPU (sm_103a).
 *
 * Problem (Kaemper & Weickert, "Domain decomposition algorithms for
 * real-time homogeneous diffusion inpainting in 4K", Sec. 2, Eq. eq:inp,
 * eq:homdiff, eq:ls): per colour channel solve A u = b with
 * A = C - (I - C) L, b = C f, where C is the 0/1 diagonal mask of known
 * pixels and L the 5-point Laplacian with reflecting image boundaries
 * (grid size 1).  Known pixels keep u = f; the others satisfy the discrete
 * Laplace equation.  All channels share one mask (Sec. 2, last paragraph).
 *
 * Method (Sec. 3-4): overlapping square blocks of side `block` at stride
 * block - overlap; each sweep solves every block's local problem
 * R_i A R_i^T v_i = R_i r^n (Eq. eq:ras-local-problem) by `local_cg_iters`
 * conjugate-gradient steps with a Robin interface condition (ORAS), and adds
 * the corrections back on disjoint owned cores (restricted add-back with a
 * 0/1 partition of unity).  The multilevel variant solves dyadically
 * subsampled problems coarse to fine (Sec. 4).
 *
 * Conventions for every entry point:
 *  - images are channel-planar, row-major float32 arrays C x H x W with no
 *    padding (element (c, y, x) at index (c*H + y)*W + x);
 *  - masks are H x W bytes, nonzero = known pixel;
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream); work is enqueued on it.  Calls that must read a convergence
 *    test back to the host synchronise that stream before returning; this
 *    is stated per function;
 *  - device pointers must be device-accessible memory of the current device
 *    (e.g. torch CUDA tensors); host pointers ordinary host memory;
 *  - the library never takes ownership of caller buffers;
 *  - return codes are DD_* below; no entry point aborts the process.
 *  - handles are not thread-safe; distinct handles are independent.
 */
#ifndef DD_INPAINT_H
#define DD_INPAINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status codes */
#define DD_OK             0
#define DD_EINVAL         1  /* bad size, NULL pointer, block <= overlap, bad enum */
#define DD_EEMPTYMASK     2  /* no known pixel: A is singular under reflecting boundaries */
#define DD_ENOMEM         3  /* device or host allocation failed */
#define DD_ENOTCONVERGED  4  /* sweep limit reached; the best iterate is still written */
#define DD_ENUMERIC       5  /* NaN or Inf met in a residual norm */
#define DD_ECUDA          6  /* a CUDA runtime call failed (message: dd_last_error) */
#define DD_ETIMEOUT       7  /* a bounded device-side wait gave up */
#define DD_EAGAIN         8  /* asynchronous work not finished yet (dd_inpaint_query) */

/* level solvers */
#define DD_SOLVER_ORAS    0  /* restricted additive Schwarz with Robin interfaces (Sec. 3-4) */
#define DD_SOLVER_CG      1  /* conjugate gradients on the whole image: the comparison solver of
                                Sec. 5 (with levels > 1: multilevel CG of Bornemann & Deuflhard) */

/* multilevel modes */
#define DD_ML_CASCADE     0  /* coarse-to-fine initialisation (Sec. 4) */
#define DD_ML_CORRECTION  1  /* cascade initialisation, then a coarse-grid correction of the residual
                                after each fine sweep, or after each one from the first slow pass on
                                (params.correction_trigger; FP32, ORAS, levels >= 2) */

/* precision modes (storage of the Schwarz iterate; arithmetic is FP32) */
#define DD_PREC_FP32      0  /* plain FP32 ORAS on u, FP64-verified stop test */
#define DD_PREC_FP32_REF  1  /* FP32 inner solves + FP64 outer residual correction */
#define DD_PREC_FP16_REF  2  /* FP16 storage inner solves + FP64 outer residual correction */
#define DD_PREC_BF16_REF  3  /* BF16 storage inner solves + FP64 outer residual correction */

typedef struct dd_inpaint *dd_handle;
typedef struct dd_batch *dd_batch_handle;

typedef struct dd_params {
    int    block;            /* block side in pixels: 16, 32, 64 or 96 (default 32, Sec. 4) */
    int    overlap;          /* overlap in pixels, 0 <= overlap < block (default 6, Sec. 4) */
    int    local_cg_iters;   /* CG steps per local problem and sweep, >= 1 (default 16) */
    int    levels;           /* solved resolution levels, 1..8 (default 3, Sec. 4) */
    int    ml_mode;          /* DD_ML_CASCADE (default) or DD_ML_CORRECTION */
    int    coarse_factor;    /* 2 (default; 0 also means 2), 4 or 8: each solved level is this many
                                times coarser per axis than the next finer one.  With 4 or 8 the
                                dyadic levels in between are built by the 2x2 restriction and
                                passed through by the prolongation, without sweeps; at most 8
                                dyadic levels in all.  DD_ML_CORRECTION corrects on the coarsest
                                level */
    float  robin_p;          /* Robin interface weight p > 0 (1 = RAS); <= 0 selects the default */
    int    precision;        /* DD_PREC_* (default DD_PREC_FP32_REF) */
    int    max_sweeps;       /* fine-level sweep limit per solve (default 400) */
    int    inputs_on_device; /* 1: mask/values pointers are device memory; 0: host */
    double coarse_tol;       /* relative residual that ends a coarse level (default 1e-2) */
    double inner_tol;        /* relative residual decrease per outer correction (default 3e-3) */
    int    max_corrections;  /* outer FP64 corrections limit (default 30) */
    int    coarse_sweeps;    /* sweep limit per coarse level (default 12) */
    int    timing;           /* 1: time every fine-level sweep launch with CUDA events (dd_stats) */
    int    tile_warps;       /* warps holding one block tile: 0 = default; block 16: 1;
                                block 32: 1, 2 or 4; block 64: 4 or 8; block 96: 12 */
    int    solver;           /* DD_SOLVER_ORAS (default) or DD_SOLVER_CG (needs DD_PREC_FP32);
                                with CG, max_sweeps / coarse_sweeps count CG iterations */
    int    correction_sweeps; /* DD_ML_CORRECTION: ORAS sweeps on the coarse correction equation
                                after each fine sweep, from zero (default 2) */
    double local_rtol;       /* in [0, 1): a block's local CG also stops once its residual fell by this
                                factor (default 0: always local_cg_iters steps, as in the paper) */
    int    device_loop;      /* 1 (default): a level's sweeps (or CG iterations) repeat inside a
                                CUDA graph loop on the device until its stop test or sweep limit,
                                no launch after the stop; 0: launched in fixed chunks whose launches
                                after the stop do no work.  Timing (timing = 1) always uses
                                launches */
    int    test_stall_polls; /* tests only, 0 (default) = off.  > 0: in every sweep launch, each
                                CTA's first wait for a staged tile polls a barrier that no copy
                                ever completes, this many times, and then gives up as it would
                                for a hung copy.  The solve then ends with DD_ETIMEOUT (the
                                copies in flight are waited for, nothing faults) and the handle
                                stays usable.  It exercises the timeout path without a fault */
    double correction_trigger; /* DD_ML_CORRECTION: 0 (default) corrects after every fine sweep.  In
                                (0, 1): the fine sweeps run alone until the second pass in a row
                                that reduced the fine relative residual by less than this factor
                                (w_n > trigger w_{n-1}) while it is still above 4 tol: plain sweeps
                                have slowed down to the contraction of a smooth error mode, which
                                the coarse grid removes.  From the next sweep on every sweep is
                                followed by the correction; a correction that does not reduce the
                                residual pauses them until a plain pass is slow again.  Decided on the
                                device; in device loops the two phases are two graph loops, so the
                                plain phase costs what the cascade alone does */
    double final_local_rtol; /* 0 (default): every sweep uses local_rtol.  In (0, 1): a sweep that the
                                device stop test predicts to be a level's last one (its input
                                residual, extrapolated from the last two sweeps, within a factor
                                1/0.6 of the tolerance) ends its local CG once the local residual
                                fell by this factor instead.  The last sweep only has to close a
                                small gap, so looser local solves do; if it falls short, the
                                following sweeps run as usual (the global test decides, Sec. 4) */
    int    correction_cg;    /* DD_ML_CORRECTION: 0 (default) solves the coarse correction equation
                                by correction_sweeps ORAS sweeps from zero.  > 0: by conjugate
                                gradients on a coarse level held in one SM's shared memory (one CTA
                                per channel, FP64 dot products), at most this many iterations, to
                                relative residual 1e-3.  That level has at most 12288 pixels: below
                                the cascade's coarsest level the 2x2 restriction continues with
                                correction-only levels (no sweeps) until one fits, within 8 dyadic
                                levels in all (else DD_EINVAL at create) */
    double local_atol;       /* 0 (default): no absolute local stop.  In (0, 1): a block's local CG
                                also stops once its residual norm is at most local_atol * tol *
                                ||b - A u0|| / sqrt(blocks per channel), the block's share of the
                                level's stop test scaled by local_atol; blocks whose residual is
                                already below it take no CG step.  Below 1 the level cannot stall:
                                while its residual is above tol, some block is above its share and
                                iterates.  Applies when the level's tolerance is positive */
} dd_params;

#define DD_MAX_STAT_CHANNELS 16
#define DD_MAX_LEVELS 8

typedef struct dd_stats {
    int    sweeps_total;                       /* ORAS sweeps of the last solve, all levels */
    int    sweeps_per_level[DD_MAX_LEVELS];    /* per dyadic level, 0 = finest (with coarse_factor
                                                  4 or 8 the pass-through levels show 0) */
    int    corrections;                        /* FP64 outer corrections applied */
    int    converged;                          /* 1 if the stop test held */
    int    channels;
    double rel_residual[DD_MAX_STAT_CHANNELS]; /* FP64 ||b-Au||/||b-Au0|| of the output, u0 = Cf */
    double ms_total;                           /* time of the last solve on its stream (CUDA events
                                                  around all of its work, a host-controlled
                                                  continuation included) */
    size_t device_bytes;                       /* device memory owned by the handle */
    long long kernel_launches;                 /* CUDA kernels launched through the handle since create */
    long long local_unknowns;                  /* unknown pixels summed over the fine level's blocks,
                                                  one channel (work of one local problem set) */
    int    fine_sweep_launches;                /* timed fine-level sweep launches (params.timing) */
    double fine_sweep_ms;                      /* their summed device time */
    long long fine_cg_pixel_steps;             /* params.timing: over the fine level's full sweeps, the sum
                                                  of unknown block pixels x local CG steps taken */
    long long fine_swept_unknowns;             /* params.timing: unknown block pixels of those sweeps */
    int    host_continued;                     /* 1: the enqueued part of the solve ended above tol and
                                                  dd_inpaint_solve_finish continued under host control,
                                                  rewriting u_out (work enqueued on the stream after
                                                  dd_inpaint_solve_async saw the earlier result) */
    int    coarse_corrections;                 /* DD_ML_CORRECTION: coarse-grid corrections applied to
                                                  the fine iterate in the last solve */
} dd_stats;

/* Fill *p with the defaults listed above. */
void dd_params_default(dd_params *p);

/* Human-readable text for a DD_* code (static storage). */
const char *dd_strerror(int code);

/* Text of the last DD_ECUDA / DD_EINVAL cause on this thread (static per thread). */
const char *dd_last_error(void);

/*
 * Create a solver for one frame (H x W, C channels) and copy its data.
 *   mask:   H*W bytes, nonzero = known (host or device per inputs_on_device);
 *   values: C*H*W floats, read only where mask != 0;
 *   params: NULL = defaults;  out: receives the handle.
 * The caller's buffers may be freed when the call returns.  Allocates all
 * device memory the solves need (dd_stats.device_bytes).  Synchronous.
 * Errors: DD_EINVAL, DD_EEMPTYMASK, DD_ENOMEM, DD_ECUDA (no handle is made).
 */
int dd_inpaint_create(int H, int W, int C, const uint8_t *mask, const float *values,
                      const dd_params *params, dd_handle *out);

/*
 * Solve to relative residual `tol` (per channel ||b - A u|| / ||b - A u0||,
 * u0 = C f; stop when the maximum over channels is <= tol) and write the
 * solution to u_out (DEVICE, C*H*W floats, caller-owned).  With device_loop
 * = 1 (the default) each level's sweeps repeat on the device until its stop
 * test and the host reads the result once; with device_loop = 0 the stop test
 * is read back after each chunk of launches.  Either way the call synchronises
 * `stream`.  Starts from the handle's iterate if dd_inpaint_set_data(...,
 * keep_iterate=1) asked for a warm start, else from the multilevel
 * initialisation.  For the same inputs and parameters the result, the sweep
 * counts and the residual norms are bitwise repeatable, whatever else runs on
 * the GPU (the residual sums are exact fixed-point sums).
 * Errors: DD_EINVAL, DD_ENOTCONVERGED (u_out still holds the best iterate),
 * DD_ENUMERIC, DD_ETIMEOUT, DD_ECUDA.
 */
int dd_inpaint_solve(dd_handle h, float *u_out, double tol, void *stream);

/* Release the handle and its device memory.  NULL-safe; returns DD_OK. */
int dd_inpaint_destroy(dd_handle h);

/*
 * Replace mask and values (same H, W, C; pointers as in create).  With
 * keep_iterate = 1 the current fine iterate is kept as the next solve's
 * starting point (known pixels reset to the new values): warm start for
 * video.  Synchronous.  Errors: DD_EINVAL, DD_EEMPTYMASK, DD_ECUDA; after an
 * error the handle needs a successful set_data before the next solve.
 */
int dd_inpaint_set_data(dd_handle h, const uint8_t *mask, const float *values, int keep_iterate);

/* Copy the statistics of the last solve.  Errors: DD_EINVAL. */
int dd_inpaint_stats(dd_handle h, dd_stats *out);

/* ---------------------------------------------------------------------------
 * Asynchronous use (precision DD_PREC_FP32, or any DD_PREC_*_REF precision with
 * device_loop = 1, whose correction loop then runs on the device).  The solve
 * is split into an enqueue that returns at once and a finish that waits for
 * the result, so one host thread can keep several handles (on several streams)
 * busy and data copies can overlap solves.  Sec. 3-4 of the paper (the same
 * method).
 * ------------------------------------------------------------------------- */

/*
 * As dd_inpaint_set_data, but only enqueued on stream (host inputs must be
 * pinned for the copy to be asynchronous).  The empty-mask test is reported
 * by the next dd_inpaint_solve_finish (DD_EEMPTYMASK).  Errors: DD_EINVAL
 * (NULL pointers, a solve in flight), DD_ECUDA.
 */
int dd_inpaint_set_data_async(dd_handle h, const uint8_t *mask, const float *values, int keep_iterate,
                              void *stream);

/*
 * Enqueue a solve to relative residual tol on stream: the multilevel
 * initialisation, the fine sweeps under the device stop test (with
 * device_loop = 0: the first 16; with a correction precision: the whole
 * correction loop), the output of the resolved iterate to u_out (DEVICE,
 * C*H*W floats) and its residual.  Returns without waiting.  Errors:
 * DD_EINVAL (a correction precision with device_loop = 0, a solve in flight),
 * DD_EEMPTYMASK, DD_ECUDA.
 */
int dd_inpaint_solve_async(dd_handle h, float *u_out, double tol, void *stream);

/* DD_OK if the enqueued solve's device work is done, DD_EAGAIN if not (or if
 * it was started by a batch launch), DD_EINVAL if none is in flight. */
int dd_inpaint_query(dd_handle h);

/*
 * Wait for the enqueued solve and return its status as dd_inpaint_solve would.
 * If the enqueued part did not reach tol (with params.device_loop = 0: the
 * first 16 fine sweeps; with device loops: the sweep limit, or an FP32 stop
 * test that the FP64-accurate residual overrules), the remaining sweeps run
 * here on stream under host control, u_out is rewritten and
 * stats.host_continued is set.
 */
int dd_inpaint_solve_finish(dd_handle h, void *stream);

/*
 * Batched solves in one CUDA graph (mode DD_BATCH_GRAPH, see
 * dd_batch_create_mode): the FP32 solves of n handles, each on its
 * own forked stream, are captured once and replayed by dd_batch_launch, so
 * frames of different sizes run concurrently and the whole batch is one graph
 * launch.  handles: n distinct FP32 handles; u_out[i]: DEVICE output of handle
 * i (C*H*W floats, fixed for the life of the batch); tol baked into the graph.
 * Each launch solves the data currently loaded in every handle, starting from
 * the multilevel initialisation.  With params.device_loop = 1 every level's
 * sweeps run in a WHILE node of the batch graph (the pass count is known after
 * dd_batch_finish and enters each handle's kernel_launches); kernels_per_launch
 * (may be NULL) receives the number of kernel nodes outside those loops.
 * Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA.
 */
int dd_batch_create(int n, const dd_handle *handles, float *const *u_out, double tol, dd_batch_handle *out,
                    long long *kernels_per_launch);

/* batch modes */
#define DD_BATCH_GRAPH       0  /* each frame's solve on a stream of its own, all in one graph */
#define DD_BATCH_PERSISTENT  1  /* level by level: one persistent launch per sweep over the blocks of all
                                   frames (their channels and uneven boundary blocks included), each
                                   frame with its own stop test, in one graph */

/*
 * As dd_batch_create, with the batch mode.  DD_BATCH_PERSISTENT needs
 * DD_PREC_FP32 / DD_SOLVER_ORAS / DD_ML_CASCADE handles with device_loop = 1,
 * timing 0 and the same block, overlap and tile_warps (sizes, masks, level
 * counts and the other parameters may differ); at most 1024 handles.  Every
 * level of the cascade is then one graph loop whose passes each sweep all
 * frames still iterating on that level in a single persistent launch; a frame
 * drops out at its own stop test or sweep limit.  The results are those of the
 * frames' solves alone (the same kernel arithmetic per block).
 * Errors: DD_EINVAL (mode or handle requirements), DD_ENOMEM, DD_ECUDA.
 */
int dd_batch_create_mode(int n, const dd_handle *handles, float *const *u_out, double tol, int mode,
                         dd_batch_handle *out, long long *kernels_per_launch);

/* Launch the batch graph on stream (returns at once).  Errors: DD_EINVAL
 * (previous launch not finished), DD_EEMPTYMASK, DD_ECUDA. */
int dd_batch_launch(dd_batch_handle b, void *stream);

/*
 * Wait for the launch and finish every handle's solve (unconverged ones
 * continue on stream).  status (may be NULL): n per-handle codes.  Returns the
 * first non-DD_OK code, else DD_OK.  Statistics are then per handle.
 */
int dd_batch_finish(dd_batch_handle b, void *stream, int *status);

/* Release the batch (waits for a launch in flight).  NULL-safe. */
int dd_batch_destroy(dd_batch_handle b);

/* ---------------------------------------------------------------------------
 * Step-level entry points (one step of the method on caller device buffers;
 * used to check each step against an independent implementation).
 * ------------------------------------------------------------------------- */

/*
 * Set the finest-level iterate from u (DEVICE, C*H*W floats) exactly as
 * given (no reset of known pixels).  Subsequent dd_inpaint_sweep calls start
 * from it.  Enqueued on stream.  Errors: DD_EINVAL, DD_ECUDA.
 */
int dd_inpaint_set_iterate(dd_handle h, const float *u, void *stream);

/* Copy the finest-level iterate to u_out (DEVICE, C*H*W floats). */
int dd_inpaint_get_iterate(dd_handle h, float *u_out, void *stream);

/*
 * Apply n ORAS sweeps (Sec. 3, u^{n+1} = u^n + sum_i R_i^T D_i v_i^n) to the
 * finest-level iterate, in FP32 storage, with the handle's block, overlap,
 * Robin weight and CG step count; with DD_ML_CORRECTION each sweep is followed
 * by the coarse-grid correction (one pass of that mode).  If rnorm_out is not
 * NULL it receives C values: ||b - A u^n||_2 of the INPUT iterate of the last
 * sweep (FP32 terms, FP64 accumulation); the call then synchronises stream.
 * Errors: DD_EINVAL, DD_ECUDA.
 */
int dd_inpaint_sweep(dd_handle h, int n, double *rnorm_out, void *stream);

/*
 * Dyadic subsampling of mask and known values (Sec. 4): coarse pixel
 * (Y, X) covers fine pixels {2Y, 2Y+1} x {2X, 2X+1} inside the image; it is
 * known iff one of them is known, and its value is the mean of the known fine
 * values (0 where unknown).  Sizes Hc = ceil(H/2), Wc = ceil(W/2).
 *   mask (H*W bytes), f (C*H*W floats): DEVICE inputs;
 *   mask_c (Hc*Wc bytes), f_c (C*Hc*Wc floats): DEVICE outputs.
 * Enqueued on stream.  Errors: DD_EINVAL, DD_ECUDA.
 */
int dd_restrict(int H, int W, int C, const uint8_t *mask, const float *f,
                uint8_t *mask_c, float *f_c, void *stream);

/*
 * Coarse-to-fine prolongation: cell-centred bilinear interpolation of
 * u_c (C x Hc x Wc) onto C x H x W (fine pixel i sits at coarse coordinate
 * (i - 0.5)/2, clamped to the coarse grid).  If mask/f are not NULL, pixels
 * with mask != 0 are then set to f (the initialisation of Sec. 4).
 * All pointers DEVICE.  Enqueued on stream.  Errors: DD_EINVAL, DD_ECUDA.
 */
int dd_prolong(int Hc, int Wc, int H, int W, int C, const float *u_c, const uint8_t *mask,
               const float *f, float *u, void *stream);

/*
 * Small-grid coarse solve (the coarse problem of Sec. 4, the operator of
 * Sec. 2 on a coarse grid): conjugate gradients on A e = g with e = 0 where
 * mask != 0 (reflecting image borders, h = 1), from e = 0, until
 * ||g - A e|| <= tol ||g|| or max_iter iterations.  One CTA per channel holds
 * the grid in shared memory: H*W <= 12288.
 *   mask (H*W bytes), g, e (C*H*W floats): DEVICE, dense;
 *   iters: HOST array of C ints (iterations taken) or NULL.
 * Enqueued on stream; with iters != NULL the call synchronises stream.
 * Errors: DD_EINVAL (sizes, NULL pointers), DD_ECUDA.
 */
int dd_coarse_cg(int H, int W, int C, const uint8_t *mask, const float *g, float *e, int max_iter, double tol,
                 int *iters, void *stream);

/*
 * FP64 residual norms ||b - A u||_2 per channel of a float32 iterate u, and
 * the reference norms ||b - A u0||_2, u0 = C f (Sec. 2, Eq. eq:ls).  mask, f, u
 * are DEVICE; norms and ref_norms HOST arrays of C doubles (either may be
 * NULL).  Synchronises stream.  Errors: DD_EINVAL, DD_ECUDA.
 */
int dd_residual_norms(int H, int W, int C, const uint8_t *mask, const float *f,
                      const float *u, double *norms, double *ref_norms, void *stream);

/*
 * Allocation-free solve (the paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory).  Some callers must not call
 * cudaMalloc: code inside a host framework that owns the device allocator (for
 * example a caching pool it does not want bypassed), plug-ins that may not grow
 * the process's device footprint, and real-time paths where an allocation's
 * latency or failure is not acceptable.  This call runs the same one-level FP32
 * ORAS sweeps as dd_inpaint_solve with levels = 1 and precision = DD_PREC_FP32,
 * but takes all its scratch from one fixed-size device array that is part of
 * the library (about 42 MiB).  The array is committed on a device when the
 * library's module is loaded there: under CUDA's default lazy module loading
 * that is this call's first use on the device, which then pays the load
 * latency and can fail with DD_ECUDA if device memory is short, so a real-time
 * caller should make one warm-up call at start-up.  The array stays until the
 * process exits.  The call itself runs no cudaMalloc, cudaFree or other
 * allocating routine.
 *   mask (H*W bytes), values (C*H*W floats), u_out (C*H*W floats): DEVICE;
 *   params: NULL = defaults; block, overlap, local_cg_iters, local_rtol,
 *   robin_p, tile_warps, max_sweeps and test_stall_polls are used; solver must
 *   be DD_SOLVER_ORAS; levels, ml_mode, coarse_factor, precision and the
 *   other fields are ignored;
 *   tol: relative residual target as in dd_inpaint_solve (FP64-verified).
 * Capacity: C <= 16, C*H*roundup(W,32) <= 4194304, at most 16384 blocks per
 * channel, blocks x threads per block <= 1048576 (32 threads per block for
 * block = 16 or 32 with one warp, up to 256 for block = 64) and 65536 blocks
 * of the residual pass over all channels; larger inputs return DD_EINVAL
 * (dd_last_error() says which limit) before any GPU work.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the array and it keeps the previous call's
 * contents: calls whose GPU work overlaps (other streams or host threads) race
 * and give wrong results, so serialise them.  Synchronises stream.
 * Errors: DD_EINVAL, DD_EEMPTYMASK, DD_ENOTCONVERGED (u_out still written),
 * DD_ENUMERIC, DD_ETIMEOUT, DD_ECUDA.
 */
int dd_inpaint_solve_static(int H, int W, int C, const uint8_t *mask, const float *values, float *u_out,
                            const dd_params *params, double tol, void *stream);

/* ---------------------------------------------------------------------------
 * Device budget and measurement (the paper has no counterpart).
 * ------------------------------------------------------------------------- */

/*
 * Cap the device memory that all live handles of this process may hold
 * together (bytes; 0, the default, means no cap beyond the GPU's own).  An
 * allocation that would exceed the cap fails as an out-of-memory would:
 * dd_inpaint_create returns DD_ENOMEM and makes no handle.  Existing handles
 * are not affected.  Thread-safe.
 */
void dd_set_device_budget(size_t bytes);

/* Device bytes held by all live handles of this process (dd_stats.device_bytes
 * summed).  Thread-safe. */
size_t dd_device_bytes_in_use(void);

/*
 * FP32 FMA throughput of the current device, measured: a grid of the maximum
 * resident warps per SM runs independent chains of packed FP32 FMAs
 * (__ffma2_rn), timed with CUDA events on stream, best of `reps` launches
 * after one warm-up.  *tflops receives TFLOP/s (2 flops per FMA); *sm_count
 * (may be NULL) the device's SM count.  This is the denominator of the sweep
 * kernel's roofline.  Allocates and frees a few KB of device memory.
 * Synchronises stream.  Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA.
 */
int dd_fp32_fma_peak(int reps, double *tflops, int *sm_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DD_INPAINT_H */
