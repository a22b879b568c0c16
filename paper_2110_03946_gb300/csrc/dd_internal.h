// Internal interfaces between the translation units of the dd_inpaint library.
// Not part of the public C ABI (that is include/dd_inpaint.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace dd {

// Storage type of a Schwarz iterate (arithmetic is always FP32).
enum class Store : int { F32 = 0, F16 = 1, BF16 = 2 };

inline size_t store_bytes(Store s) { return s == Store::F32 ? 4 : 2; }

// Block layout of one resolution level (Sec. 4 of the paper): blocks of side b
// at stride s = b - o, count max(1, ceil((n - o)/s)) per axis, the last block
// clipped to the image; pixel x of an axis is owned by block
// clamp(floor((x - floor(o/2))/s), 0, n - 1).
struct TileGeom {
    int H = 0, W = 0, pitch = 0;  // image size; row pitch of the level's buffers (elements)
    int b = 32, o = 6, s = 26, half_o = 3;
    int nw = 1;                   // warps that hold one block tile
    int ntx = 0, nty = 0, ntiles = 0;
};

int axis_blocks(int n, int b, int o);
// nw <= 0 selects default_tile_warps(b)
TileGeom make_geom(int H, int W, int pitch, int b, int o, int nw = 0);

// Kernel shape chosen for a block side and warps per tile: threads per
// block-tile and the number of 32-bit mask words per tile (known bits +
// owned bits per thread).  Supported: b = 16 (1 warp), 32 (1, 2 or 4 warps),
// 64 (4 or 8 warps), 96 (12 warps).
bool block_supported(int b);
int default_tile_warps(int b);
bool tile_warps_supported(int b, int nw);
int tile_threads(int b, int nw);
size_t tmask_words(const TileGeom& g);

// Per-tile, per-thread bit masks: bit set in word 0 = pixel known or outside
// the tile, bit set in word 1 = pixel owned by the tile (restricted add-back).
// With count, *count += the unknown in-tile pixels summed over all tiles (one
// channel's local problem sizes).
cudaError_t launch_build_tmask(const TileGeom& g, const uint8_t* mask, int mask_pitch,
                               uint32_t* tmask, cudaStream_t st, unsigned long long* count = nullptr);

// *out += number of unknown in-tile pixels over all tiles (one channel).
cudaError_t launch_count_unknown(const TileGeom& g, const uint32_t* tmask, unsigned long long* out,
                                 cudaStream_t st);

// TMA descriptor of a C x H x W iterate (row pitch `pitch` elements) whose box
// is the block tile plus halo of block side b: built once per buffer.
cudaError_t make_tile_map(CUtensorMap* out, Store st, const void* base, int H, int W, int pitch, int C, int b);

// Residual norms and stop test fused into the sweep.  Each tile's FP32 sum of
// squared owned residuals of the input iterate is added exactly into a 128-bit
// fixed-point sum (unit about 2^-72 ref[c]^2, saturating at 2^32 ref[c]^2,
// values below the unit truncated): the lanes of a CTA batch their tiles' sums,
// and a CTA adds its sums into acc[2c], acc[2c + 1] (low, high word) with
// integer atomics when it leaves a channel.  Integer addition does not depend on
// the order, so the norms and every decision made from them are bitwise
// repeatable, whichever CTA takes which tile.  flag[2] counts the tiles whose
// sums are in acc; the CTA that completes the count (all C x ntiles tiles) forms
// norms2[c] and sets flag[0]:
//   1 when max_c sqrt(norms2[c]) / ref[c] <= tol (tol < 0: never),
//   2 on NaN/Inf (flag[6] set by a CTA that saw one), 3 when stall > 0 and
//   every channel's residual fell by less than the factor 1/stall since the
//   previous full sweep, 5 when a bounded wait of this or an earlier launch
//   gave up (*err != 0);
// flag[1] = the launch index (state[3]) then, and acc, flag[2], flag[6] are
// zeroed for the next sweep.  flag[0] != 0 makes later launches no-ops.
// flag[3] (the launch's completion ticket) and flag[4] (its tile counter) are
// 0 between single-frame launches.
// The iterate pair is chosen on the device: state[0] is the buffer holding the
// current iterate (the launch reads it and writes the other one), state[1]
// counts full sweeps, state[2] = 1 makes the next launch a probe that only
// evaluates the residual of the current iterate (no CG, no write-back), and
// state[3] counts the launches that ran (the stall test needs a previous
// sweep), so that a launch needs no per-launch argument and the same launch
// can repeat inside a graph loop.  After a full sweep the stop test requests a
// probe when the residual ratio of the last two sweeps predicts that the new
// iterate meets tol.  norms2 holds 2C + 2 doubles: current norms, norms of the
// previous full sweep, and the previous full sweep's worst relative residual.
constexpr int kFlagWords = 8;     // flag array length: words 0-4 and 6 per sequence, 5 the sticky error word
struct SweepStop {
    unsigned long long* acc;   // 2 x C words, zero between sweeps
    double* norms2;
    const double* ref;
    const double* tol;   // device: the tolerance (set by launch_reset_sweep_state), so a
                         // captured launch does not depend on it
    double stall;
    int* flag;
    int* state;
    int force_probe;   // 1: this launch is a probe whatever state[2] says
    // optional work counters of full sweeps: work[0] += sum over blocks of
    // (unknown block pixels) x (local CG steps taken), work[1] += unknown block
    // pixels, and work[2 + i] = 1 if launch i since the reset (i < kTimedLaunches)
    // was a full sweep (0: a probe, or not run because the stop flag was set)
    unsigned long long* work;
    // sticky error word of the handle: set to 1 when a bounded wait for a
    // staged tile gives up (reset words of a sweep sequence do not clear it);
    // the stop test then sets flag[0] = 5, which ends the sequence
    int* err;
    // test hook (0: off): the first staged-tile wait of every CTA polls an
    // mbarrier that no copy completes, stall_polls times, and then gives up as
    // a hung copy would (the DD_ETIMEOUT path, exercised without a fault)
    int stall_polls;
    // > 0: the local relative tolerance of a sweep that the stop test predicts
    // to be the last one (its input residual within 1/kFinalContraction of tol);
    // 0: every sweep uses the launch's local_rtol
    float final_local_rtol;
    // > 0: a block's local CG also stops once its residual norm is at most
    // local_atol * tol * ||b - A u0||_c / sqrt(blocks per channel) (tol > 0 only)
    float local_atol;
};
constexpr int kTimedLaunches = 64;   // launches per sequence whose kind work[2 + i] records

// Division by a divisor fixed for a launch (dividend < 2^31): the round-up
// method of Granlund & Montgomery (PLDI 1994), q = (umulhi(n, m) + n) >> s
// with s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
    uint32_t m, s;
};
FastDiv make_fastdiv(uint32_t d);

// A sweep's view of one frame (one level of one handle): the iterate pair and
// its descriptors, the block masks, the geometry, the local solver's
// parameters and the stop words.  Single-frame launches pass it by value;
// batched launches read an array of them from device memory (64-byte aligned,
// not modified while a launch runs).
struct SweepFrame {   // aligned as CUtensorMap (at least 64 bytes)
    CUtensorMap map_u[2];
    CUtensorMap map_g;
    void* u_buf[2];
    const uint32_t* tmask;
    unsigned long long* acc;
    double* norms2;
    const double* ref;
    const double* tol;
    int* flag;
    int* state;
    int* err;
    unsigned long long* work;
    int* resolve_out;          // batched levels: the level's result record (launch_batch_resolve)
    double stall;
    long long plane;
    FastDiv dv_tiles, dv_ntx;
    int H, W, pitch, C, s, ntx, ntiles, has_g;
    float p_robin, local_rtol2, local_rtol2_final, local_atol2;
    int k, stall_polls, force_probe;
    int cap;                   // batched levels: full sweeps after which the frame drops out
    double level_tol;          // batched levels: the stop tolerance launch_batch_reset sets
};

// The two iterate buffers of a level and their TMA descriptors.
struct SweepPair {
    const CUtensorMap* map[2];
    void* u[2];
};

// One ORAS sweep (or probe) over all tiles of all C channels (planes `plane`
// elements apart), from buffer state[0] of `pair` into the other buffer.
//   map_g: optional source g on unknown pixels (solves A u = C f + (I - C) g
//   with u = f held on known pixels).
//   local_rtol in [0, 1): a block's local CG also stops once its residual fell
//   by that factor (0: always k steps).
cudaError_t launch_sweep(Store st, const TileGeom& g, int C, long long plane, const SweepPair& pair,
                         const CUtensorMap* map_g, const uint32_t* tmask, const SweepStop& stop, float p_robin,
                         int k, cudaStream_t stream, float local_rtol = 0.f);

// Kernel attributes and occupancy of the sweep for (s, g, has_g), queried once
// per process; call before capturing a sweep launch into a graph.
cudaError_t prepare_sweep(Store s, const TileGeom& g, bool has_g);

// ---- batched sweeps (one persistent launch over the tiles of several frames) ----
// The descriptor of a frame for batched launches (FP32 iterate, no source
// term): as launch_sweep would use it, with the sweep limit cap of the level
// and the level's resolve record.
void fill_sweep_frame(SweepFrame* out, const TileGeom& g, int C, long long plane, const SweepPair& pair,
                      const uint32_t* tmask, const SweepStop& stop, float p_robin, int k, float local_rtol, int cap,
                      int* resolve_out);
// The list of a batched launch: list[0] = n active frames, list[1 .. n] their
// indices in the frame array, list[1 + n .. 1 + 2n] the prefix sums of their
// tiles (C x blocks each; the last entry is the launch's tile total).
// At most kBatchMaxFrames frames.
constexpr int kBatchMaxFrames = 1024;
constexpr int kBatchListWords = 2 + 2 * kBatchMaxFrames;
// One sweep (or probe) of every frame in the list, all frames with the block
// layout of g (the same block side, overlap and warps per tile).  bctl: 3
// device ints (completion ticket, tile counter, a wait gave up), zero between
// launches.  If any wait of the launch gives up, every frame of the launch gets
// its error word set and its sequence ended (flag[0] = 5).
cudaError_t launch_sweep_batch(const TileGeom& g, const SweepFrame* frames, const int* list, int* bctl,
                               cudaStream_t st);
cudaError_t prepare_sweep_batch(const TileGeom& g);
// Loop control of a batched level (one thread), at the top of each pass of its
// device loop: ctl[0] counts the passes; the list gets the frames whose
// sequences run (flag[0] == 0 and state[1] < cap); the loop's condition is
// cleared when none does or after max_passes passes (the pass then sweeps no frame).
cudaError_t launch_batch_ctl(const SweepFrame* frames, int n, int* list, int* ctl, int max_passes,
                             cudaGraphConditionalHandle cond, cudaStream_t st);
// Before a batched level: every frame's state[0] = 0, state[1..3] = 0, flag[0..4]
// and flag[6] = 0, *tol = level_tol.
cudaError_t launch_batch_reset(const SweepFrame* frames, int n, cudaStream_t st);
// After a batched level: each frame's resolve record = {state[0], state[1],
// flag[0], ctl[0]} (as launch_resolve).
cudaError_t launch_batch_resolve(const SweepFrame* frames, int n, const int* ctl, cudaStream_t st);

// state[0] = cur, state[1] = state[2] = state[3] = 0; flag[0..4] = flag[6] = 0
// (flag[5], the sticky error word of a handle's flag array, is left alone); *tol_d = tol
// (the stop tolerance the following sweeps or CG iterations read).  With
// skip_if and *skip_if != 0, flag[0] = 4 instead: the following sweeps are
// no-ops.
cudaError_t launch_reset_sweep_state(int* state, int* flag, int cur, double* tol_d, double tol, cudaStream_t st,
                                     const int* skip_if = nullptr);

// Small-grid coarse solve (coarse_cg.cu): CG on A_c e = g with e = 0 where
// mask != 0, one CTA per channel, the grid in shared memory (H*W at most
// kCoarseCgMaxPixels), FP32 vectors and FP64 dots, from e = 0 until
// ||r|| <= tol ||g|| or max_iter iterations; iters (may be null): C ints, the
// iterations taken; a no-op if skip != null and *skip != 0.  prepare_coarse_cg
// sets the kernel's shared-memory limit (once per device, before any capture).
constexpr int kCoarseCgMaxPixels = 12288;
size_t coarse_cg_smem_bytes(int H, int W);
cudaError_t prepare_coarse_cg();
cudaError_t launch_coarse_cg(int H, int W, int C, const uint8_t* mask, int mp, const float* g, int gp,
                             long long gplane, float* e, int ep, long long eplane, int max_iter, double tol,
                             int* iters, const int* skip, cudaStream_t st);

// Two-level coarse correction (DD_ML_CORRECTION), each a no-op if *skip != 0
// (skip may be null):
// dst (ceil(H/2) x ceil(W/2)) = sum of src over each 2x2 block inside the image.
cudaError_t launch_restrict_sum(int H, int W, int C, const float* src, int sp, long long splane, float* dst, int dp,
                                long long dplane, const int* skip, cudaStream_t st);
// Safeguard of the correction: gate[0] = 1 (this pass's correction is skipped)
// if flag[0] != 0 or corrections are off (gate[1]); corrections are switched
// off for the rest of the solve once the fine residual norms2[2C] fell by less
// than a factor 0.7 since the previous pass (prev[0]).  gate and prev are reset
// (to 0) before a solve's fine loop.
// The coarse-grid correction's gate (gate[0] = skip, read by the correction kernels).
cudaError_t launch_corr_gate(const int* flag, const double* norms2, int C, const int* state, int* gate, double* prev,
                             double trigger, const double* tol, cudaStream_t st);
// Loop control of the plain phase of a fine level with a correction trigger: it
// also ends the loop when the trigger fires.
cudaError_t launch_loop_ctl_trigger(const int* flag, const int* state, int* ctl, int cap, int max_passes,
                                    cudaGraphConditionalHandle cond, const double* norms2, int C, int* gate,
                                    double* prev, double trigger, const double* tol, cudaStream_t st);
// Entry kernel of the corrected phase's loop: (ctl, flag, state, gate, cap, max_passes, cond).
const void* loop_begin_corrected_kernel_fn();

// Energy-optimal step of the correction (omega = (r, d) / (d, A d) per channel):
// corr_dir: d = bilinear prolongation of the coarse correction on mask == 0
//   pixels (0 elsewhere), written over r (pitch rp); out[c] = (r, d);
// corr_curv: out[c] = (d, A d) with A the reduced operator; omega[c] =
//   num[c] / out[c] (0 if not positive);
// corr_step: (sel_u[0] ? u1 : u0) += omega[c] d.
// part (C x nblk doubles, nblk = res64_blocks(H, W)) and ticket (zero, left
// zero) are reduction scratch.
cudaError_t launch_corr_dir(int Hc, int Wc, int H, int W, int C, const float* ec0, const float* ec1, const int* sel_c,
                            int ecp, long long ecplane, const uint8_t* mask, int mp, float* rd, int rp,
                            long long rplane, const int* skip, double* part, int nblk, unsigned int* ticket,
                            double* out, cudaStream_t st);
cudaError_t launch_corr_curv(int H, int W, int C, const float* d, int dp, long long dplane, const int* skip,
                             double* part, int nblk, unsigned int* ticket, double* out, const double* num,
                             double* omega, cudaStream_t st);
cudaError_t launch_corr_step(int H, int W, int C, const float* d, int dp, long long dplane, const double* omega,
                             float* u0, float* u1, const int* sel_u, int up, long long uplane, const int* skip,
                             cudaStream_t st);
// Loop control at the end of each pass of a graph WHILE loop (one thread):
// ctl[0] counts the passes; the loop's condition is cleared when flag[0] != 0
// (stopped, converged or failed), when state[1] (full sweeps or CG iterations
// applied) reaches cap, or after max_passes passes, which bounds the loop
// whatever the solver kernels do.
cudaError_t launch_loop_ctl(const int* flag, const int* state, int* ctl, int cap, int max_passes,
                            cudaGraphConditionalHandle cond, cudaStream_t st);
// Kernel (one block of 32 threads, arguments (int* ctl, cudaGraphConditionalHandle
// cond)) that zeroes ctl[0..3] and sets cond to 1: the first node of a device
// loop, so that a loop nested in another loop's body is re-armed on every entry.
const void* loop_begin_kernel_fn();

// ---- auxiliary passes (aux.cu) ----------------------------------------------------
// dst[c][y][x] (pitch dp) = mask ? src[c][y][x] : 0  (src pitch sp); with
// count, *count += the number of known pixels
cudaError_t launch_masked_copy(int H, int W, int C, const float* src, int sp, long long splane,
                               const uint8_t* mask, int mp, float* dst, int dp, long long dplane,
                               cudaStream_t st, unsigned long long* count = nullptr);
// plain strided copy (float)
cudaError_t launch_copy2d(int H, int W, int C, const float* src, int sp, long long splane,
                          float* dst, int dp, long long dplane, cudaStream_t st);
// zero n elements of storage type s
cudaError_t launch_fill_zero(Store s, void* dst, size_t n, cudaStream_t st);
// dst = keep known: u[c][y][x] = mask ? f : u   (float, pitched)
cudaError_t launch_reset_known(int H, int W, int C, float* u, int up, long long uplane,
                               const uint8_t* mask, int mp, const float* f, int fp, long long fplane,
                               cudaStream_t st);

// Residual r = b - A u of an FP32 iterate on unknown pixels (0 on known),
// formed with error-free FP32 transformations (~48-bit significand).  The
// pass's blocks (about one wave, at most nblk per channel) walk the tiles
// grid-stride and write per channel their sums {r^2, max |r|} to
// part[c*nblk + blk] (double2).
// If g_out != nullptr, also writes g_out = r * scale_inv[c] in storage `gst`.
struct Res64Args {
    int H, W, C;
    const float* u; int up; long long uplane;
    const uint8_t* mask; int mp;
    void* g_out; Store gst; int gp; long long gplane;
    const double* scale_inv;   // device, per channel (only with g_out)
    double2* part; int nblk;   // partial stride per channel, at least res64_blocks(H, W)
    // optional, fused: the last block writes out[c] = {sum r^2, max |r|} (and
    // sqrt_out[c] = sqrt(sum) if given); ticket: a zero device counter, left zero
    double2* out; double* sqrt_out; unsigned int* ticket;
    // optional: the iterate is (sel[0] ? u1 : u), chosen on the device (u1 has
    // u's pitch and plane), and is also copied to copy_out (pitch cp, plane cplane)
    const float* u1; const int* sel;
    float* copy_out; int cp; long long cplane;
    const int* skip;   // optional: the pass is a no-op if *skip != 0
};
int res64_blocks(int H, int W);
cudaError_t launch_res64(const Res64Args& a, cudaStream_t st);

// Reference norms ||b - A u0||, u0 = C f, of all levels of a handle in one
// launch (the residual of u0 on an unknown pixel is the sum of its known
// neighbours' values).  Per level: f (C planes of H x fp, 16-byte aligned
// rows), mask (H x mp bytes), and the outputs out[c] = {sum r^2, 0} and
// sqrt_out[c].  part: part_capacity doubles of block partials (at least
// C * ref_norm_part_words(H, W, nl) for the level sizes halving from H x W);
// ticket: a zero device counter, left zero.  The launcher fills each level's
// tile grid (gx, gy) and mask access mode.
constexpr int kRefMaxLevels = 8;
struct RefLevel {
    const float* f; int fp; long long fplane;
    const uint8_t* mask; int mp;
    int H, W;
    double2* out; double* sqrt_out;
    int gx, gy, mvec;   // set by launch_ref_norms
};
struct RefNormArgs {
    RefLevel lv[kRefMaxLevels];
    int nl, C;
    double* part; int part_capacity;
    unsigned int* ticket;
};
int ref_norm_part_words(int H, int W, int nl);
cudaError_t launch_ref_norms(RefNormArgs a, cudaStream_t st);


// Dyadic restriction (Sec. 4): mask OR over 2x2, mean of known values.
cudaError_t launch_restrict(int H, int W, int C, const uint8_t* mask, int mp, const float* f, int fp,
                            long long fplane, uint8_t* mask_c, int mcp, float* f_c, int fcp,
                            long long fcplane, cudaStream_t st);
// Cell-centred bilinear prolongation, optional reset of known pixels to f.
cudaError_t launch_prolong(int Hc, int Wc, int H, int W, int C, const float* uc, int ucp,
                           long long ucplane, const uint8_t* mask, int mp, const float* f, int fp,
                           long long fplane, float* u, int up, long long uplane, cudaStream_t st);
// u = fl32(u + s_c * e) on unknown pixels (error-free FP32 transformations: the
// FP64 result up to rare near-ties), e in storage `est`.
cudaError_t launch_correct(int H, int W, int C, float* u, int up, long long uplane, const void* e,
                           Store est, int ep, long long eplane, const uint8_t* mask, int mp,
                           const double* scale, cudaStream_t st, const void* e1 = nullptr,
                           const int* sel = nullptr, const int* skip = nullptr);
// The outer control of the device-driven FP64 correction loop (one thread, see
// aux.cu): ctl[8] ints; clears cond when the loop ends (also once *err != 0).
cudaError_t launch_ref_outer_ctl(const double2* res_out, const double* ref, int C, const double* tol, int max_corr,
                                 int max_sweeps, const int* inner_state, const int* inner_ctl, const int* err,
                                 int* ctl, double* scale, double* scale_inv, double* inner_ref,
                                 cudaGraphConditionalHandle cond, cudaStream_t st);
// Summary of a sweep sequence for later steps: out[0] = buffer holding the
// result, out[1] = full sweeps applied, out[2] = the stop flag (0: not
// stopped, 1: converged, 2: NaN/Inf, 3: stalled), out[3] = passes of the
// device loop (ctl[0]; 0 without ctl).
cudaError_t launch_resolve(const int* flag, const int* sweep_state, const int* ctl, int* out, cudaStream_t st);
// Prolongation / copy reading the source buffer uc0 or uc1 chosen by *sel on the device.
cudaError_t launch_prolong_sel(int Hc, int Wc, int H, int W, int C, const float* uc0, const float* uc1,
                               const int* sel, int ucp, long long ucplane, const uint8_t* mask, int mp,
                               const float* f, int fp, long long fplane, float* u, int up, long long uplane,
                               cudaStream_t st);
// *out += number of nonzero bytes of m[0..n)
cudaError_t launch_count_nonzero(const uint8_t* m, long long n, unsigned long long* out, cudaStream_t st);
// ---- conjugate gradients on the whole image (cg.cu) ---------------------------------
struct CGArgs {
    int H, W, P, C, mp;
    long long plane;
    const uint8_t* mask;
    float* x;            // iterate (known pixels hold f)
    float* r;            // residual on unknown pixels
    float* p[2];         // search directions: iteration i reads p[i & 1] (the previous
                         // one; zero before the first) and writes p[(i + 1) & 1]
    float* q;            // A p
    double* part;        // C x cg_blocks partial sums
    double* scal;        // [0,C) (r,r), [C,2C) alpha, [2C,3C) beta
    const double* ref;   // per-channel ||b - A u0||
    int* flag;           // [0] stop flag, [1] stopping iteration, [3] ticket
    int* state;          // [1] = i, the iterations applied since the reset (read on
                         // the device, so one iteration's launches can repeat in a graph loop)
    const double* tol;   // device: the stop tolerance (set by launch_reset_sweep_state)
};
int cg_blocks(int H, int W);
// scal <- {(r, r) from res_out[c].x, alpha = beta = 0}
cudaError_t launch_cg_init(const double2* res_out, double* scal, int C, cudaStream_t st);
// one CG iteration (two kernels) under the device stop flag
cudaError_t launch_cg_iteration(const CGArgs& a, cudaStream_t st);

// Default Robin weight for block side b and overlap o (the value create uses).
float default_robin(int b, int o);
// Record the text returned by dd_last_error() on this thread.
void set_last_error(const char* msg);

}  // namespace dd
