// Host driver and C ABI of the ORAS inpainting solver (include/dd_inpaint.h).
//
// Paper mapping (Kaemper & Weickert, arXiv 2110.03946):
//   Sec. 2      problem A u = b, A = C - (I - C) L, b = C f, per channel;
//   Sec. 3      ORAS sweeps (sweep.cu);
//   Sec. 4      32-px blocks with 6-px overlap, local CG, iterate until the
//               relative residual has decayed to tol, and the coarse-to-fine
//               multilevel initialisation over dyadic levels (aux.cu).
// Beyond the paper: an outer residual correction whose residual is formed in
// FP64 (DD_PREC_*_REF) around inner ORAS solves whose iterate is stored in
// FP32, FP16 or BF16.
//
// All iteration state stays on the device.  The stop test is evaluated on the
// device after every sweep (reduce kernel + flag); later sweeps of a chunk see
// the flag and return at once, and the host reads the flag once per chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dd_inpaint.h"
#include "dd_internal.h"

using dd::Store;
using dd::TileGeom;

namespace {

thread_local std::string g_last_error;

void set_error(const std::string& s) { g_last_error = s; }

#define DD_CK(call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
            return e_ == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA;               \
        }                                                                                \
    } while (0)

// A kernel launch through the handle: checked and counted.
// A launch wrapper reports (and clears) an error left pending by an earlier
// unchecked runtime call before the launch, so the error names its real origin
// rather than the next kernel.
#define DD_LAUNCH(h, call)                                                                      \
    do {                                                                                        \
        const cudaError_t pend_ = cudaPeekAtLastError();                                        \
        if (pend_ != cudaSuccess) {                                                             \
            (void)cudaGetLastError();                                                           \
            set_error(std::string("CUDA error pending before ") + #call + ": " +                 \
                      cudaGetErrorString(pend_));                                               \
            return DD_ECUDA;                                                                    \
        }                                                                                       \
        DD_CK(call);                                                                            \
        ++(h)->launches;                                                                        \
    } while (0)

#define DD_TRY(expr)                \
    do {                            \
        int rc_ = (expr);           \
        if (rc_ != DD_OK) return rc_; \
    } while (0)

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// A level's iteration as a CUDA graph: a memset resets the pass counter, then a
// WHILE node repeats one pass (one ORAS sweep or probe, or one CG iteration,
// followed by the loop-control kernel) until the stop test, the sweep limit
// `cap` or the pass bound clears its condition.  The tolerance is read from
// device memory, so the graph depends on cap only.
struct LoopGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int cap = 0;
};

void destroy_loop(LoopGraph& G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = LoopGraph{};
}

struct Level {
    int H = 0, W = 0, P = 0;
    bool solved = true;        // false: a dyadic level between solved ones (coarse_factor 4 or 8), which
                               // only carries the restriction and the prolongation
    TileGeom geom;
    uint8_t* mask = nullptr;   // H x W dense
    float* f = nullptr;        // C x H x P, known values, 0 elsewhere
    uint32_t* tmask = nullptr;
    float* u[2] = {nullptr, nullptr};
    CUtensorMap map_u[2];      // TMA descriptors of u[0], u[1]
    unsigned long long* partial = nullptr;  // 2 x C words: exact 128-bit sums of a sweep's residual norms (zero
                                            // between sweeps)
    double* ref_d = nullptr;   // C
    std::vector<double> ref;   // C (host copy, read after load_data's single sync)
    int* state_d = nullptr;    // resolve() output of this level's last sweep sequence
    // conjugate-gradient solver (DD_SOLVER_CG): residual, two search directions, A p
    float* cg_r = nullptr;
    float* cg_p[2] = {nullptr, nullptr};
    float* cg_q = nullptr;
    double* cg_part = nullptr;   // C x cg_blocks
    double* cg_scal = nullptr;   // 3C
    LoopGraph loop;              // device loop of this level's iteration (params.device_loop)
    // DD_ML_CORRECTION (levels >= 1): restricted residual / prolonged correction
    // scratch; on the coarsest level also the source of the correction solve
    float* corr_g = nullptr;     // C x H x P
    CUtensorMap map_cg;          // TMA descriptor of corr_g (coarsest level)
    bool loop_pending = false;   // a loop ran since the launch count was last updated
    long long plane() const { return (long long)H * P; }
};

}  // namespace

struct dd_inpaint {
    int H = 0, W = 0, C = 0;
    dd_params prm{};
    Store lowst = Store::F32;
    std::vector<Level> lv;
    int nc = 0;               // levels of the cascade (lv[0 .. nc)); lv[nc ..) are correction-only levels
                              // below the cascade's coarsest, for the small-grid coarse solve
    int cur = 0;              // buffer of lv[0] holding the fine iterate
    bool warm = false;        // next solve starts from the kept iterate
    bool valid = false;       // mask/values loaded and not empty
    // correction equation buffers (fine level): e ping-pong and source g
    void* e[2] = {nullptr, nullptr};
    void* g = nullptr;
    CUtensorMap map_e[2], map_g;
    double* inner_ref_d = nullptr;  // C
    double* ones_d = nullptr;       // C ones (residual pass without scaling)
    double* scale_d = nullptr;      // C
    double* scale_inv_d = nullptr;  // C
    // residual / stop-test scratch
    double2* res_part = nullptr;
    int res_part_n = 0;             // res_part holds C x res_part_n double2
    int res_nblk = 0;
    double2* res_out = nullptr;     // C per level
    unsigned int* res_ticket = nullptr;   // completion ticket of the fused residual reduction (zero)
    double* norms2_d = nullptr;     // C
    int* flag_d = nullptr;          // [0] stop flag, [1] conv_at, [3] ticket, [4] tile counter, [5] sticky
                                    // error word of every sweep sequence of the handle (kFlagWords ints)
    int* sstate_d = nullptr;        // sweep state: current buffer, full sweeps, probe request, launches
    int* ctl_d = nullptr;           // device-loop pass counter (4 ints)
    double* tol_d = nullptr;        // stop tolerance of the running level (set by each reset)
    unsigned long long* work_d = nullptr;   // timed fine sweeps: [0] pixel x CG steps, [1] pixels,
                                            // [2 + i] launch i was a full sweep (kWorkWords words)
    unsigned long long* h_work = nullptr;   // pinned mirror
    // DD_ML_CORRECTION: fine residual, and the stop state of the coarse correction solve
    float* corr_r = nullptr;        // C x H x P (level 0)
    int* flag_c = nullptr;          // kFlagWords ints
    int* state_c = nullptr;         // 4 ints
    double* norms2_c = nullptr;     // 2C + 2
    double* tol_c = nullptr;        // 1
    double* corr_dots = nullptr;    // 3C: (r, d), (d, A d), omega
    int* corr_gate = nullptr;       // kGateWords: [0] skip this pass's correction, [1] corrections off,
                                    // [2] corrections applied, [3]-[5] history, [6] gate launches
                                    // (corr_gate_kernel)
    double* corr_prev = nullptr;    // [0] the fine residual at the previous full pass, [1] the contraction of
                                    // the pass that fired the trigger
    cudaStream_t cap_stream = nullptr;   // private stream on which loop bodies are captured
    cudaStream_t cap_stream2 = nullptr;  // ... and the bodies of loops nested in them
    // device-driven FP64 correction loop (precision != FP32, device_loop = 1)
    int* ref_ctl_d = nullptr;       // 4 + kFlagWords ints, see ref_outer_ctl_kernel
    double* ref_tol_d = nullptr;    // the solve's tolerance
    int* h_ref_ctl = nullptr;       // pinned mirror (8 ints)
    LoopGraph ref_loop;             // the outer loop as a graph of its own
    // pinned host mirrors
    double2* h_res = nullptr;
    double* h_small = nullptr;      // 3*C doubles scratch
    int* h_flag = nullptr;          // [0..2] flag words, [3] error word, [4..5] sweep state, [6] coarse
                                    // corrections applied, [7] correction gate launches
    int* h_state = nullptr;         // 4 ints per level
    double* h_ref = nullptr;        // C: fine-level reference norms read back with a solve
    unsigned long long* h_cnt = nullptr;   // [0] unknown block pixels, [1] known pixels
    // asynchronous solve in flight (dd_inpaint_solve_async / _finish)
    bool pending = false;
    bool pending_cascaded = false;
    bool counts_pending = false;    // set_data_async: pixel counts not read yet
    bool ev_recorded = false;       // ev0/ev1 bracket the pending solve
    float* pending_out = nullptr;
    double pending_tol = 0.0;
    std::vector<void*> allocs;
    size_t bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    static constexpr int kChunk = 8;                 // sweeps per stop-test read-back
    static constexpr int kFirst = 16;                // fine sweeps enqueued before the first read-back
    cudaEvent_t sw_ev[2 * kFirst] = {};              // per-sweep timing events (params.timing)
    unsigned long long* count_d = nullptr;           // [0] unknown block pixels, [1] known pixels
    long long launches = 0;                          // kernels launched through this handle
    long long local_unknowns = 0;
    dd_stats stats{};
};

namespace {

// Device bytes held by all live handles, and the caller's cap on them (0: none).
std::atomic<unsigned long long> g_bytes_in_use{0};
std::atomic<unsigned long long> g_budget{0};

int dalloc(dd_inpaint* h, void** p, size_t n) {
    if (n == 0) n = 16;
    const unsigned long long cap = g_budget.load();
    const unsigned long long held = g_bytes_in_use.fetch_add(n) + n;
    if (cap != 0 && held > cap) {
        g_bytes_in_use.fetch_sub(n);
        *p = nullptr;
        set_error("the device budget set by dd_set_device_budget would be exceeded");
        return DD_ENOMEM;
    }
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) {
        g_bytes_in_use.fetch_sub(n);
        (void)cudaGetLastError();
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return DD_ENOMEM;
    }
    h->allocs.push_back(*p);
    h->bytes += n;
    return DD_OK;
}

template <typename T>
int dalloc_t(dd_inpaint* h, T** p, size_t count) {
    void* v = nullptr;
    int rc = dalloc(h, &v, count * sizeof(T));
    *p = static_cast<T*>(v);
    return rc;
}

int dzero(void* p, size_t n) {
    if (cudaMemset(p, 0, n) != cudaSuccess) {
        set_error("cudaMemset failed");
        return DD_ECUDA;
    }
    return DD_OK;
}

// Stop-flag words of a sweep sequence, zeroed (the tile counter must start at 0).
int alloc_flag(dd_inpaint* h, int** f) {
    int rc = dalloc_t(h, f, dd::kFlagWords);
    return rc != DD_OK ? rc : dzero(*f, dd::kFlagWords * sizeof(int));
}

// Words of the work counters of timed sweeps: two sums and one kind per launch.
constexpr int kWorkWords = 2 + dd::kTimedLaunches;

// Words of the coarse-grid correction's gate (corr_gate_kernel).
constexpr int kGateWords = 8;

// The sticky error word shared by all sweep sequences of a handle.
int* err_word(dd_inpaint* h) { return h->flag_d + 5; }

// A sweep sequence's stop words on the handle's flag array, with the handle's
// error word and test hook.
dd::SweepStop make_stop(dd_inpaint* h, unsigned long long* partial, const double* ref_d, double stall,
                        unsigned long long* work = nullptr) {
    return dd::SweepStop{partial, h->norms2_d, ref_d, h->tol_d, stall, h->flag_d, h->sstate_d, 0,
                         work, err_word(h), h->prm.test_stall_polls, (float)h->prm.final_local_rtol,
                         (float)h->prm.local_atol};
}

// Clear the error word at the start of a solve (enqueued, so it also works in a capture).
int clear_error(dd_inpaint* h, cudaStream_t st) {
    DD_CK(cudaMemsetAsync(err_word(h), 0, sizeof(int), st));
    return DD_OK;
}

Store low_store(int precision) {
    switch (precision) {
        case DD_PREC_FP16_REF: return Store::F16;
        case DD_PREC_BF16_REF: return Store::BF16;
        default: return Store::F32;
    }
}

int validate(int H, int W, int C, const dd_params& p) {
    if (H <= 0 || W <= 0 || C <= 0) { set_error("H, W and C must be positive"); return DD_EINVAL; }
    if ((long long)H * W > (1LL << 31) / 4) { set_error("image too large"); return DD_EINVAL; }
    if (!dd::block_supported(p.block)) { set_error("block must be 16, 32, 64 or 96"); return DD_EINVAL; }
    if (p.solver != DD_SOLVER_ORAS && p.solver != DD_SOLVER_CG) { set_error("bad solver"); return DD_EINVAL; }
    if (p.solver == DD_SOLVER_CG && p.precision != DD_PREC_FP32) {
        set_error("DD_SOLVER_CG needs precision DD_PREC_FP32");
        return DD_EINVAL;
    }
    if (p.tile_warps != 0 && !dd::tile_warps_supported(p.block, p.tile_warps)) {
        set_error("tile_warps: 16 -> 1; 32 -> 1, 2 or 4; 64 -> 4 or 8; 96 -> 12");
        return DD_EINVAL;
    }
    if (p.overlap < 0 || p.overlap >= p.block) { set_error("need 0 <= overlap < block"); return DD_EINVAL; }
    if (p.device_loop != 0 && p.device_loop != 1) { set_error("device_loop must be 0 or 1"); return DD_EINVAL; }
    if (p.local_cg_iters < 1 || p.local_cg_iters > 4096) { set_error("local_cg_iters out of range"); return DD_EINVAL; }
    if (p.levels < 1 || p.levels > DD_MAX_LEVELS) { set_error("levels must be 1..8"); return DD_EINVAL; }
    if (p.ml_mode != DD_ML_CASCADE && p.ml_mode != DD_ML_CORRECTION) { set_error("bad ml_mode"); return DD_EINVAL; }
    if (p.ml_mode == DD_ML_CORRECTION &&
        (p.precision != DD_PREC_FP32 || p.solver != DD_SOLVER_ORAS || p.levels < 2 || p.correction_sweeps < 1)) {
        set_error("DD_ML_CORRECTION needs DD_PREC_FP32, DD_SOLVER_ORAS, levels >= 2 and correction_sweeps >= 1");
        return DD_EINVAL;
    }
    if (p.precision < DD_PREC_FP32 || p.precision > DD_PREC_BF16_REF) { set_error("bad precision"); return DD_EINVAL; }
    if (p.coarse_factor != 0 && p.coarse_factor != 2 && p.coarse_factor != 4 && p.coarse_factor != 8) {
        set_error("coarse_factor must be 2, 4 or 8");
        return DD_EINVAL;
    }
    if (p.test_stall_polls < 0) { set_error("test_stall_polls must be >= 0"); return DD_EINVAL; }
    if (p.max_sweeps < 0 || p.coarse_sweeps < 0 || p.max_corrections < 0) {
        set_error("negative limit");
        return DD_EINVAL;
    }
    if (!(p.coarse_tol > 0.0) || !(p.inner_tol > 0.0) || !(p.inner_tol < 1.0)) {
        set_error("bad tolerance");
        return DD_EINVAL;
    }
    if (!(p.local_rtol >= 0.0) || !(p.local_rtol < 1.0)) {
        set_error("local_rtol must be in [0, 1)");
        return DD_EINVAL;
    }
    if (!(p.correction_trigger >= 0.0) || !(p.correction_trigger < 1.0)) {
        set_error("correction_trigger must be in [0, 1)");
        return DD_EINVAL;
    }
    if (!(p.final_local_rtol >= 0.0) || !(p.final_local_rtol < 1.0)) {
        set_error("final_local_rtol must be in [0, 1)");
        return DD_EINVAL;
    }
    if (!(p.local_atol >= 0.0) || !(p.local_atol < 1.0)) {   // >= 1 could stall above tol
        set_error("local_atol must be in [0, 1)");
        return DD_EINVAL;
    }
    if (p.correction_cg < 0 || p.correction_cg > 100000) {
        set_error("correction_cg must be in [0, 100000]");
        return DD_EINVAL;
    }
    return DD_OK;
}

float robin_default(int b, int o) {
    // Optimised Robin parameter of overlapping Schwarz (Gander, SIAM J. Numer.
    // Anal. 44 (2006)): p = 2^(-1/3) k_min^(2/3) L^(-1/3), k_min = pi/b, L = o,
    // scaled by 3 for the inpainting operator, whose many interior Dirichlet
    // pixels damp the low frequencies the estimate is made for.
    const double kmin = 3.14159265358979323846 / b;
    const double L = std::max(o, 1);
    return (float)(3.0 * std::pow(2.0, -1.0 / 3.0) * std::pow(kmin, 2.0 / 3.0) * std::pow(L, -1.0 / 3.0));
}

// Copy caller data (mask, values) into level 0 and rebuild all levels.  All
// work is enqueued on st; the only host synchronisation reads back the pixel
// counts and reference norms once at the end.  Returns DD_EEMPTYMASK if no
// pixel is known.
int load_data(dd_inpaint* h, const uint8_t* mask, const float* values, cudaStream_t st, bool sync = true) {
    Level& L0 = h->lv[0];
    const size_t npx = (size_t)h->H * h->W;
    const float* dvals = values;
    if (!h->prm.inputs_on_device) {
        DD_CK(cudaMemcpyAsync(L0.mask, mask, npx, cudaMemcpyHostToDevice, st));
        // values staged through u[1] as a dense C x H x W array (it has room: P >= W)
        DD_CK(cudaMemcpyAsync(L0.u[1], values, npx * h->C * sizeof(float), cudaMemcpyHostToDevice, st));
        dvals = L0.u[1];
    } else {
        DD_CK(cudaMemcpyAsync(L0.mask, mask, npx, cudaMemcpyDeviceToDevice, st));
    }
    // the pixel counts (unknown block pixels of level 0, known pixels) come with the passes
    DD_CK(cudaMemsetAsync(h->count_d, 0, 2 * sizeof(unsigned long long), st));
    DD_LAUNCH(h, dd::launch_masked_copy(h->H, h->W, h->C, dvals, h->W, (long long)npx, L0.mask, h->W, L0.f, L0.P,
                                        L0.plane(), st, h->count_d + 1));
    for (size_t l = 1; l < h->lv.size(); ++l) {
        Level& F = h->lv[l - 1];
        Level& Cc = h->lv[l];
        DD_LAUNCH(h, dd::launch_restrict(F.H, F.W, h->C, F.mask, F.W, F.f, F.P, F.plane(), Cc.mask, Cc.W, Cc.f,
                                         Cc.P, Cc.plane(), st));
    }
    for (auto& L : h->lv)
        DD_LAUNCH(h, dd::launch_build_tmask(L.geom, L.mask, L.W, L.tmask, st, &L == &L0 ? h->count_d : nullptr));
    // reference norms ||b - A u0||, u0 = C f, of every level and channel in one launch, kept on the device
    const int nl = (int)h->lv.size();
    {
        dd::RefNormArgs ra{};
        ra.nl = nl;
        ra.C = h->C;
        for (int l = 0; l < nl; ++l) {
            Level& L = h->lv[l];
            dd::RefLevel& R = ra.lv[l];
            R.f = L.f; R.fp = L.P; R.fplane = L.plane();
            R.mask = L.mask; R.mp = L.W;
            R.H = L.H; R.W = L.W;
            R.out = h->res_out + (size_t)l * h->C;
            R.sqrt_out = L.ref_d;
        }
        ra.part = reinterpret_cast<double*>(h->res_part);
        ra.part_capacity = 2 * h->C * h->res_part_n;
        ra.ticket = h->res_ticket;
        DD_LAUNCH(h, dd::launch_ref_norms(ra, st));
    }
    DD_CK(cudaMemcpyAsync(h->h_cnt, h->count_d, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    if (!sync) {   // counts and reference norms are read back with the next solve
        h->counts_pending = true;
        return DD_OK;
    }
    h->counts_pending = false;
    DD_CK(cudaMemcpyAsync(h->h_res, h->res_out, sizeof(double2) * h->C * nl, cudaMemcpyDeviceToHost, st));
    DD_CK(cudaStreamSynchronize(st));
    const unsigned long long cnt[2] = {h->h_cnt[0], h->h_cnt[1]};
    h->local_unknowns = (long long)cnt[0];
    for (int l = 0; l < nl; ++l) {
        Level& L = h->lv[l];
        L.ref.resize(h->C);
        for (int c = 0; c < h->C; ++c) L.ref[c] = std::sqrt(h->h_res[(size_t)l * h->C + c].x);
    }
    if (cnt[1] == 0) { set_error("empty mask"); return DD_EEMPTYMASK; }
    return DD_OK;
}

int count_known(const uint8_t* mask, size_t n, bool on_device, long long* out) {
    std::vector<uint8_t> tmp;
    const uint8_t* m = mask;
    if (on_device) {
        tmp.resize(n);
        DD_CK(cudaMemcpy(tmp.data(), mask, n, cudaMemcpyDeviceToHost));
        m = tmp.data();
    }
    long long k = 0;
    for (size_t i = 0; i < n; ++i) k += m[i] != 0;
    *out = k;
    return DD_OK;
}

// ORAS sweeps on one level until the (lagged) relative residual of the
// current iterate, measured against ref_d, is <= tol, or max_sweeps sweeps.
// bufs[cur] holds the input; on return cur indexes the result.
int run_sweeps(dd_inpaint* h, const TileGeom& g, Store st_t, void* const bufs[2], const CUtensorMap* maps,
               int& cur, const CUtensorMap* map_g, const uint32_t* tmask, unsigned long long* partial,
               const double* ref_d, double tol, double stall, int max_sweeps, cudaStream_t st, int* applied,
               bool* converged, bool fine = false) {
    const long long plane = (long long)g.H * g.pitch;
    DD_LAUNCH(h, dd::launch_reset_sweep_state(h->sstate_d, h->flag_d, cur, h->tol_d, tol, st));
    *converged = false;
    *applied = 0;
    const bool timed = fine && h->prm.timing != 0;
    const dd::SweepPair pair{{&maps[0], &maps[1]}, {bufs[0], bufs[1]}};
    dd::SweepStop stop = make_stop(h, partial, ref_d, stall, timed ? h->work_d : nullptr);
    if (timed) DD_CK(cudaMemsetAsync(h->work_d + 2, 0, sizeof(unsigned long long) * dd::kTimedLaunches, st));
    int full_done = 0, launched = 0;
    while (true) {
        // full sweeps until max_sweeps; then one probe evaluates the last iterate
        const bool last_probe = full_done >= max_sweeps;
        const int n = last_probe ? 1 : std::min(dd_inpaint::kChunk, max_sweeps - full_done);
        for (int i = 0; i < n; ++i) {
            stop.force_probe = last_probe ? 1 : 0;
            if (timed && !last_probe) DD_CK(cudaEventRecord(h->sw_ev[2 * i], st));
            DD_LAUNCH(h, dd::launch_sweep(st_t, g, h->C, plane, pair, map_g, tmask, stop, h->prm.robin_p,
                                          h->prm.local_cg_iters, st, (float)h->prm.local_rtol));
            if (timed && !last_probe) DD_CK(cudaEventRecord(h->sw_ev[2 * i + 1], st));
        }
        DD_CK(cudaMemcpyAsync(h->h_flag, h->flag_d, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
        DD_CK(cudaMemcpyAsync(h->h_flag + 3, err_word(h), sizeof(int), cudaMemcpyDeviceToHost, st));
        DD_CK(cudaMemcpyAsync(h->h_flag + 4, h->sstate_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        if (timed)
            DD_CK(cudaMemcpyAsync(h->h_work, h->work_d, sizeof(unsigned long long) * kWorkWords,
                                  cudaMemcpyDeviceToHost, st));
        DD_CK(cudaStreamSynchronize(st));
        if (h->h_flag[3] != 0) {
            set_error("a bounded device wait for a staged tile gave up");
            return DD_ETIMEOUT;
        }
        const int new_full = h->h_flag[5];
        if (timed && !last_probe) {
            // the launches of this chunk that ran as full sweeps (not probes)
            for (int i = 0; i < n && launched + i < dd::kTimedLaunches; ++i) {
                if (h->h_work[2 + launched + i] == 0) continue;
                float ms = 0.f;
                DD_CK(cudaEventElapsedTime(&ms, h->sw_ev[2 * i], h->sw_ev[2 * i + 1]));
                h->stats.fine_sweep_ms += ms;
                h->stats.fine_sweep_launches += 1;
            }
        }
        launched += n;
        full_done = new_full;
        cur = h->h_flag[4];
        *applied = full_done;
        if (h->h_flag[0] == 2) {
            set_error("non-finite residual norm");
            return DD_ENUMERIC;
        }
        if (h->h_flag[0] == 1 || h->h_flag[0] == 3) {
            *converged = h->h_flag[0] == 1;
            return DD_OK;
        }
        if (last_probe) return DD_OK;
    }
}

// FP64 residual of the fine FP32 iterate: per-channel relative residuals;
// optionally writes the scaled residual into h->g (storage lowst).
int fine_residual64(dd_inpaint* h, cudaStream_t st, std::vector<double>& rel, std::vector<double>& rmax,
                    std::vector<double>& rnorm) {
    Level& L = h->lv[0];
    dd::Res64Args a{};
    a.H = L.H; a.W = L.W; a.C = h->C;
    a.u = L.u[h->cur]; a.up = L.P; a.uplane = L.plane();
    a.mask = L.mask; a.mp = L.W;
    a.g_out = nullptr; a.gst = h->lowst;
    a.part = h->res_part; a.nblk = h->res_nblk;
    a.out = h->res_out; a.ticket = h->res_ticket;
    DD_LAUNCH(h, dd::launch_res64(a, st));
    DD_CK(cudaMemcpyAsync(h->h_res, h->res_out, sizeof(double2) * h->C, cudaMemcpyDeviceToHost, st));
    DD_CK(cudaStreamSynchronize(st));
    rel.assign(h->C, 0.0);
    rmax.assign(h->C, 0.0);
    rnorm.assign(h->C, 0.0);
    for (int c = 0; c < h->C; ++c) {
        rnorm[c] = std::sqrt(h->h_res[c].x);
        rmax[c] = h->h_res[c].y;
        const double den = L.ref[c] > 0.0 ? L.ref[c] : 1.0;
        rel[c] = rnorm[c] / den;
        if (!std::isfinite(rel[c])) { set_error("non-finite residual"); return DD_ENUMERIC; }
    }
    return DD_OK;
}

int write_scaled_residual(dd_inpaint* h, cudaStream_t st) {
    Level& L = h->lv[0];
    dd::Res64Args a{};
    a.H = L.H; a.W = L.W; a.C = h->C;
    a.u = L.u[h->cur]; a.up = L.P; a.uplane = L.plane();
    a.mask = L.mask; a.mp = L.W;
    a.g_out = h->g; a.gst = h->lowst; a.gp = L.P; a.gplane = L.plane();
    a.scale_inv = h->scale_inv_d;
    a.part = h->res_part; a.nblk = h->res_nblk;
    DD_LAUNCH(h, dd::launch_res64(a, st));
    return DD_OK;
}

// Whether a level's iteration runs as a device loop (a graph WHILE node) rather
// than as plain launches: per-sweep event timing needs the launches.
bool loop_mode(const dd_inpaint* h, bool timed) { return h->prm.device_loop != 0 && !timed; }

// Kernels per pass of a device loop: the sweep (or CG's two) and the loop control.
// Whether fine passes end with the coarse-grid correction.
bool corrects(const dd_inpaint* h) { return h->prm.ml_mode == DD_ML_CORRECTION && h->lv.size() >= 2; }

// Relative residual to which the small-grid CG solves the coarse correction equation.
constexpr double kCorrectionCgTol = 1e-3;

// Kernels of the coarse-grid correction after one fine sweep, without its gate:
// fine residual, restrictions, the coarse solve (reset + ORAS sweeps, or the
// small-grid CG), prolongations, and the three step kernels.
int correction_kernels(const dd_inpaint* h) {
    const int nl = (int)h->lv.size();
    const int coarse = h->prm.correction_cg > 0 ? 1 : 1 + h->prm.correction_sweeps;
    return 1 + (nl - 1) + coarse + (nl - 2) + 3;
}

// Kernels of one pass of a device loop: the sweep (or CG's two) and the loop
// control; on a correcting fine level the correction kernels (gate and body)
// are counted apart, from the gate's launch count (count_loop_launches).
int pass_kernels_of(const dd_inpaint* h, const Level& L) {
    (void)L;
    return h->prm.solver == DD_SOLVER_CG ? 3 : 2;
}

dd::CGArgs cg_args(const dd_inpaint* h, const Level& L) {
    dd::CGArgs a{};
    a.H = L.H; a.W = L.W; a.P = L.P; a.C = h->C; a.mp = L.W;
    a.plane = L.plane();
    a.mask = L.mask;
    a.x = L.u[0]; a.r = L.cg_r; a.q = L.cg_q;
    a.p[0] = L.cg_p[0]; a.p[1] = L.cg_p[1];
    a.part = L.cg_part; a.scal = L.cg_scal; a.ref = L.ref_d;
    a.flag = h->flag_d; a.state = h->sstate_d;
    a.tol = h->tol_d;
    return a;
}

// One pass of level L's iteration: an ORAS sweep (or probe) from the buffer
// the device state names, or one CG iteration.
// Coarse-grid correction of the fine iterate (the buffer sstate_d[0] names),
// all on st, each step a no-op once the fine stop flag is set:
//   r   = b - A u on the fine level (FP64-accurate residual pass),
//   g_c = r summed over 2x2 blocks down to the coarsest level (the h = 1
//         stencil there carries the factor 4 per level),
//   e_c = correction_sweeps ORAS sweeps on A_c e_c = g_c from e_c = 0, with
//         e_c = 0 on coarse-known pixels,
//   d   = e_c prolonged bilinearly level by level, on unknown fine pixels,
//   u  += omega d with omega = (r, d) / (d, A d) per channel, the step that
//         minimises the A-norm of the error along d: the rediscretised coarse
//         problem is not the Galerkin one, and its plain correction can
//         overshoot.
// A gate skips the correction once the fine stop flag is set, and switches
// corrections off for the rest of the solve once a pass reduced the fine
// residual by less than a factor 0.7: with the non-symmetric ORAS smoother
// the corrected iteration can still grow slowly, where plain ORAS converges.
// The gate runs first (enqueue_correction) and the correction kernels each
// return at once when it says skip.
int enqueue_correction_body(dd_inpaint* h, cudaStream_t st) {
    const int nl = (int)h->lv.size();
    Level& F = h->lv[0];
    Level& Lc = h->lv[nl - 1];
    const int* skip = h->corr_gate;
    dd::Res64Args a{};
    a.H = F.H; a.W = F.W; a.C = h->C;
    a.u = F.u[0]; a.u1 = F.u[1]; a.sel = h->sstate_d; a.up = F.P; a.uplane = F.plane();
    a.mask = F.mask; a.mp = F.W;
    a.g_out = h->corr_r; a.gst = Store::F32; a.gp = F.P; a.gplane = F.plane();
    a.scale_inv = h->ones_d;
    a.part = h->res_part; a.nblk = h->res_nblk;
    a.skip = skip;
    DD_CK(dd::launch_res64(a, st));
    const float* src = h->corr_r;
    int sp = F.P;
    long long splane = F.plane();
    for (int l = 1; l < nl; ++l) {
        Level& L = h->lv[l];
        const Level& Lf = h->lv[l - 1];
        DD_CK(dd::launch_restrict_sum(Lf.H, Lf.W, h->C, src, sp, splane, L.corr_g, L.P, L.plane(), skip, st));
        src = L.corr_g;
        sp = L.P;
        splane = L.plane();
    }
    const float* e0 = Lc.u[0];
    const float* e1 = Lc.u[1];
    const int* sel = h->state_c;
    if (h->prm.correction_cg > 0) {   // the small-grid CG: e_c into u[0]
        DD_CK(dd::launch_coarse_cg(Lc.H, Lc.W, h->C, Lc.mask, Lc.W, Lc.corr_g, Lc.P, Lc.plane(), Lc.u[0], Lc.P,
                                   Lc.plane(), h->prm.correction_cg, kCorrectionCgTol, nullptr, skip, st));
        e1 = Lc.u[0];
        sel = nullptr;
    } else {   // correction_sweeps ORAS sweeps from e_c = 0
        const size_t cbytes = sizeof(float) * (size_t)h->C * Lc.plane();
        DD_CK(cudaMemsetAsync(Lc.u[0], 0, cbytes, st));
        DD_CK(cudaMemsetAsync(Lc.u[1], 0, cbytes, st));
        DD_CK(dd::launch_reset_sweep_state(h->state_c, h->flag_c, 0, h->tol_c, -1.0, st, skip));
        const dd::SweepPair pair{{&Lc.map_u[0], &Lc.map_u[1]}, {Lc.u[0], Lc.u[1]}};
        const dd::SweepStop stop{Lc.partial, h->norms2_c, Lc.ref_d, h->tol_c, 0.0, h->flag_c, h->state_c,
                                 0, nullptr, err_word(h), h->prm.test_stall_polls};
        for (int i = 0; i < h->prm.correction_sweeps; ++i)
            DD_CK(dd::launch_sweep(Store::F32, Lc.geom, h->C, Lc.plane(), pair, &Lc.map_cg, Lc.tmask, stop,
                                   h->prm.robin_p, h->prm.local_cg_iters, st, (float)h->prm.local_rtol));
    }
    int eH = Lc.H, eW = Lc.W, ep = Lc.P;
    long long eplane = Lc.plane();
    for (int l = nl - 2; l >= 1; --l) {
        Level& L = h->lv[l];
        DD_CK(dd::launch_prolong_sel(eH, eW, L.H, L.W, h->C, e0, e1, sel, ep, eplane, nullptr, L.W, nullptr, L.P,
                                     L.plane(), L.corr_g, L.P, L.plane(), st));
        e0 = e1 = L.corr_g;
        sel = nullptr;
        eH = L.H; eW = L.W; ep = L.P;
        eplane = L.plane();
    }
    // energy-optimal step along the prolonged correction d (written over r)
    double* part = reinterpret_cast<double*>(h->res_part);
    DD_CK(dd::launch_corr_dir(eH, eW, F.H, F.W, h->C, e0, e1, sel, ep, eplane, F.mask, F.W, h->corr_r, F.P,
                              F.plane(), skip, part, h->res_nblk, h->res_ticket, h->corr_dots, st));
    DD_CK(dd::launch_corr_curv(F.H, F.W, h->C, h->corr_r, F.P, F.plane(), skip, part, h->res_nblk, h->res_ticket,
                               h->corr_dots + h->C, h->corr_dots, h->corr_dots + 2 * h->C, st));
    DD_CK(dd::launch_corr_step(F.H, F.W, h->C, h->corr_r, F.P, F.plane(), h->corr_dots + 2 * h->C, F.u[0], F.u[1],
                               h->sstate_d, F.P, F.plane(), skip, st));
    return DD_OK;
}

// The correction as plain launches: the gate and every kernel of the body.
int enqueue_correction(dd_inpaint* h, cudaStream_t st) {
    DD_CK(dd::launch_corr_gate(h->flag_d, h->norms2_d, h->C, h->sstate_d, h->corr_gate, h->corr_prev,
                               h->prm.correction_trigger, h->tol_d, st));
    return enqueue_correction_body(h, st);
}

// Corrections on, no residual history: before a solve's fine iterations.
int reset_correction(dd_inpaint* h, cudaStream_t st) {
    DD_CK(cudaMemsetAsync(h->corr_gate, 0, kGateWords * sizeof(int), st));
    DD_CK(cudaMemsetAsync(h->corr_prev, 0, 2 * sizeof(double), st));
    return DD_OK;
}

int capture_append(cudaStream_t st, const std::function<int(cudaGraph_t, const cudaGraphNode_t*,
                                                            const cudaGraphEdgeData*, size_t, cudaGraphNode_t*)>& add);

// with_correction: a correcting fine level's sweep is followed by the
// correction (its gate decides whether it does anything).
int enqueue_pass(dd_inpaint* h, Level& L, cudaStream_t st, bool count_work = false, bool with_correction = true) {
    if (h->prm.solver == DD_SOLVER_CG) {
        DD_CK(dd::launch_cg_iteration(cg_args(h, L), st));
        return DD_OK;
    }
    const dd::SweepPair pair{{&L.map_u[0], &L.map_u[1]}, {L.u[0], L.u[1]}};
    const dd::SweepStop stop = make_stop(h, L.partial, L.ref_d, 0.0, count_work ? h->work_d : nullptr);
    DD_CK(dd::launch_sweep(Store::F32, L.geom, h->C, L.plane(), pair, nullptr, L.tmask, stop, h->prm.robin_p,
                           h->prm.local_cg_iters, st, (float)h->prm.local_rtol));
    if (with_correction && &L == &h->lv[0] && corrects(h)) DD_TRY(enqueue_correction(h, st));
    return DD_OK;
}

// Add a device loop to graph g after the nodes deps: an entry kernel (pass
// counter 0, condition 1), then a WHILE node whose body (pass(body_stream),
// then the loop control) is captured on body_stream.  *last = the WHILE node.  The loop ends
// when flag_d[0] is set, when sstate_d[1] reaches cap or after max_passes.
// control (may be empty): launches the loop control in place of loop_ctl_kernel.
// corrected_phase: the loop is the corrected phase of a fine level with a
// correction trigger; its entry kernel lets it run only if the trigger fired,
// and the pass counter continues from the plain phase.
int add_loop_fn(dd_inpaint* h, int cap, int max_passes, cudaGraph_t g, const cudaGraphNode_t* deps,
                const cudaGraphEdgeData* edges, size_t ndeps, cudaStream_t body_stream,
                const std::function<int(cudaStream_t)>& pass, cudaGraphNode_t* last,
                const std::function<cudaError_t(cudaStream_t, cudaGraphConditionalHandle)>& control = {},
                bool corrected_phase = false) {
    cudaGraphConditionalHandle cond;
    DD_CK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
    // entry node: pass counter 0, condition 1 (re-armed on every entry when nested)
    int* ctl = h->ctl_d;
    void* kargs[2] = {&ctl, &cond};
    const int* flag = h->flag_d;
    const int* state = h->sstate_d;
    const int* gate = h->corr_gate;
    int cap_v = cap, maxp_v = max_passes;
    void* kargs_c[7] = {&ctl, &flag, &state, &gate, &cap_v, &maxp_v, &cond};
    cudaGraphNodeParams kp{};
    kp.type = cudaGraphNodeTypeKernel;
    kp.kernel.func = const_cast<void*>(corrected_phase ? dd::loop_begin_corrected_kernel_fn()
                                                       : dd::loop_begin_kernel_fn());
    kp.kernel.gridDim = dim3(1, 1, 1);
    kp.kernel.blockDim = dim3(32, 1, 1);
    kp.kernel.sharedMemBytes = 0;
    kp.kernel.kernelParams = corrected_phase ? kargs_c : kargs;
    cudaGraphNode_t reset = nullptr, loop = nullptr;
    DD_CK(cudaGraphAddNode(&reset, g, deps, edges, ndeps, &kp));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    DD_CK(cudaGraphAddNode(&loop, g, &reset, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    DD_CK(cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const int rc = pass(body_stream);
    const cudaError_t el = rc != DD_OK ? cudaSuccess
                           : control ? control(body_stream, cond)
                                 : dd::launch_loop_ctl(h->flag_d, h->sstate_d, h->ctl_d, cap, max_passes, cond,
                                                       body_stream);
    cudaGraph_t captured = body;
    const cudaError_t ec = cudaStreamEndCapture(body_stream, &captured);
    if (rc != DD_OK) return rc;
    DD_CK(el);
    DD_CK(ec);
    *last = loop;
    return DD_OK;
}

// Level L's loop (its sweeps or CG iterations).  The pass bound: CG applies an
// iteration in every pass; ORAS follows a failed probe by a full sweep, so at
// most 2 cap + 1 passes reach cap full sweeps.
int add_loop(dd_inpaint* h, Level& L, int cap, cudaGraph_t g, const cudaGraphNode_t* deps,
             const cudaGraphEdgeData* edges, size_t ndeps, cudaGraphNode_t* last) {
    if (h->prm.solver == DD_SOLVER_ORAS) DD_CK(dd::prepare_sweep(Store::F32, L.geom, false));
    const int max_passes = h->prm.solver == DD_SOLVER_CG ? cap + 1 : 2 * cap + 2;
    if (&L == &h->lv[0] && corrects(h) && h->prm.correction_trigger > 0.0) {
        // plain phase: sweep -> loop control, which also ends the loop when the
        // trigger fires; then the corrected phase (sweep -> correction -> loop
        // control), which runs only if it fired
        cudaGraphNode_t plain = nullptr;
        DD_TRY(add_loop_fn(
            h, cap, max_passes, g, deps, edges, ndeps, h->cap_stream,
            [&](cudaStream_t bs) { return enqueue_pass(h, L, bs, false, false); }, &plain,
            [&](cudaStream_t bs, cudaGraphConditionalHandle cw) {
                return dd::launch_loop_ctl_trigger(h->flag_d, h->sstate_d, h->ctl_d, cap, max_passes, cw,
                                                   h->norms2_d, h->C, h->corr_gate, h->corr_prev,
                                                   h->prm.correction_trigger, h->tol_d, bs);
            }));
        return add_loop_fn(h, cap, max_passes, g, &plain, nullptr, 1, h->cap_stream,
                           [&](cudaStream_t bs) { return enqueue_pass(h, L, bs); }, last, {}, true);
    }
    return add_loop_fn(h, cap, max_passes, g, deps, edges, ndeps, h->cap_stream,
                       [&](cudaStream_t bs) { return enqueue_pass(h, L, bs); }, last);
}

// Append nodes to the graph that st is capturing, after st's current
// dependencies (add(graph, deps, edges, n, &last)); st then continues from last.
int capture_append(cudaStream_t st, const std::function<int(cudaGraph_t, const cudaGraphNode_t*,
                                                            const cudaGraphEdgeData*, size_t, cudaGraphNode_t*)>& add) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    DD_CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, &edges, &nd));
    if (cs != cudaStreamCaptureStatusActive) {
        set_error("device loop: the stream is not capturing");
        return DD_ECUDA;
    }
    // the arrays returned above are valid until the next capture call on st
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    std::vector<cudaGraphEdgeData> ev;
    if (edges) ev.assign(edges, edges + nd);
    cudaGraphNode_t last = nullptr;
    DD_TRY(add(cg, dv.data(), edges ? ev.data() : nullptr, nd, &last));
    DD_CK(cudaStreamUpdateCaptureDependencies(st, &last, nullptr, 1, cudaStreamSetCaptureDependencies));
    return DD_OK;
}

// Level L's loop as a graph of its own for (cap, tol), built on first use and
// kept while both stay the same.
int loop_graph(dd_inpaint* h, Level& L, int cap, cudaGraphExec_t* out) {
    LoopGraph& G = L.loop;
    if (G.exec != nullptr && G.cap == cap) {
        *out = G.exec;
        return DD_OK;
    }
    destroy_loop(G);
    DD_CK(cudaGraphCreate(&G.graph, 0));
    cudaGraphNode_t last = nullptr;
    const int rc = add_loop(h, L, cap, G.graph, nullptr, nullptr, 0, &last);
    if (rc != DD_OK) {
        destroy_loop(G);
        return rc;
    }
    DD_CK(cudaGraphInstantiate(&G.exec, G.graph, 0));
    G.cap = cap;
    *out = G.exec;
    return DD_OK;
}

// Run level L's loop on st and resolve its result into L.state_d.  Outside a
// capture the level's own graph is launched; inside a stream capture (a
// dd_batch graph) the loop's nodes join the graph being captured.
int run_loop(dd_inpaint* h, Level& L, int cap, cudaStream_t st, bool capture) {
    if (cap > 0 && capture) {   // (a WHILE body runs at least once)
        DD_TRY(capture_append(st, [&](cudaGraph_t cg, const cudaGraphNode_t* d, const cudaGraphEdgeData* e, size_t n,
                                      cudaGraphNode_t* last) { return add_loop(h, L, cap, cg, d, e, n, last); }));
    } else if (cap > 0) {
        cudaGraphExec_t ex = nullptr;
        DD_TRY(loop_graph(h, L, cap, &ex));
        DD_CK(cudaGraphLaunch(ex, st));
    } else {
        DD_CK(cudaMemsetAsync(h->ctl_d, 0, 4 * sizeof(int), st));
    }
    DD_LAUNCH(h, dd::launch_resolve(h->flag_d, h->sstate_d, h->ctl_d, L.state_d, st));
    L.loop_pending = true;
    return DD_OK;
}

// After the level states have been read back (h_state, 4 ints per level):
// add the kernels the device loops ran to the launch count.
void count_loop_launches(dd_inpaint* h) {
    for (size_t l = 0; l < h->lv.size() && l < DD_MAX_LEVELS; ++l) {
        if (!h->lv[l].loop_pending) continue;
        h->lv[l].loop_pending = false;
        h->launches += (long long)h->h_state[4 * l + 3] * pass_kernels_of(h, h->lv[l]);
        if (l == 0 && corrects(h)) h->launches += (long long)h->h_flag[7] * (1 + correction_kernels(h));
    }
}

// ORAS on level L from the iterate in u[0], at most n full sweeps, under the
// device stop test; the result is resolved into L.state_d.  No host
// synchronisation.  Plain launches (loop = false): n launches, those after the
// stop do no work.
int enqueue_sweeps(dd_inpaint* h, Level& L, int n, double tol, cudaStream_t st, bool timed, bool loop,
                   bool capture) {
    DD_LAUNCH(h, dd::launch_reset_sweep_state(h->sstate_d, h->flag_d, 0, h->tol_d, tol, st));
    if (&L == &h->lv[0] && corrects(h)) DD_TRY(reset_correction(h, st));
    if (loop) return run_loop(h, L, n, st, capture);
    if (timed) DD_CK(cudaMemsetAsync(h->work_d, 0, sizeof(unsigned long long) * kWorkWords, st));
    for (int i = 0; i < n; ++i) {
        if (timed && i < dd_inpaint::kFirst) DD_CK(cudaEventRecord(h->sw_ev[2 * i], st));
        DD_TRY(enqueue_pass(h, L, st, timed));
        h->launches += pass_kernels_of(h, L) - 1 + ((&L == &h->lv[0] && corrects(h)) ? 1 + correction_kernels(h) : 0);
        if (timed && i < dd_inpaint::kFirst) DD_CK(cudaEventRecord(h->sw_ev[2 * i + 1], st));
    }
    DD_LAUNCH(h, dd::launch_resolve(h->flag_d, h->sstate_d, nullptr, L.state_d, st));
    return DD_OK;
}

// At most n CG iterations on level L from the iterate in u[0] (the residual is
// formed afresh, so this also restarts CG), then record the result (always in
// u[0]) into L.state_d.  No host synchronisation.
int enqueue_cg(dd_inpaint* h, Level& L, int n, double tol, cudaStream_t st, bool loop, bool capture) {
    DD_LAUNCH(h, dd::launch_reset_sweep_state(h->sstate_d, h->flag_d, 0, h->tol_d, tol, st));
    const int nblk = dd::res64_blocks(L.H, L.W);
    dd::Res64Args ra{};
    ra.H = L.H; ra.W = L.W; ra.C = h->C;
    ra.u = L.u[0]; ra.up = L.P; ra.uplane = L.plane();
    ra.mask = L.mask; ra.mp = L.W;
    ra.g_out = L.cg_r; ra.gst = Store::F32; ra.gp = L.P; ra.gplane = L.plane();
    ra.scale_inv = h->ones_d;
    ra.part = h->res_part; ra.nblk = nblk;
    ra.out = h->res_out; ra.ticket = h->res_ticket;
    DD_LAUNCH(h, dd::launch_res64(ra, st));
    DD_LAUNCH(h, dd::launch_cg_init(h->res_out, L.cg_scal, h->C, st));
    DD_CK(cudaMemsetAsync(L.cg_p[0], 0, sizeof(float) * (size_t)h->C * L.plane(), st));
    if (loop) return run_loop(h, L, n, st, capture);
    for (int i = 0; i < n; ++i) {
        DD_TRY(enqueue_pass(h, L, st));
        h->launches += 2;
    }
    DD_LAUNCH(h, dd::launch_resolve(h->flag_d, h->sstate_d, nullptr, L.state_d, st));
    return DD_OK;
}

// A level solve under the device stop test: ORAS sweeps or CG iterations.
int enqueue_level(dd_inpaint* h, Level& L, int n, double tol, cudaStream_t st, bool timed, bool capture) {
    const bool loop = loop_mode(h, timed);
    if (h->prm.solver == DD_SOLVER_CG) return enqueue_cg(h, L, n, tol, st, loop, capture);
    return enqueue_sweeps(h, L, n, tol, st, timed, loop, capture);
}

// Coarse-to-fine initialisation (Sec. 4): coarsest level from u0 = C f, each
// level swept to coarse_tol (at most coarse_sweeps sweeps) and prolonged as the
// next level's start; the fine level's start is left in u[0].  Everything is
// enqueued without host synchronisation: each level's result buffer is chosen
// on the device.
int cascade(dd_inpaint* h, cudaStream_t st, bool capture) {
    const int nl = h->nc;
    for (int l = nl - 1; l >= 1; --l) {
        Level& L = h->lv[l];
        if (l == nl - 1) {
            DD_LAUNCH(h, dd::launch_copy2d(L.H, L.W, h->C, L.f, L.P, L.plane(), L.u[0], L.P, L.plane(), st));
        } else {
            Level& Cc = h->lv[l + 1];
            DD_LAUNCH(h, dd::launch_prolong_sel(Cc.H, Cc.W, L.H, L.W, h->C, Cc.u[0], Cc.u[1], Cc.state_d, Cc.P,
                                                Cc.plane(), L.mask, L.W, L.f, L.P, L.plane(), L.u[0], L.P,
                                                L.plane(), st));
        }
        if (L.solved) {
            DD_TRY(enqueue_level(h, L, h->prm.coarse_sweeps, h->prm.coarse_tol, st, false, capture));
        } else {   // pass-through level: its result is the prolonged start in u[0], no sweeps
            DD_CK(cudaMemsetAsync(L.state_d, 0, 4 * sizeof(int), st));
        }
    }
    Level& F = h->lv[0];
    if (nl > 1) {
        Level& Cc = h->lv[1];
        DD_LAUNCH(h, dd::launch_prolong_sel(Cc.H, Cc.W, F.H, F.W, h->C, Cc.u[0], Cc.u[1], Cc.state_d, Cc.P,
                                            Cc.plane(), F.mask, F.W, F.f, F.P, F.plane(), F.u[0], F.P, F.plane(),
                                            st));
    } else {
        DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.f, F.P, F.plane(), F.u[0], F.P, F.plane(), st));
    }
    h->cur = 0;
    return DD_OK;
}

// The fine level's result (the buffer lv[0].state_d names) copied to the
// dense output u_out by the residual pass, which also forms its FP64-accurate
// residual norms into h_res[0..C) (read back on st).
int output_and_residual(dd_inpaint* h, float* u_out, cudaStream_t st) {
    Level& L = h->lv[0];
    dd::Res64Args a{};
    a.H = L.H; a.W = L.W; a.C = h->C;
    a.u = L.u[0]; a.u1 = L.u[1]; a.sel = L.state_d; a.up = L.P; a.uplane = L.plane();
    a.mask = L.mask; a.mp = L.W;
    a.g_out = nullptr; a.gst = Store::F32;
    a.part = h->res_part; a.nblk = h->res_nblk;
    a.out = h->res_out; a.ticket = h->res_ticket;
    a.copy_out = u_out; a.cp = L.W; a.cplane = (long long)L.H * L.W;
    DD_LAUNCH(h, dd::launch_res64(a, st));
    DD_CK(cudaMemcpyAsync(h->h_res, h->res_out, sizeof(double2) * h->C, cudaMemcpyDeviceToHost, st));
    return DD_OK;
}

int rel_from_h_res(dd_inpaint* h, std::vector<double>& rel, std::vector<double>& rmax, std::vector<double>& rnorm) {
    const Level& L = h->lv[0];
    rel.assign(h->C, 0.0);
    rmax.assign(h->C, 0.0);
    rnorm.assign(h->C, 0.0);
    for (int c = 0; c < h->C; ++c) {
        rnorm[c] = std::sqrt(h->h_res[c].x);
        rmax[c] = h->h_res[c].y;
        rel[c] = rnorm[c] / (L.ref[c] > 0.0 ? L.ref[c] : 1.0);
        if (!std::isfinite(rel[c])) { set_error("non-finite residual"); return DD_ENUMERIC; }
    }
    return DD_OK;
}

// Read the per-level sweep counts resolved on the device (after a sync).
void take_level_stats(dd_inpaint* h) {
    for (int l = 1; l < h->nc && l < DD_MAX_LEVELS; ++l) h->stats.sweeps_per_level[l] = h->h_state[4 * l + 1];
    for (int l = 1; l < h->nc; ++l) h->stats.sweeps_total += h->h_state[4 * l + 1];
}

// Fine-level launches enqueued before the first read-back.
int first_chunk(const dd_inpaint* h) {
    const int n = h->prm.solver == DD_SOLVER_CG ? 256 : dd_inpaint::kFirst;
    return std::min(n, h->prm.max_sweeps);
}

// The end of an enqueued FP32 solve: the output of the fine level's resolved
// iterate with its FP64-accurate residual, and the read-back of everything the
// finish step needs (level states, flags, reference norms, pixel counts).
int enqueue_output_readback(dd_inpaint* h, float* u_out, double tol, cudaStream_t st, bool capture, bool timed) {
    const int nl = h->nc;
    Level& F = h->lv[0];
    DD_TRY(output_and_residual(h, u_out, st));
    DD_CK(cudaMemcpyAsync(h->h_state, F.state_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    for (int l = 1; l < nl; ++l)
        DD_CK(cudaMemcpyAsync(h->h_state + 4 * l, h->lv[l].state_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DD_CK(cudaMemcpyAsync(h->h_flag, h->flag_d, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DD_CK(cudaMemcpyAsync(h->h_flag + 3, err_word(h), sizeof(int), cudaMemcpyDeviceToHost, st));
    DD_CK(cudaMemcpyAsync(h->h_ref, F.ref_d, sizeof(double) * h->C, cudaMemcpyDeviceToHost, st));
    DD_CK(cudaMemcpyAsync(h->h_cnt, h->count_d, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    if (corrects(h)) {   // corrections applied, gate launches
        DD_CK(cudaMemcpyAsync(h->h_flag + 6, h->corr_gate + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
        DD_CK(cudaMemcpyAsync(h->h_flag + 7, h->corr_gate + 6, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    if (timed)
        DD_CK(cudaMemcpyAsync(h->h_work, h->work_d, sizeof(unsigned long long) * kWorkWords, cudaMemcpyDeviceToHost,
                              st));
    if (!capture) DD_CK(cudaEventRecord(h->ev1, st));
    h->pending = true;
    h->pending_out = u_out;
    h->pending_tol = tol;
    return DD_OK;
}

// FP32 path, part 1: enqueue the cascade, the first fine chunk, the output of
// the resolved buffer, its residual and the read-back of everything the host
// needs.  No host synchronisation.  capture = 1 inside a stream capture
// (no events, no timing).
int fp32_enqueue(dd_inpaint* h, float* u_out, double tol, cudaStream_t st, bool capture) {
    std::memset(&h->stats, 0, sizeof(h->stats));
    h->stats.channels = h->C;
    h->stats.device_bytes = h->bytes;
    const int nl = (int)h->lv.size();
    Level& F = h->lv[0];
    h->ev_recorded = !capture;
    if (!capture) DD_CK(cudaEventRecord(h->ev0, st));
    DD_TRY(clear_error(h, st));
    h->pending_cascaded = !h->warm;
    if (!h->warm) {
        DD_TRY(cascade(h, st, capture));
    } else if (h->cur != 0) {
        DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.u[1], F.P, F.plane(), F.u[0], F.P, F.plane(), st));
        h->cur = 0;
    }
    h->warm = false;
    // a device loop runs to the sweep limit; launches stop at the first chunk
    const bool timed = h->prm.timing != 0 && !capture;
    const int n1 = loop_mode(h, timed) ? h->prm.max_sweeps : first_chunk(h);
    DD_TRY(enqueue_level(h, F, n1, tol, st, timed, capture));
    DD_TRY(enqueue_output_readback(h, u_out, tol, st, capture, timed));
    (void)nl;
    return DD_OK;
}

// FP32 path, part 2: wait for the enqueued work, read the result and, if the
// first chunk did not reach tol (or the FP32 fused estimate was optimistic),
// continue under host control on st.
int fp32_finish(dd_inpaint* h, cudaStream_t st) {
    if (!h->pending) { set_error("no solve in flight"); return DD_EINVAL; }
    h->pending = false;
    Level& F = h->lv[0];
    const int nl = (int)h->lv.size();
    float* u_out = h->pending_out;
    const double tol = h->pending_tol;
    if (h->ev_recorded) DD_CK(cudaEventSynchronize(h->ev1));
    else DD_CK(cudaStreamSynchronize(st));
    // pixel counts and reference norms of the data this solve used
    h->local_unknowns = (long long)h->h_cnt[0];
    h->stats.local_unknowns = h->local_unknowns;
    if (h->counts_pending) {
        h->counts_pending = false;
        if (h->h_cnt[1] == 0) { h->valid = false; set_error("empty mask"); return DD_EEMPTYMASK; }
    }
    F.ref.assign(h->h_ref, h->h_ref + h->C);
    if (h->h_flag[3] != 0) { set_error("a bounded device wait for a staged tile gave up"); return DD_ETIMEOUT; }
    if (h->pending_cascaded) take_level_stats(h);
    count_loop_launches(h);
    h->stats.coarse_corrections = corrects(h) ? h->h_flag[6] : 0;
    const int status = h->h_state[2], applied = h->h_state[1];
    if (status == 2) { set_error("non-finite residual norm"); return DD_ENUMERIC; }
    const int n1 = first_chunk(h);
    if (h->prm.timing != 0 && h->ev_recorded && h->prm.solver == DD_SOLVER_ORAS) {
        h->stats.fine_cg_pixel_steps = (long long)h->h_work[0];
        h->stats.fine_swept_unknowns = (long long)h->h_work[1];
        for (int i = 0; i < n1 && i < dd::kTimedLaunches; ++i) {   // the launches that ran as full sweeps
            if (h->h_work[2 + i] == 0) continue;
            float ms = 0.f;
            DD_CK(cudaEventElapsedTime(&ms, h->sw_ev[2 * i], h->sw_ev[2 * i + 1]));
            h->stats.fine_sweep_ms += ms;
            h->stats.fine_sweep_launches += 1;
        }
    }
    int fine_sweeps = applied;
    h->cur = h->h_state[0];
    std::vector<double> rel, rmax, rnorm;
    DD_TRY(rel_from_h_res(h, rel, rmax, rnorm));
    double worst = *std::max_element(rel.begin(), rel.end());
    bool converged = false;
    if (worst <= tol) {   // the FP64-accurate residual of the output decides
        converged = true;
    } else {
        h->stats.host_continued = 1;
        double target = status == 1 ? tol * 0.5 : tol;
        for (int attempt = 0; attempt < 4 && fine_sweeps < h->prm.max_sweeps; ++attempt) {
            int app = 0;
            bool conv = false;
            if (h->prm.solver == DD_SOLVER_CG) {
                // restart CG from the current iterate (fresh residual), read back once per chunk
                const bool loop = loop_mode(h, false);
                while (!conv && fine_sweeps + app < h->prm.max_sweeps) {
                    const int left = h->prm.max_sweeps - fine_sweeps - app;
                    const int n = loop ? left : std::min(64, left);
                    DD_TRY(enqueue_cg(h, F, n, target, st, loop, false));
                    DD_CK(cudaMemcpyAsync(h->h_state, F.state_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
                    DD_CK(cudaStreamSynchronize(st));
                    count_loop_launches(h);
                    app += h->h_state[1];
                    conv = h->h_state[2] == 1;
                    if (h->h_state[2] == 2) { set_error("non-finite residual norm"); return DD_ENUMERIC; }
                }
                h->cur = 0;
            } else {
                void* bufs[2] = {F.u[0], F.u[1]};
                DD_TRY(run_sweeps(h, F.geom, Store::F32, bufs, F.map_u, h->cur, nullptr, F.tmask, F.partial,
                                  F.ref_d, target, 0.0, h->prm.max_sweeps - fine_sweeps, st, &app, &conv, true));
            }
            fine_sweeps += app;
            DD_TRY(fine_residual64(h, st, rel, rmax, rnorm));
            worst = *std::max_element(rel.begin(), rel.end());
            if (worst <= tol) { converged = true; break; }
            if (!conv) break;
            target *= 0.5;
        }
        DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.u[h->cur], F.P, F.plane(), u_out, F.W,
                                       (long long)F.H * F.W, st));
        if (h->ev_recorded) DD_CK(cudaEventRecord(h->ev1, st));   // ms_total spans the continuation
        DD_CK(cudaStreamSynchronize(st));
    }
    (void)nl;
    h->stats.sweeps_per_level[0] = fine_sweeps;
    h->stats.sweeps_total += fine_sweeps;
    h->stats.converged = converged ? 1 : 0;
    for (int c = 0; c < h->C && c < DD_MAX_STAT_CHANNELS; ++c) h->stats.rel_residual[c] = rel[c];
    if (h->ev_recorded) {
        float ms = 0.f;
        if (cudaEventQuery(h->ev1) == cudaSuccess) DD_CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        h->stats.ms_total = ms;
    }
    h->stats.kernel_launches = h->launches;
    return converged ? DD_OK : DD_ENOTCONVERGED;
}

// ---- device-driven FP64 correction loop (precision != FP32, device_loop = 1) ----------
// One inner pass: a sweep of the correction equation A e = g_hat on the fine
// level in the low storage type, from the e buffer the device state names.
int ref_pass(dd_inpaint* h, cudaStream_t st) {
    Level& F = h->lv[0];
    const dd::SweepPair pair{{&h->map_e[0], &h->map_e[1]}, {h->e[0], h->e[1]}};
    const double stall = h->lowst == Store::F32 ? 0.0 : 0.7;
    const dd::SweepStop stop = make_stop(h, F.partial, h->inner_ref_d, stall);
    DD_CK(dd::launch_sweep(h->lowst, F.geom, h->C, F.plane(), pair, &h->map_g, F.tmask, stop, h->prm.robin_p,
                           h->prm.local_cg_iters, st, (float)h->prm.local_rtol));
    return DD_OK;
}

// The outer loop (WHILE node) of the correction scheme, added to g after deps.
// Its body, captured on cap_stream, is one correction:
//   res64(u) -> ref_outer_ctl (stop, or the scales of this correction) ->
//   scaled residual g_hat in the low type -> e = 0 -> the inner sweeps as a
//   nested device loop (bodies on cap_stream2) to inner_tol ->
//   u += scale * e (FP64 arithmetic);
// every step after the control is skipped once the loop has ended.
int add_ref_outer(dd_inpaint* h, cudaGraph_t g, const cudaGraphNode_t* deps, const cudaGraphEdgeData* edges,
                  size_t ndeps, cudaGraphNode_t* last) {
    Level& F = h->lv[0];
    DD_CK(dd::prepare_sweep(h->lowst, F.geom, true));
    cudaGraphConditionalHandle cond;
    DD_CK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop = nullptr;
    DD_CK(cudaGraphAddNode(&loop, g, deps, edges, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t bs = h->cap_stream;
    DD_CK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const int* skip = h->ref_ctl_d + 5;
    auto steps = [&]() -> int {
        dd::Res64Args a{};
        a.H = F.H; a.W = F.W; a.C = h->C;
        a.u = F.u[0]; a.up = F.P; a.uplane = F.plane();
        a.mask = F.mask; a.mp = F.W;
        a.g_out = nullptr; a.gst = Store::F32;
        a.part = h->res_part; a.nblk = h->res_nblk;
        a.out = h->res_out; a.ticket = h->res_ticket;
        DD_CK(dd::launch_res64(a, bs));
        DD_CK(dd::launch_ref_outer_ctl(h->res_out, F.ref_d, h->C, h->ref_tol_d, h->prm.max_corrections,
                                       h->prm.max_sweeps, h->sstate_d, h->ctl_d, err_word(h), h->ref_ctl_d,
                                       h->scale_d, h->scale_inv_d, h->inner_ref_d, cond, bs));
        dd::Res64Args b{};
        b.H = F.H; b.W = F.W; b.C = h->C;
        b.u = F.u[0]; b.up = F.P; b.uplane = F.plane();
        b.mask = F.mask; b.mp = F.W;
        b.g_out = h->g; b.gst = h->lowst; b.gp = F.P; b.gplane = F.plane();
        b.scale_inv = h->scale_inv_d;
        b.part = h->res_part; b.nblk = h->res_nblk;
        b.skip = skip;
        DD_CK(dd::launch_res64(b, bs));
        DD_CK(cudaMemsetAsync(h->e[0], 0, dd::store_bytes(h->lowst) * (size_t)h->C * F.plane(), bs));
        DD_CK(dd::launch_reset_sweep_state(h->sstate_d, h->flag_d, 0, h->tol_d, h->prm.inner_tol, bs, skip));
        const int cap = h->prm.max_sweeps;
        DD_TRY(capture_append(bs, [&](cudaGraph_t cg, const cudaGraphNode_t* d, const cudaGraphEdgeData* e, size_t n,
                                      cudaGraphNode_t* l) {
            return add_loop_fn(h, cap, 2 * cap + 2, cg, d, e, n, h->cap_stream2,
                               [&](cudaStream_t s2) { return ref_pass(h, s2); }, l);
        }));
        DD_CK(dd::launch_correct(F.H, F.W, h->C, F.u[0], F.P, F.plane(), h->e[0], h->lowst, F.P, F.plane(), F.mask,
                                 F.W, h->scale_d, bs, h->e[1], h->sstate_d, skip));
        return DD_OK;
    };
    const int rc = steps();
    cudaGraph_t captured = body;
    const cudaError_t ec = cudaStreamEndCapture(bs, &captured);
    if (rc != DD_OK) return rc;
    DD_CK(ec);
    *last = loop;
    return DD_OK;
}

// The outer loop as a graph of its own (built when the handle is created).
int ref_graph(dd_inpaint* h, cudaGraphExec_t* out) {
    LoopGraph& G = h->ref_loop;
    if (G.exec != nullptr) {
        *out = G.exec;
        return DD_OK;
    }
    destroy_loop(G);
    DD_CK(cudaGraphCreate(&G.graph, 0));
    cudaGraphNode_t last = nullptr;
    const int rc = add_ref_outer(h, G.graph, nullptr, nullptr, 0, &last);
    if (rc != DD_OK) {
        destroy_loop(G);
        return rc;
    }
    DD_CK(cudaGraphInstantiate(&G.exec, G.graph, 0));
    *out = G.exec;
    return DD_OK;
}

// Correction modes, part 1: the cascade, the whole correction loop on the
// device, the output copy and the read-back of everything the host needs.
// No host synchronisation.
int ref_enqueue(dd_inpaint* h, float* u_out, double tol, cudaStream_t st, bool capture) {
    std::memset(&h->stats, 0, sizeof(h->stats));
    h->stats.channels = h->C;
    h->stats.device_bytes = h->bytes;
    const int nl = (int)h->lv.size();
    Level& F = h->lv[0];
    h->ev_recorded = !capture;
    if (!capture) DD_CK(cudaEventRecord(h->ev0, st));
    DD_TRY(clear_error(h, st));
    h->pending_cascaded = !h->warm;
    if (!h->warm) {
        DD_TRY(cascade(h, st, capture));
    } else if (h->cur != 0) {
        DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.u[1], F.P, F.plane(), F.u[0], F.P, F.plane(), st));
        h->cur = 0;
    }
    h->warm = false;
    // ref_ctl[0..8] = 0 and the tolerance (the sweep-state reset kernel on the control words)
    DD_LAUNCH(h, dd::launch_reset_sweep_state(h->ref_ctl_d, h->ref_ctl_d + 4, 0, h->ref_tol_d, tol, st));
    if (capture) {
        DD_TRY(capture_append(st, [&](cudaGraph_t cg, const cudaGraphNode_t* d, const cudaGraphEdgeData* e, size_t n,
                                      cudaGraphNode_t* l) { return add_ref_outer(h, cg, d, e, n, l); }));
    } else {
        cudaGraphExec_t ex = nullptr;
        DD_TRY(ref_graph(h, &ex));
        DD_CK(cudaGraphLaunch(ex, st));
    }
    DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.u[0], F.P, F.plane(), u_out, F.W, (long long)F.H * F.W, st));
    DD_CK(cudaMemcpyAsync(h->h_res, h->res_out, sizeof(double2) * h->C, cudaMemcpyDeviceToHost, st));
    DD_CK(cudaMemcpyAsync(h->h_ref_ctl, h->ref_ctl_d, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
    for (int l = 1; l < nl; ++l)
        DD_CK(cudaMemcpyAsync(h->h_state + 4 * l, h->lv[l].state_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DD_CK(cudaMemcpyAsync(h->h_flag, h->flag_d, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DD_CK(cudaMemcpyAsync(h->h_flag + 3, err_word(h), sizeof(int), cudaMemcpyDeviceToHost, st));
    DD_CK(cudaMemcpyAsync(h->h_ref, F.ref_d, sizeof(double) * h->C, cudaMemcpyDeviceToHost, st));
    DD_CK(cudaMemcpyAsync(h->h_cnt, h->count_d, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    if (!capture) DD_CK(cudaEventRecord(h->ev1, st));
    h->pending = true;
    h->pending_out = u_out;
    h->pending_tol = tol;
    return DD_OK;
}

// Correction modes, part 2: wait, read the outcome and the statistics.
int ref_finish(dd_inpaint* h, cudaStream_t st) {
    if (!h->pending) { set_error("no solve in flight"); return DD_EINVAL; }
    h->pending = false;
    Level& F = h->lv[0];
    if (h->ev_recorded) DD_CK(cudaEventSynchronize(h->ev1));
    else DD_CK(cudaStreamSynchronize(st));
    h->local_unknowns = (long long)h->h_cnt[0];
    h->stats.local_unknowns = h->local_unknowns;
    if (h->counts_pending) {
        h->counts_pending = false;
        if (h->h_cnt[1] == 0) { h->valid = false; set_error("empty mask"); return DD_EEMPTYMASK; }
    }
    F.ref.assign(h->h_ref, h->h_ref + h->C);
    if (h->h_flag[3] != 0) { set_error("a bounded device wait for a staged tile gave up"); return DD_ETIMEOUT; }
    if (h->pending_cascaded) take_level_stats(h);
    count_loop_launches(h);
    const int* c = h->h_ref_ctl;
    // per outer pass: residual, control, scaled residual, reset, correction;
    // per inner pass: the sweep and the loop control
    h->launches += 5LL * c[3] + 2LL * c[4];
    h->stats.corrections = c[0];
    h->stats.sweeps_per_level[0] = c[1];
    h->stats.sweeps_total += c[1];
    std::vector<double> rel, rmax, rnorm;
    if (c[2] == 3) { set_error("non-finite residual norm"); return DD_ENUMERIC; }
    DD_TRY(rel_from_h_res(h, rel, rmax, rnorm));
    const bool converged = c[2] == 1;
    h->stats.converged = converged ? 1 : 0;
    for (int ch = 0; ch < h->C && ch < DD_MAX_STAT_CHANNELS; ++ch) h->stats.rel_residual[ch] = rel[ch];
    if (h->ev_recorded) {
        float ms = 0.f;
        if (cudaEventQuery(h->ev1) == cudaSuccess) DD_CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        h->stats.ms_total = ms;
    }
    h->stats.kernel_launches = h->launches;
    return converged ? DD_OK : DD_ENOTCONVERGED;
}

// The solve as an enqueue (no host synchronisation) and a finish, for every
// precision: FP32 iterate, or the device-driven correction loop.
bool device_ref(const dd_inpaint* h) { return h->prm.precision != DD_PREC_FP32 && h->prm.device_loop != 0; }

int enqueue_solve(dd_inpaint* h, float* u_out, double tol, cudaStream_t st, bool capture) {
    return device_ref(h) ? ref_enqueue(h, u_out, tol, st, capture) : fp32_enqueue(h, u_out, tol, st, capture);
}

int finish_solve(dd_inpaint* h, cudaStream_t st) { return device_ref(h) ? ref_finish(h, st) : fp32_finish(h, st); }

int solve_impl(dd_inpaint* h, float* u_out, double tol, cudaStream_t st) {
    if (h->prm.precision == DD_PREC_FP32 || device_ref(h)) {
        DD_TRY(enqueue_solve(h, u_out, tol, st, false));
        return finish_solve(h, st);
    }
    if (h->counts_pending) {   // data loaded asynchronously: check it before the correction loop
        DD_CK(cudaStreamSynchronize(st));
        h->counts_pending = false;
        if (h->h_cnt[1] == 0) { h->valid = false; set_error("empty mask"); return DD_EEMPTYMASK; }
        h->local_unknowns = (long long)h->h_cnt[0];
        DD_CK(cudaMemcpy(h->h_ref, h->lv[0].ref_d, sizeof(double) * h->C, cudaMemcpyDeviceToHost));
        h->lv[0].ref.assign(h->h_ref, h->h_ref + h->C);
    }
    std::memset(&h->stats, 0, sizeof(h->stats));
    h->stats.channels = h->C;
    h->stats.device_bytes = h->bytes;
    h->stats.local_unknowns = h->local_unknowns;
    const int nl = (int)h->lv.size();
    DD_CK(cudaEventRecord(h->ev0, st));
    DD_TRY(clear_error(h, st));
    Level& F = h->lv[0];
    if (!h->warm) {
        DD_TRY(cascade(h, st, false));
    } else if (h->cur != 0) {
        DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.u[1], F.P, F.plane(), F.u[0], F.P, F.plane(), st));
        h->cur = 0;
    }
    const bool cascaded = !h->warm;
    h->warm = false;
    std::vector<double> rel, rmax, rnorm;
    int fine_sweeps = 0;
    bool converged = false;
    const long long dense_plane = (long long)F.H * F.W;
    {
        const Store lt = h->lowst;
        for (int corr = 0;; ++corr) {
            DD_TRY(fine_residual64(h, st, rel, rmax, rnorm));
            if (corr == 0 && cascaded) {
                for (int l = 1; l < nl; ++l)
                    DD_CK(cudaMemcpyAsync(h->h_state + 4 * l, h->lv[l].state_d, 4 * sizeof(int),
                                          cudaMemcpyDeviceToHost, st));
                DD_CK(cudaStreamSynchronize(st));
                take_level_stats(h);
                count_loop_launches(h);
            }
            const double worst = *std::max_element(rel.begin(), rel.end());
            if (worst <= tol) { converged = true; break; }
            if (corr >= h->prm.max_corrections || fine_sweeps >= h->prm.max_sweeps) break;
            for (int c = 0; c < h->C; ++c) {
                const double sc = rmax[c] > 0.0 ? rmax[c] : 1.0;
                h->h_small[c] = sc;
                h->h_small[h->C + c] = 1.0 / sc;
                h->h_small[2 * h->C + c] = rnorm[c] / sc;
            }
            DD_CK(cudaMemcpyAsync(h->scale_d, h->h_small, sizeof(double) * h->C, cudaMemcpyHostToDevice, st));
            DD_CK(cudaMemcpyAsync(h->scale_inv_d, h->h_small + h->C, sizeof(double) * h->C, cudaMemcpyHostToDevice,
                                  st));
            DD_CK(cudaMemcpyAsync(h->inner_ref_d, h->h_small + 2 * h->C, sizeof(double) * h->C,
                                  cudaMemcpyHostToDevice, st));
            DD_TRY(write_scaled_residual(h, st));
            DD_CK(dd::launch_fill_zero(lt, h->e[0], (size_t)h->C * F.plane(), st));
            int ecur = 0, app = 0;
            bool conv = false;
            void* bufs[2] = {h->e[0], h->e[1]};
            const double stall = lt == Store::F32 ? 0.0 : 0.7;
            DD_TRY(run_sweeps(h, F.geom, lt, bufs, h->map_e, ecur, &h->map_g, F.tmask, F.partial, h->inner_ref_d,
                              h->prm.inner_tol, stall, h->prm.max_sweeps - fine_sweeps, st, &app, &conv, true));
            fine_sweeps += app;
            DD_LAUNCH(h, dd::launch_correct(F.H, F.W, h->C, F.u[h->cur], F.P, F.plane(), bufs[ecur], lt, F.P,
                                            F.plane(), F.mask, F.W, h->scale_d, st));
            h->stats.corrections = corr + 1;
            DD_CK(cudaStreamSynchronize(st));   // h_small is reused by the next correction
        }
    }
    h->stats.sweeps_per_level[0] = fine_sweeps;
    h->stats.sweeps_total += fine_sweeps;
    h->stats.converged = converged ? 1 : 0;
    for (int c = 0; c < h->C && c < DD_MAX_STAT_CHANNELS; ++c) h->stats.rel_residual[c] = rel.empty() ? 0 : rel[c];
    DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.u[h->cur], F.P, F.plane(), u_out, F.W, dense_plane, st));
    DD_CK(cudaEventRecord(h->ev1, st));
    DD_CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    DD_CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->stats.ms_total = ms;
    h->stats.kernel_launches = h->launches;
    return converged ? DD_OK : DD_ENOTCONVERGED;
}

void free_all(dd_inpaint* h) {
    for (Level& L : h->lv) destroy_loop(L.loop);
    destroy_loop(h->ref_loop);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
    if (h->h_ref_ctl) cudaFreeHost(h->h_ref_ctl);
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    g_bytes_in_use.fetch_sub(h->bytes);
    h->bytes = 0;
    if (h->h_res) cudaFreeHost(h->h_res);
    if (h->h_small) cudaFreeHost(h->h_small);
    if (h->h_flag) cudaFreeHost(h->h_flag);
    if (h->h_state) cudaFreeHost(h->h_state);
    if (h->h_ref) cudaFreeHost(h->h_ref);
    if (h->h_cnt) cudaFreeHost(h->h_cnt);
    if (h->h_work) cudaFreeHost(h->h_work);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (auto& e : h->sw_ev)
        if (e) cudaEventDestroy(e);
}

int create_impl(int H, int W, int C, const uint8_t* mask, const float* values, const dd_params* params,
                dd_handle* out) {
    if (out == nullptr || mask == nullptr || values == nullptr) { set_error("NULL argument"); return DD_EINVAL; }
    *out = nullptr;
    dd_params p;
    if (params) p = *params; else dd_params_default(&p);
    DD_TRY(validate(H, W, C, p));
    if (!(p.robin_p > 0.f)) p.robin_p = robin_default(p.block, p.overlap);
    if (!p.inputs_on_device) {   // device masks are counted on the device by load_data
        long long nknown = 0;
        DD_TRY(count_known(mask, (size_t)H * W, false, &nknown));
        if (nknown == 0) { set_error("empty mask"); return DD_EEMPTYMASK; }
    }

    dd_inpaint* h = new (std::nothrow) dd_inpaint();
    if (!h) { set_error("host allocation"); return DD_ENOMEM; }
    h->H = H; h->W = W; h->C = C; h->prm = p;
    h->lowst = low_store(p.precision);
    auto fail = [&](int rc) { free_all(h); delete h; return rc; };
    int rc = DD_OK;
    // dyadic levels: (levels - 1) log2(coarse_factor) halvings, at most DD_MAX_LEVELS
    // levels in all, stopping once a dimension would fall below 2 pixels; the
    // solved levels are every log2(coarse_factor)-th one and the coarsest
    const int fstep = p.coarse_factor == 8 ? 3 : p.coarse_factor == 4 ? 2 : 1;
    int nl = std::min(DD_MAX_LEVELS, (p.levels - 1) * fstep + 1);
    {
        int hh = H, ww = W, l = 1;
        while (l < nl && hh > 2 && ww > 2) { hh = (hh + 1) / 2; ww = (ww + 1) / 2; ++l; }
        nl = l;
        h->nc = nl;
        // the small-grid coarse CG of the correction holds its level in shared memory:
        // correction-only levels continue the 2x2 restriction below the cascade's
        // coarsest level until one fits (no sweeps on them)
        if (p.ml_mode == DD_ML_CORRECTION && p.correction_cg > 0 && nl >= 2)
            while ((long long)hh * ww > dd::kCoarseCgMaxPixels && nl < DD_MAX_LEVELS && hh > 2 && ww > 2) {
                hh = (hh + 1) / 2; ww = (ww + 1) / 2; ++nl;
            }
    }
    h->lv.resize(nl);
    for (int l = 0; l < nl; ++l) h->lv[l].solved = l < h->nc && ((l % fstep == 0) || l == h->nc - 1);
    int hh = H, ww = W;
    for (int l = 0; l < nl; ++l) {
        Level& L = h->lv[l];
        L.H = hh; L.W = ww; L.P = round_up(ww, 32);
        L.geom = dd::make_geom(hh, ww, L.P, p.block, p.overlap, p.tile_warps);
        const size_t plane_bytes = (size_t)C * L.plane() * sizeof(float);
        if ((rc = dalloc_t(h, &L.mask, (size_t)hh * ww)) != DD_OK) return fail(rc);
        if ((rc = dalloc(h, (void**)&L.f, plane_bytes)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &L.tmask, dd::tmask_words(L.geom))) != DD_OK) return fail(rc);
        for (int b = 0; b < 2; ++b)
            if ((rc = dalloc(h, (void**)&L.u[b], plane_bytes)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &L.partial, (size_t)2 * C)) != DD_OK) return fail(rc);
        if ((rc = dzero(L.partial, sizeof(unsigned long long) * 2 * C)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &L.ref_d, (size_t)C)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &L.state_d, 4)) != DD_OK) return fail(rc);
        if (p.solver == DD_SOLVER_CG) {
            if ((rc = dalloc(h, (void**)&L.cg_r, plane_bytes)) != DD_OK) return fail(rc);
            for (int b = 0; b < 2; ++b)
                if ((rc = dalloc(h, (void**)&L.cg_p[b], plane_bytes)) != DD_OK) return fail(rc);
            if ((rc = dalloc(h, (void**)&L.cg_q, plane_bytes)) != DD_OK) return fail(rc);
            if ((rc = dalloc_t(h, &L.cg_part, (size_t)C * dd::cg_blocks(hh, ww))) != DD_OK) return fail(rc);
            if ((rc = dalloc_t(h, &L.cg_scal, (size_t)3 * C)) != DD_OK) return fail(rc);
        }
        hh = (hh + 1) / 2; ww = (ww + 1) / 2;
    }
    Level& F = h->lv[0];
    if (p.precision != DD_PREC_FP32) {
        const size_t n = (size_t)C * F.plane() * dd::store_bytes(h->lowst);
        for (int b = 0; b < 2; ++b)
            if ((rc = dalloc(h, &h->e[b], n)) != DD_OK) return fail(rc);
        if ((rc = dalloc(h, &h->g, n)) != DD_OK) return fail(rc);
    }
    for (auto& L : h->lv)
        for (int b = 0; b < 2; ++b)
            if (dd::make_tile_map(&L.map_u[b], Store::F32, L.u[b], L.H, L.W, L.P, C, p.block) != cudaSuccess) {
                set_error("cuTensorMapEncodeTiled failed");
                return fail(DD_ECUDA);
            }
    if (p.precision != DD_PREC_FP32) {
        for (int b = 0; b < 2; ++b)
            if (dd::make_tile_map(&h->map_e[b], h->lowst, h->e[b], F.H, F.W, F.P, C, p.block) != cudaSuccess) {
                set_error("cuTensorMapEncodeTiled failed");
                return fail(DD_ECUDA);
            }
        if (dd::make_tile_map(&h->map_g, h->lowst, h->g, F.H, F.W, F.P, C, p.block) != cudaSuccess) {
            set_error("cuTensorMapEncodeTiled failed");
            return fail(DD_ECUDA);
        }
    }
    if (corrects(h)) {   // coarse-grid correction buffers
        if (p.correction_cg > 0) {   // the small-grid CG holds the coarsest level in shared memory
            const Level& Lc = h->lv.back();
            if ((long long)Lc.H * Lc.W > dd::kCoarseCgMaxPixels) {
                set_error("correction_cg: no level of at most 12288 pixels within 8 dyadic levels");
                return fail(DD_EINVAL);
            }
            if (dd::prepare_coarse_cg() != cudaSuccess) {
                set_error("coarse CG: cudaFuncSetAttribute failed");
                return fail(DD_ECUDA);
            }
        }
        const size_t fb = sizeof(float) * (size_t)C * F.plane();
        if ((rc = dalloc(h, (void**)&h->corr_r, fb)) != DD_OK) return fail(rc);
        for (size_t l = 1; l < h->lv.size(); ++l) {
            Level& L = h->lv[l];
            if ((rc = dalloc(h, (void**)&L.corr_g, sizeof(float) * (size_t)C * L.plane())) != DD_OK) return fail(rc);
        }
        Level& Lc = h->lv.back();
        if (dd::make_tile_map(&Lc.map_cg, Store::F32, Lc.corr_g, Lc.H, Lc.W, Lc.P, C, p.block) != cudaSuccess) {
            set_error("cuTensorMapEncodeTiled failed");
            return fail(DD_ECUDA);
        }
        if ((rc = alloc_flag(h, &h->flag_c)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &h->state_c, 4)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &h->norms2_c, (size_t)2 * C + 2)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &h->tol_c, 1)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &h->corr_dots, (size_t)3 * C)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &h->corr_gate, kGateWords)) != DD_OK) return fail(rc);
        if ((rc = dalloc_t(h, &h->corr_prev, 2)) != DD_OK) return fail(rc);
    }
    h->res_nblk = dd::res64_blocks(H, W);
    // block partials: the residual passes (C x res_nblk double2) and the
    // reference norms of all levels (C x their blocks, doubles)
    h->res_part_n = std::max(h->res_nblk, dd::ref_norm_part_words(H, W, (int)h->lv.size()));
    if ((rc = dalloc_t(h, &h->res_part, (size_t)C * h->res_part_n)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->res_out, (size_t)C * DD_MAX_LEVELS)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->norms2_d, (size_t)2 * C + 2)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->sstate_d, 4)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->inner_ref_d, (size_t)C)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->ones_d, (size_t)C)) != DD_OK) return fail(rc);
    {
        std::vector<double> ones(C, 1.0);
        if (cudaMemcpy(h->ones_d, ones.data(), sizeof(double) * C, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("cudaMemcpy");
            return fail(DD_ECUDA);
        }
    }
    if ((rc = dalloc_t(h, &h->scale_d, (size_t)C)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->scale_inv_d, (size_t)C)) != DD_OK) return fail(rc);
    if ((rc = alloc_flag(h, &h->flag_d)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->ctl_d, 4)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->tol_d, 1)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->res_ticket, 1)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->work_d, kWorkWords)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->ref_ctl_d, 4 + dd::kFlagWords)) != DD_OK) return fail(rc);
    if ((rc = dalloc_t(h, &h->ref_tol_d, 1)) != DD_OK) return fail(rc);
    if (cudaMallocHost(&h->h_ref_ctl, 8 * sizeof(int)) != cudaSuccess) {
        set_error("cudaMallocHost failed");
        return fail(DD_ENOMEM);
    }
    if (cudaMallocHost(&h->h_work, kWorkWords * sizeof(unsigned long long)) != cudaSuccess) {
        set_error("cudaMallocHost failed");
        return fail(DD_ENOMEM);
    }
    if (cudaMemset(h->res_ticket, 0, sizeof(unsigned int)) != cudaSuccess) {
        set_error("cudaMemset");
        return fail(DD_ECUDA);
    }
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("cudaStreamCreateWithFlags failed");
        return fail(DD_ECUDA);
    }
    if (cudaMallocHost(&h->h_res, sizeof(double2) * C * DD_MAX_LEVELS) != cudaSuccess ||
        cudaMallocHost(&h->h_state, sizeof(int) * 4 * DD_MAX_LEVELS) != cudaSuccess ||
        cudaMallocHost(&h->h_ref, sizeof(double) * C) != cudaSuccess ||
        cudaMallocHost(&h->h_cnt, sizeof(unsigned long long) * 2) != cudaSuccess ||
        cudaMallocHost(&h->h_small, sizeof(double) * 3 * C) != cudaSuccess ||
        cudaMallocHost(&h->h_flag, sizeof(int) * 8) != cudaSuccess) {
        set_error("cudaMallocHost failed");
        return fail(DD_ENOMEM);
    }
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
        set_error("cudaEventCreate failed");
        return fail(DD_ECUDA);
    }
    for (auto& e : h->sw_ev)
        if (cudaEventCreate(&e) != cudaSuccess) { set_error("cudaEventCreate failed"); return fail(DD_ECUDA); }
    if ((rc = dalloc_t(h, &h->count_d, 2)) != DD_OK) return fail(rc);
    cudaStream_t st = nullptr;
    if ((rc = load_data(h, mask, values, st)) != DD_OK) return fail(rc);
    h->valid = true;
    if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("sync"); return fail(DD_ECUDA); }
    // the device loops of every level, instantiated now rather than in the first solve
    // (with FP32_REF / FP16_REF / BF16_REF the fine level sweeps under host control)
    if (p.device_loop != 0) {
        for (size_t l = 0; l < h->lv.size(); ++l) {
            if ((l == 0 && p.precision != DD_PREC_FP32) || !h->lv[l].solved) continue;
            cudaGraphExec_t ex = nullptr;
            if ((rc = loop_graph(h, h->lv[l], l == 0 ? p.max_sweeps : p.coarse_sweeps, &ex)) != DD_OK) return fail(rc);
        }
        if (p.precision != DD_PREC_FP32) {   // the correction loop with its nested inner loop
            cudaGraphExec_t ex = nullptr;
            if ((rc = ref_graph(h, &ex)) != DD_OK) return fail(rc);
        }
    }
    *out = h;
    return DD_OK;
}

}  // namespace

// Internal helpers shared with other translation units (dd_internal.h).
namespace dd {
float default_robin(int b, int o) { return robin_default(b, o); }
void set_last_error(const char* msg) { set_error(msg ? msg : ""); }
}  // namespace dd

// ------------------------------------------------------------------ C ABI
extern "C" {

void dd_params_default(dd_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->block = 32;
    p->overlap = 6;
    p->local_cg_iters = 16;
    p->levels = 3;
    p->ml_mode = DD_ML_CASCADE;
    p->coarse_factor = 2;
    p->robin_p = 0.f;
    p->precision = DD_PREC_FP32_REF;
    p->max_sweeps = 400;
    p->inputs_on_device = 0;
    p->coarse_tol = 1e-2;
    p->inner_tol = 3e-3;
    p->max_corrections = 30;
    p->coarse_sweeps = 12;
    p->timing = 0;
    p->tile_warps = 0;
    p->solver = DD_SOLVER_ORAS;
    p->device_loop = 1;
    p->correction_sweeps = 2;
    p->local_rtol = 0.0;
    p->correction_trigger = 0.0;
    p->final_local_rtol = 0.0;
    p->correction_cg = 0;
    p->local_atol = 0.0;
}

const char* dd_strerror(int code) {
    switch (code) {
        case DD_OK: return "ok";
        case DD_EINVAL: return "invalid argument";
        case DD_EEMPTYMASK: return "empty mask (A is singular)";
        case DD_ENOMEM: return "out of memory";
        case DD_ENOTCONVERGED: return "not converged within the sweep limit";
        case DD_ENUMERIC: return "non-finite residual";
        case DD_ECUDA: return "CUDA error";
        case DD_ETIMEOUT: return "device wait timed out";
        case DD_EAGAIN: return "not finished yet";
    }
    return "unknown error";
}

const char* dd_last_error(void) { return g_last_error.c_str(); }

void dd_set_device_budget(size_t bytes) { g_budget.store((unsigned long long)bytes); }

size_t dd_device_bytes_in_use(void) { return (size_t)g_bytes_in_use.load(); }

int dd_inpaint_create(int H, int W, int C, const uint8_t* mask, const float* values, const dd_params* params,
                      dd_handle* out) {
    return create_impl(H, W, C, mask, values, params, out);
}

int dd_inpaint_solve(dd_handle h, float* u_out, double tol, void* stream) {
    if (!h || !u_out || !(tol > 0.0)) { set_error("bad solve arguments"); return DD_EINVAL; }
    if (!h->valid) { set_error("no valid data (the last set_data failed)"); return DD_EEMPTYMASK; }
    return solve_impl(h, u_out, tol, static_cast<cudaStream_t>(stream));
}

int dd_inpaint_destroy(dd_handle h) {
    if (!h) return DD_OK;
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return DD_OK;
}

int dd_inpaint_set_data(dd_handle h, const uint8_t* mask, const float* values, int keep_iterate) {
    if (!h || !mask || !values) { set_error("NULL argument"); return DD_EINVAL; }
    if (!h->prm.inputs_on_device) {
        long long nknown = 0;
        DD_TRY(count_known(mask, (size_t)h->H * h->W, false, &nknown));
        if (nknown == 0) { set_error("empty mask"); return DD_EEMPTYMASK; }
    }
    cudaStream_t st = nullptr;
    Level& F = h->lv[0];
    // keep the fine iterate in buffer 0 (load_data stages values through u[1])
    if (keep_iterate && h->cur != 0)
        DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.u[1], F.P, F.plane(), F.u[0], F.P, F.plane(), st));
    h->cur = 0;
    h->valid = false;
    DD_TRY(load_data(h, mask, values, st));
    h->valid = true;
    if (keep_iterate) {
        DD_LAUNCH(h, dd::launch_reset_known(F.H, F.W, h->C, F.u[0], F.P, F.plane(), F.mask, F.W, F.f, F.P, F.plane(),
                                            st));
        h->warm = true;
    } else {
        h->warm = false;
    }
    DD_CK(cudaStreamSynchronize(st));
    return DD_OK;
}

int dd_inpaint_stats(dd_handle h, dd_stats* out) {
    if (!h || !out) { set_error("NULL argument"); return DD_EINVAL; }
    *out = h->stats;
    out->device_bytes = h->bytes;   // valid from create on, before any solve
    out->channels = h->C;
    return DD_OK;
}

int dd_inpaint_set_data_async(dd_handle h, const uint8_t* mask, const float* values, int keep_iterate,
                              void* stream) {
    if (!h || !mask || !values) { set_error("NULL argument"); return DD_EINVAL; }
    if (h->pending) { set_error("a solve is in flight: finish it first"); return DD_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Level& F = h->lv[0];
    if (keep_iterate && h->cur != 0)
        DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.u[1], F.P, F.plane(), F.u[0], F.P, F.plane(), st));
    h->cur = 0;
    h->valid = true;   // the empty-mask test is done when the next solve finishes
    DD_TRY(load_data(h, mask, values, st, false));
    if (keep_iterate)
        DD_LAUNCH(h, dd::launch_reset_known(F.H, F.W, h->C, F.u[0], F.P, F.plane(), F.mask, F.W, F.f, F.P,
                                            F.plane(), st));
    h->warm = keep_iterate != 0;
    return DD_OK;
}

int dd_inpaint_solve_async(dd_handle h, float* u_out, double tol, void* stream) {
    if (!h || !u_out || !(tol > 0.0)) { set_error("bad solve arguments"); return DD_EINVAL; }
    if (h->prm.precision != DD_PREC_FP32 && !device_ref(h)) {
        set_error("asynchronous correction-mode solves need device_loop = 1");
        return DD_EINVAL;
    }
    if (h->pending) { set_error("a solve is already in flight"); return DD_EINVAL; }
    if (!h->valid) { set_error("no valid data (the last set_data failed)"); return DD_EEMPTYMASK; }
    return enqueue_solve(h, u_out, tol, static_cast<cudaStream_t>(stream), false);
}

int dd_inpaint_query(dd_handle h) {
    if (!h || !h->pending) { set_error("no solve in flight"); return DD_EINVAL; }
    if (!h->ev_recorded) return DD_EAGAIN;
    const cudaError_t e = cudaEventQuery(h->ev1);
    if (e == cudaSuccess) return DD_OK;
    if (e == cudaErrorNotReady) return DD_EAGAIN;
    set_error(std::string("cudaEventQuery: ") + cudaGetErrorString(e));
    return DD_ECUDA;
}

int dd_inpaint_solve_finish(dd_handle h, void* stream) {
    if (!h) { set_error("NULL argument"); return DD_EINVAL; }
    return finish_solve(h, static_cast<cudaStream_t>(stream));
}

int dd_inpaint_set_iterate(dd_handle h, const float* u, void* stream) {
    if (!h || !u) { set_error("NULL argument"); return DD_EINVAL; }
    Level& F = h->lv[0];
    h->cur = 0;
    DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, u, F.W, (long long)F.H * F.W, F.u[0], F.P, F.plane(),
                            static_cast<cudaStream_t>(stream)));
    h->warm = true;
    return DD_OK;
}

int dd_inpaint_get_iterate(dd_handle h, float* u_out, void* stream) {
    if (!h || !u_out) { set_error("NULL argument"); return DD_EINVAL; }
    Level& F = h->lv[0];
    DD_LAUNCH(h, dd::launch_copy2d(F.H, F.W, h->C, F.u[h->cur], F.P, F.plane(), u_out, F.W, (long long)F.H * F.W,
                            static_cast<cudaStream_t>(stream)));
    return DD_OK;
}

int dd_inpaint_sweep(dd_handle h, int n, double* rnorm_out, void* stream) {
    if (!h || n < 0) { set_error("bad sweep arguments"); return DD_EINVAL; }
    if (h->prm.solver != DD_SOLVER_ORAS) { set_error("dd_inpaint_sweep needs DD_SOLVER_ORAS"); return DD_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Level& F = h->lv[0];
    DD_LAUNCH(h, dd::launch_reset_sweep_state(h->sstate_d, h->flag_d, h->cur, h->tol_d, -1.0, st));
    DD_TRY(clear_error(h, st));
    const dd::SweepPair pair{{&F.map_u[0], &F.map_u[1]}, {F.u[0], F.u[1]}};
    const dd::SweepStop stop = make_stop(h, F.partial, F.ref_d, 0.0);
    if (corrects(h)) DD_TRY(reset_correction(h, st));
    for (int i = 0; i < n; ++i) {   // tol < 0: every launch is a full sweep
        DD_LAUNCH(h, dd::launch_sweep(Store::F32, F.geom, h->C, F.plane(), pair, nullptr, F.tmask, stop,
                                      h->prm.robin_p, h->prm.local_cg_iters, st, (float)h->prm.local_rtol));
        if (corrects(h)) {   // one pass of DD_ML_CORRECTION: the sweep, then the coarse-grid correction
            DD_TRY(enqueue_correction(h, st));
            h->launches += 1 + correction_kernels(h);
        }
        h->cur = 1 - h->cur;
    }
    if (n > 0) {
        int err = 0;
        DD_CK(cudaMemcpyAsync(&err, err_word(h), sizeof(int), cudaMemcpyDeviceToHost, st));
        DD_CK(cudaStreamSynchronize(st));
        if (err != 0) { set_error("a bounded device wait for a staged tile gave up"); return DD_ETIMEOUT; }
    }
    if (rnorm_out != nullptr && n > 0) {
        std::vector<double> tmp(h->C);
        DD_CK(cudaMemcpyAsync(tmp.data(), h->norms2_d, sizeof(double) * h->C, cudaMemcpyDeviceToHost, st));
        DD_CK(cudaStreamSynchronize(st));
        for (int c = 0; c < h->C; ++c) rnorm_out[c] = std::sqrt(tmp[c]);
    }
    return DD_OK;
}

int dd_restrict(int H, int W, int C, const uint8_t* mask, const float* f, uint8_t* mask_c, float* f_c,
                void* stream) {
    if (H <= 0 || W <= 0 || C <= 0 || !mask || !f || !mask_c || !f_c) { set_error("bad arguments"); return DD_EINVAL; }
    const int Hc = (H + 1) / 2, Wc = (W + 1) / 2;
    DD_CK(dd::launch_restrict(H, W, C, mask, W, f, W, (long long)H * W, mask_c, Wc, f_c, Wc, (long long)Hc * Wc,
                              static_cast<cudaStream_t>(stream)));
    return DD_OK;
}

int dd_prolong(int Hc, int Wc, int H, int W, int C, const float* u_c, const uint8_t* mask, const float* f,
               float* u, void* stream) {
    if (Hc <= 0 || Wc <= 0 || H <= 0 || W <= 0 || C <= 0 || !u_c || !u || ((mask == nullptr) != (f == nullptr))) {
        set_error("bad arguments");
        return DD_EINVAL;
    }
    DD_CK(dd::launch_prolong(Hc, Wc, H, W, C, u_c, Wc, (long long)Hc * Wc, mask, W, f, W, (long long)H * W, u, W,
                             (long long)H * W, static_cast<cudaStream_t>(stream)));
    return DD_OK;
}

int dd_coarse_cg(int H, int W, int C, const uint8_t* mask, const float* g, float* e, int max_iter, double tol,
                 int* iters, void* stream) {
    if (H <= 0 || W <= 0 || C <= 0 || !mask || !g || !e || max_iter < 0 || !(tol >= 0.0)) {
        set_error("bad arguments");
        return DD_EINVAL;
    }
    if ((long long)H * W > dd::kCoarseCgMaxPixels) {
        set_error("dd_coarse_cg: more than 12288 pixels");
        return DD_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DD_CK(dd::prepare_coarse_cg());
    int* it_d = nullptr;
    if (iters != nullptr) DD_CK(cudaMallocAsync(reinterpret_cast<void**>(&it_d), sizeof(int) * C, st));
    const long long plane = (long long)H * W;
    const cudaError_t e1 = dd::launch_coarse_cg(H, W, C, mask, W, g, W, plane, e, W, plane, max_iter, tol, it_d,
                                                nullptr, st);
    cudaError_t e2 = cudaSuccess;
    if (it_d != nullptr) {
        if (e1 == cudaSuccess) e2 = cudaMemcpyAsync(iters, it_d, sizeof(int) * C, cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(it_d, st);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    }
    DD_CK(e1);
    DD_CK(e2);
    return DD_OK;
}

int dd_residual_norms(int H, int W, int C, const uint8_t* mask, const float* f, const float* u, double* norms,
                      double* ref_norms, void* stream) {
    if (H <= 0 || W <= 0 || C <= 0 || !mask || !f || !u) { set_error("bad arguments"); return DD_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nblk = dd::res64_blocks(H, W);
    double2* part = nullptr;
    double2* outd = nullptr;
    unsigned int* ticket = nullptr;
    float* u0 = nullptr;
    std::vector<double2> hout(C);
    auto cleanup = [&]() {
        if (part) cudaFree(part);
        if (outd) cudaFree(outd);
        if (ticket) cudaFree(ticket);
        if (u0) cudaFree(u0);
    };
    if (cudaMalloc(&part, sizeof(double2) * nblk * C) != cudaSuccess ||
        cudaMalloc(&outd, sizeof(double2) * C) != cudaSuccess ||
        cudaMalloc(&ticket, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&u0, sizeof(float) * (size_t)C * H * W) != cudaSuccess) {
        cleanup();
        set_error("cudaMalloc failed");
        return DD_ENOMEM;
    }
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st) != cudaSuccess) {   // the passes leave it zero
        cleanup();
        set_error("cudaMemsetAsync failed");
        return DD_ECUDA;
    }
    for (int pass = 0; pass < 2; ++pass) {
        double* dst = pass == 0 ? norms : ref_norms;
        if (!dst) continue;
        const float* src = u;
        if (pass == 1) {
            if (dd::launch_masked_copy(H, W, C, f, W, (long long)H * W, mask, W, u0, W, (long long)H * W, st) !=
                cudaSuccess) { cleanup(); set_error("launch"); return DD_ECUDA; }
            src = u0;
        }
        dd::Res64Args a{};
        a.H = H; a.W = W; a.C = C; a.u = src; a.up = W; a.uplane = (long long)H * W;
        a.mask = mask; a.mp = W; a.g_out = nullptr; a.gst = Store::F32; a.part = part; a.nblk = nblk;
        a.out = outd; a.ticket = ticket;
        if (dd::launch_res64(a, st) != cudaSuccess ||
            cudaMemcpyAsync(hout.data(), outd, sizeof(double2) * C, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cleanup();
            set_error("residual pass failed");
            return DD_ECUDA;
        }
        for (int c = 0; c < C; ++c) dst[c] = std::sqrt(hout[c].x);
    }
    cleanup();
    return DD_OK;
}

// ------------------------------------------------------------------ batches
struct dd_batch {
    std::vector<dd_handle> hs;
    std::vector<float*> outs;
    double tol = 0.0;
    int mode = DD_BATCH_GRAPH;
    cudaStream_t cap = nullptr;
    cudaStream_t body = nullptr;            // private stream on which batched loop bodies are captured
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> evs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    long long kernels = 0;
    bool launched = false;
    // DD_BATCH_PERSISTENT: per dyadic level (0 = finest) the descriptors of the
    // frames that sweep there, the handles they belong to, and the batch's list
    // and control words
    std::vector<dd::SweepFrame*> frames_d;
    std::vector<std::vector<int>> members;
    std::vector<int> max_cap;
    int* list_d = nullptr;                  // dd::kBatchListWords ints
    int* bctl_d = nullptr;                  // [0, 3) launch ticket, tile counter, failed wait; [4, 8) loop passes
    TileGeom geom;                          // the block layout shared by all frames
};

static void batch_free(dd_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->evs) cudaEventDestroy(e);
    for (auto s2 : b->side) cudaStreamDestroy(s2);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->body) cudaStreamDestroy(b->body);
    if (b->done) cudaEventDestroy(b->done);
    for (auto p : b->frames_d)
        if (p) cudaFree(p);
    if (b->list_d) cudaFree(b->list_d);
    if (b->bctl_d) cudaFree(b->bctl_d);
    delete b;
}

namespace {

// Persistent batches: the frames' requirements (FP32 ORAS cascade with device
// loops and one block layout) and their per-level sweep descriptors.
int batch_check_persistent(const std::vector<dd_handle>& hs) {
    const dd_params& p0 = hs[0]->prm;
    for (auto h : hs) {
        const dd_params& p = h->prm;
        if (p.precision != DD_PREC_FP32 || p.solver != DD_SOLVER_ORAS || p.ml_mode != DD_ML_CASCADE ||
            p.device_loop != 1 || p.timing != 0) {
            set_error("a persistent batch needs FP32 ORAS cascade handles with device loops and no timing");
            return DD_EINVAL;
        }
        if (p.block != p0.block || p.overlap != p0.overlap || h->lv[0].geom.nw != hs[0]->lv[0].geom.nw) {
            set_error("the handles of a persistent batch need the same block, overlap and tile warps");
            return DD_EINVAL;
        }
    }
    if ((int)hs.size() > dd::kBatchMaxFrames) { set_error("too many frames for one persistent batch"); return DD_EINVAL; }
    return DD_OK;
}

int batch_build_frames(dd_batch* b) {
    int nlev = 0;
    for (auto h : b->hs) nlev = std::max(nlev, (int)h->lv.size());
    b->frames_d.assign(nlev, nullptr);
    b->members.assign(nlev, {});
    b->max_cap.assign(nlev, 0);
    for (int l = 0; l < nlev; ++l) {
        std::vector<dd::SweepFrame> host;
        for (int i = 0; i < (int)b->hs.size(); ++i) {
            dd_handle h = b->hs[i];
            if (l >= (int)h->lv.size() || !h->lv[l].solved) continue;
            Level& L = h->lv[l];
            const int cap = l == 0 ? h->prm.max_sweeps : h->prm.coarse_sweeps;
            const dd::SweepPair pair{{&L.map_u[0], &L.map_u[1]}, {L.u[0], L.u[1]}};
            dd::SweepFrame f;
            dd::fill_sweep_frame(&f, L.geom, h->C, L.plane(), pair, L.tmask, make_stop(h, L.partial, L.ref_d, 0.0),
                                 h->prm.robin_p, h->prm.local_cg_iters, (float)h->prm.local_rtol, cap, L.state_d);
            if (f.flag == nullptr) { set_error("batch: bad sweep descriptor"); return DD_EINVAL; }
            f.level_tol = l == 0 ? b->tol : h->prm.coarse_tol;
            host.push_back(f);
            b->members[l].push_back(i);
            b->max_cap[l] = std::max(b->max_cap[l], cap);
        }
        if (host.empty()) continue;
        DD_CK(cudaMalloc(&b->frames_d[l], sizeof(dd::SweepFrame) * host.size()));
        DD_CK(cudaMemcpy(b->frames_d[l], host.data(), sizeof(dd::SweepFrame) * host.size(), cudaMemcpyHostToDevice));
    }
    DD_CK(cudaMalloc(&b->list_d, sizeof(int) * dd::kBatchListWords));
    DD_CK(cudaMemset(b->list_d, 0, sizeof(int) * dd::kBatchListWords));
    DD_CK(cudaMalloc(&b->bctl_d, sizeof(int) * 8));
    DD_CK(cudaMemset(b->bctl_d, 0, sizeof(int) * 8));
    b->geom = b->hs[0]->lv[0].geom;
    DD_CK(dd::prepare_sweep_batch(b->geom));
    return DD_OK;
}

// The batched loop of level l, appended to the graph being captured on st: an
// entry kernel (pass counter 0, condition 1), then a WHILE node whose body is
// the loop control (the list of the frames whose sequences run; condition
// cleared when none does) followed by one batched sweep of those frames.
int batch_add_loop(dd_batch* b, int l, cudaStream_t st) {
    const int n = (int)b->members[l].size();
    const int max_passes = 2 * b->max_cap[l] + 3;
    int* const ctl = b->bctl_d + 4;
    return capture_append(st, [&](cudaGraph_t g, const cudaGraphNode_t* deps, const cudaGraphEdgeData* edges,
                                  size_t ndeps, cudaGraphNode_t* last) -> int {
        cudaGraphConditionalHandle cond;
        DD_CK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
        int* ctl_arg = ctl;
        void* kargs[2] = {&ctl_arg, &cond};
        cudaGraphNodeParams kp{};
        kp.type = cudaGraphNodeTypeKernel;
        kp.kernel.func = const_cast<void*>(dd::loop_begin_kernel_fn());
        kp.kernel.gridDim = dim3(1, 1, 1);
        kp.kernel.blockDim = dim3(32, 1, 1);
        kp.kernel.kernelParams = kargs;
        cudaGraphNode_t entry = nullptr, loop = nullptr;
        DD_CK(cudaGraphAddNode(&entry, g, deps, edges, ndeps, &kp));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        DD_CK(cudaGraphAddNode(&loop, g, &entry, nullptr, 1, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        DD_CK(cudaStreamBeginCaptureToGraph(b->body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = dd::launch_batch_ctl(b->frames_d[l], n, b->list_d, ctl, max_passes, cond, b->body);
        cudaError_t e2 = e1 == cudaSuccess ? dd::launch_sweep_batch(b->geom, b->frames_d[l], b->list_d, b->bctl_d,
                                                                    b->body)
                                           : cudaSuccess;
        cudaGraph_t captured = body;
        const cudaError_t ec = cudaStreamEndCapture(b->body, &captured);
        DD_CK(e1);
        DD_CK(e2);
        DD_CK(ec);
        *last = loop;
        return DD_OK;
    });
}

// Fork from cap onto the side streams of the frames in idx, run per(i, stream)
// on each, join back into cap.
int batch_fork(dd_batch* b, const std::vector<int>& idx, const std::function<int(int, cudaStream_t)>& per) {
    const int n = (int)b->hs.size();
    DD_CK(cudaEventRecord(b->evs[2 * n], b->cap));
    for (int i : idx) {
        DD_CK(cudaStreamWaitEvent(b->side[i], b->evs[2 * n], 0));
        DD_TRY(per(i, b->side[i]));
        DD_CK(cudaEventRecord(b->evs[2 * i], b->side[i]));
        DD_CK(cudaStreamWaitEvent(b->cap, b->evs[2 * i], 0));
    }
    return DD_OK;
}

// The whole batch on the capturing stream b->cap: per frame the coarsest
// level's start; then, level by level from the coarsest, each frame's start
// prolonged from the level below it (side streams), and one batched device
// loop of sweeps over all frames that solve on the level; finally each frame's
// output, FP64-accurate residual and read-back (side streams).
int batch_enqueue_persistent(dd_batch* b) {
    const int n = (int)b->hs.size();
    const int nlev = (int)b->frames_d.size();
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    DD_TRY(batch_fork(b, all, [&](int i, cudaStream_t st) -> int {
        dd_handle h = b->hs[i];
        std::memset(&h->stats, 0, sizeof(h->stats));
        h->stats.channels = h->C;
        h->stats.device_bytes = h->bytes;
        h->ev_recorded = false;
        h->warm = false;
        h->pending_cascaded = true;
        DD_TRY(clear_error(h, st));
        Level& Lc = h->lv.back();
        DD_LAUNCH(h, dd::launch_copy2d(Lc.H, Lc.W, h->C, Lc.f, Lc.P, Lc.plane(), Lc.u[0], Lc.P, Lc.plane(), st));
        return DD_OK;
    }));
    for (int l = nlev - 1; l >= 0; --l) {
        // starts of level l prolonged from level l + 1; pass-through levels record buffer 0
        std::vector<int> idx;
        for (int i = 0; i < n; ++i) {
            const int nli = (int)b->hs[i]->lv.size();   // frames with fewer levels join at their coarsest
            if (l < nli - 1 || (l < nli && !b->hs[i]->lv[l].solved)) idx.push_back(i);
        }
        if (!idx.empty())
            DD_TRY(batch_fork(b, idx, [&](int i, cudaStream_t st) -> int {
                dd_handle h = b->hs[i];
                Level& L = h->lv[l];
                if (l < (int)h->lv.size() - 1) {
                    Level& Cc = h->lv[l + 1];
                    DD_LAUNCH(h, dd::launch_prolong_sel(Cc.H, Cc.W, L.H, L.W, h->C, Cc.u[0], Cc.u[1], Cc.state_d,
                                                        Cc.P, Cc.plane(), L.mask, L.W, L.f, L.P, L.plane(), L.u[0],
                                                        L.P, L.plane(), st));
                }
                if (!L.solved) DD_CK(cudaMemsetAsync(L.state_d, 0, 4 * sizeof(int), st));
                return DD_OK;
            }));
        const int nf = (int)b->members[l].size();
        if (nf == 0) continue;
        DD_CK(dd::launch_batch_reset(b->frames_d[l], nf, b->cap));
        DD_TRY(batch_add_loop(b, l, b->cap));
        DD_CK(dd::launch_batch_resolve(b->frames_d[l], nf, b->bctl_d + 4, b->cap));
        b->kernels += 3;
    }
    return batch_fork(b, all, [&](int i, cudaStream_t st) -> int {
        dd_handle h = b->hs[i];
        for (Level& L : h->lv) L.loop_pending = false;   // batched loops are counted by the batch
        return enqueue_output_readback(h, b->outs[i], b->tol, st, true, false);
    });
}

}  // namespace

int dd_batch_create_mode(int n, const dd_handle* handles, float* const* u_out, double tol, int mode,
                         dd_batch_handle* out, long long* kernels_per_launch) {
    if (n <= 0 || !handles || !u_out || !out || !(tol > 0.0)) { set_error("bad batch arguments"); return DD_EINVAL; }
    if (mode != DD_BATCH_GRAPH && mode != DD_BATCH_PERSISTENT) { set_error("bad batch mode"); return DD_EINVAL; }
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!handles[i] || !u_out[i]) { set_error("NULL handle or output"); return DD_EINVAL; }
        if (handles[i]->prm.precision != DD_PREC_FP32 && !device_ref(handles[i])) {
            set_error("batches of correction-mode handles need device_loop = 1");
            return DD_EINVAL;
        }
        if (handles[i]->pending) { set_error("a handle has a solve in flight"); return DD_EINVAL; }
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) { set_error("a handle appears twice"); return DD_EINVAL; }
    }
    std::vector<dd_handle> hs(handles, handles + n);
    if (mode == DD_BATCH_PERSISTENT) DD_TRY(batch_check_persistent(hs));
    dd_batch* b = new (std::nothrow) dd_batch();
    if (!b) { set_error("host allocation"); return DD_ENOMEM; }
    b->hs = hs;
    b->outs.assign(u_out, u_out + n);
    b->tol = tol;
    b->mode = mode;
    auto bail = [&](const char* what, cudaError_t e) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        batch_free(b);
        return DD_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream", e);
    if ((e = cudaStreamCreateWithFlags(&b->body, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream", e);
    if ((e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess) return bail("event", e);
    b->side.resize(n, nullptr);
    b->evs.resize(2 * n + 1, nullptr);
    for (int i = 0; i < n; ++i)
        if ((e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking)) != cudaSuccess)
            return bail("stream", e);
    for (auto& ev : b->evs)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return bail("event", e);
    if (mode == DD_BATCH_PERSISTENT) {
        const int rcf = batch_build_frames(b);
        if (rcf != DD_OK) { batch_free(b); return rcf; }
    }
    long long before = 0;
    for (auto h : b->hs) before += h->launches;
    if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail("capture", e);
    int rc = DD_OK;
    if (mode == DD_BATCH_PERSISTENT) {
        rc = batch_enqueue_persistent(b);
        for (auto h : b->hs) h->pending = false;
    } else {
        // fork one stream per frame, enqueue each frame's solve, join
        if ((e = cudaEventRecord(b->evs[2 * n], b->cap)) != cudaSuccess) rc = DD_ECUDA;
        for (int i = 0; i < n && rc == DD_OK; ++i) {
            if (cudaStreamWaitEvent(b->side[i], b->evs[2 * n], 0) != cudaSuccess) { rc = DD_ECUDA; break; }
            b->hs[i]->warm = false;   // a captured solve always starts with the cascade
            rc = enqueue_solve(b->hs[i], b->outs[i], tol, b->side[i], true);
            b->hs[i]->pending = false;
            if (rc == DD_OK && cudaEventRecord(b->evs[2 * i], b->side[i]) != cudaSuccess) rc = DD_ECUDA;
            if (rc == DD_OK && cudaStreamWaitEvent(b->cap, b->evs[2 * i], 0) != cudaSuccess) rc = DD_ECUDA;
        }
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    b->graph = g;
    if (rc != DD_OK || e != cudaSuccess) {
        if (rc == DD_OK) set_error(std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        batch_free(b);
        return rc == DD_OK ? DD_ECUDA : rc;
    }
    {
        cudaGraphInstantiateParams ip{};
        ip.flags = 0;
        if ((e = cudaGraphInstantiateWithParams(&b->exec, b->graph, &ip)) != cudaSuccess) {
            cudaGraphNodeType t = cudaGraphNodeTypeEmpty;
            if (ip.errNode_out) cudaGraphNodeGetType(ip.errNode_out, &t);
            set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e) + " (result " +
                      std::to_string((int)ip.result_out) + ", node type " + std::to_string((int)t) + ")");
            batch_free(b);
            return DD_ECUDA;
        }
    }
    long long after = 0;
    for (auto h : b->hs) {
        after += h->launches;
        for (Level& L : h->lv) L.loop_pending = false;   // captured, not run
    }
    b->kernels += after - before;
    if (kernels_per_launch) *kernels_per_launch = b->kernels;
    *out = b;
    return DD_OK;
}

int dd_batch_create(int n, const dd_handle* handles, float* const* u_out, double tol, dd_batch_handle* out,
                    long long* kernels_per_launch) {
    return dd_batch_create_mode(n, handles, u_out, tol, DD_BATCH_GRAPH, out, kernels_per_launch);
}

int dd_batch_launch(dd_batch_handle b, void* stream) {
    if (!b) { set_error("NULL batch"); return DD_EINVAL; }
    if (b->launched) { set_error("the previous launch has not been finished"); return DD_EINVAL; }
    for (size_t i = 0; i < b->hs.size(); ++i) {
        dd_handle h = b->hs[i];
        if (h->pending) { set_error("a handle of the batch has a solve in flight"); return DD_EINVAL; }
        if (!h->valid) { set_error("a handle of the batch has no valid data"); return DD_EEMPTYMASK; }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DD_CK(cudaGraphLaunch(b->exec, st));
    DD_CK(cudaEventRecord(b->done, st));
    for (size_t i = 0; i < b->hs.size(); ++i) {
        dd_handle h = b->hs[i];
        h->pending = true;
        h->pending_out = b->outs[i];
        h->pending_tol = b->tol;
        h->pending_cascaded = true;
        h->ev_recorded = false;
        h->warm = false;
        for (Level& L : h->lv) L.loop_pending = h->prm.device_loop != 0;   // passes counted at finish
    }
    b->launched = true;
    return DD_OK;
}

int dd_batch_finish(dd_batch_handle b, void* stream, int* status) {
    if (!b || !b->launched) { set_error("no batch launch in flight"); return DD_EINVAL; }
    b->launched = false;
    DD_CK(cudaEventSynchronize(b->done));
    int worst = DD_OK;
    for (size_t i = 0; i < b->hs.size(); ++i) {
        const int rc = finish_solve(b->hs[i], static_cast<cudaStream_t>(stream));
        if (status) status[i] = rc;
        if (rc != DD_OK && worst == DD_OK) worst = rc;
    }
    return worst;
}

int dd_batch_destroy(dd_batch_handle b) {
    if (!b) return DD_OK;
    if (b->launched) cudaEventSynchronize(b->done);
    for (auto h : b->hs) h->pending = false;
    batch_free(b);
    return DD_OK;
}

}  // extern "C"
