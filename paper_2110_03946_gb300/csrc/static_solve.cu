// dd_inpaint_solve_static: a one-level FP32 ORAS solve that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running where the allocator is
// owned by someone else (a host framework with its own caching pool, a
// plug-in that must not grow the process's device footprint), code that is
// only allowed to touch memory it was handed, and real-time paths where an
// allocation's latency or failure is not acceptable.  This entry point gives
// them the same sweep kernels as dd_inpaint_solve, with all scratch (the two
// pitched iterate buffers, block masks, per-block residual partials, residual
// partials of the FP64 check, norms and flags) carved from one file-scope
// device array of fixed size.  The caller still passes inputs and the output.
//
// Properties a caller must know:
//  * the array (kScratchBytes, about 42 MiB) is committed on a device when the
//    library's module is loaded there; with CUDA's default lazy module loading
//    that is the first call on that device (its cudaGetSymbolAddress), which can
//    then fail with DD_ECUDA when device memory is short and pays the load
//    latency, so a real-time caller makes one warm-up call at start-up; the
//    array stays until the process exits;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (once per device, with that device current); make
//    that first call before any stream capture;
//  * every call uses the same array, which keeps the previous call's contents;
//    calls whose GPU work overlaps (other streams, other host threads) race
//    and give wrong results: serialise them;
//  * sizes beyond the capacity are rejected with DD_EINVAL before any GPU work.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/dd_inpaint.h"
#include "dd_internal.h"

namespace {

constexpr long long kMaxIterElems = 1LL << 22;   // C * H * pitch of one iterate buffer
constexpr long long kMaxTiles = 16384;           // blocks per channel
constexpr long long kMaxTileWords = kMaxTiles * 2 * 64;    // block masks: 2 words per thread, blocks x threads <= 2^20
constexpr long long kMaxPartials = 2LL * DD_MAX_STAT_CHANNELS;   // exact residual sums per channel (words)
constexpr long long kMaxResBlocks = 65536;       // C * blocks of the FP64 residual pass
constexpr int kMaxChannels = DD_MAX_STAT_CHANNELS;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffU0 = 0;
constexpr size_t kOffU1 = kOffU0 + align256(kMaxIterElems * 4);
constexpr size_t kOffTmask = kOffU1 + align256(kMaxIterElems * 4);
constexpr size_t kOffPartial = kOffTmask + align256(kMaxTileWords * 4);
constexpr size_t kOffResPart = kOffPartial + align256(kMaxPartials * 8);
constexpr size_t kOffResOut = kOffResPart + align256(kMaxResBlocks * 16);
constexpr size_t kOffNorms = kOffResOut + align256(kMaxChannels * 16);
constexpr size_t kOffRef = kOffNorms + align256((2 * kMaxChannels + 2) * 8);
constexpr size_t kOffFlag = kOffRef + align256(kMaxChannels * 8);
constexpr size_t kOffState = kOffFlag + align256(dd::kFlagWords * 4);
constexpr size_t kOffTol = kOffState + align256(4 * 4);
constexpr size_t kOffCount = kOffTol + align256(8);
constexpr size_t kOffTicket = kOffCount + align256(8);
constexpr size_t kScratchBytes = kOffTicket + align256(4);

}  // namespace

// The scratch array (device memory of the module, zero at load).
static __device__ __align__(256) unsigned char g_dd_static_scratch[kScratchBytes];

namespace {

std::mutex g_setup_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};

// Error paths only: record the message for dd_last_error() and return the code.
int fail(int code, const char* msg) {
    dd::set_last_error(msg);
    return code;
}

// Device address of the scratch array on the current device (set up once).
int scratch_base(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(DD_ECUDA, "cudaGetDevice failed or device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_dd_static_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(DD_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return DD_OK;
}

#define SS_CK(call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return fail(DD_ECUDA, #call " failed");                    \
    } while (0)

// FP64 residual norms of an FP32 iterate; norms and maxima back on the host.
// ticket: a zero counter (the pass leaves it zero).
int res_norms(int H, int W, int C, const float* u, int P, const uint8_t* mask, double2* part, int nblk,
              double2* out_d, unsigned int* ticket, double2* out_h, cudaStream_t st) {
    dd::Res64Args a{};
    a.H = H; a.W = W; a.C = C;
    a.u = u; a.up = P; a.uplane = (long long)H * P;
    a.mask = mask; a.mp = W;
    a.g_out = nullptr; a.gst = dd::Store::F32;
    a.part = part; a.nblk = nblk;
    a.out = out_d; a.ticket = ticket;
    SS_CK(dd::launch_res64(a, st));
    SS_CK(cudaMemcpyAsync(out_h, out_d, sizeof(double2) * C, cudaMemcpyDeviceToHost, st));
    SS_CK(cudaStreamSynchronize(st));
    return DD_OK;
}

}  // namespace

extern "C" int dd_inpaint_solve_static(int H, int W, int C, const uint8_t* mask, const float* values, float* u_out,
                                       const dd_params* params, double tol, void* stream) {
    if (H <= 0 || W <= 0 || C <= 0 || !mask || !values || !u_out || !(tol > 0.0))
        return fail(DD_EINVAL, "bad arguments");
    dd_params p;
    if (params) p = *params; else dd_params_default(&p);
    if (!dd::block_supported(p.block) || p.overlap < 0 || p.overlap >= p.block || p.local_cg_iters < 1 ||
        p.local_cg_iters > 4096 || p.max_sweeps < 0 || p.test_stall_polls < 0 ||
        (p.tile_warps != 0 && !dd::tile_warps_supported(p.block, p.tile_warps)))
        return fail(DD_EINVAL, "bad params");
    if (!(p.local_rtol >= 0.0) || !(p.local_rtol < 1.0)) return fail(DD_EINVAL, "local_rtol must be in [0, 1)");
    if (p.solver != DD_SOLVER_ORAS) return fail(DD_EINVAL, "dd_inpaint_solve_static runs DD_SOLVER_ORAS only");
    if (C > kMaxChannels) return fail(DD_EINVAL, "C exceeds the static scratch capacity (16 channels)");
    const int P = (W + 31) / 32 * 32;
    const long long elems = (long long)C * H * P;
    const dd::TileGeom g = dd::make_geom(H, W, P, p.block, p.overlap, p.tile_warps);
    const int nblk = dd::res64_blocks(H, W);
    if (elems > kMaxIterElems || g.ntiles > kMaxTiles || (long long)nblk * C > kMaxResBlocks ||
        (long long)dd::tmask_words(g) > kMaxTileWords)
        return fail(DD_EINVAL, "image exceeds the static scratch capacity: C*H*roundup(W,32) <= 4194304 and "
                               "at most 16384 blocks per channel");
    const float pr = p.robin_p > 0.f ? p.robin_p : dd::default_robin(p.block, p.overlap);

    unsigned char* base = nullptr;
    if (int rc = scratch_base(&base); rc != DD_OK) return rc;
    float* u[2] = {reinterpret_cast<float*>(base + kOffU0), reinterpret_cast<float*>(base + kOffU1)};
    uint32_t* tmask = reinterpret_cast<uint32_t*>(base + kOffTmask);
    unsigned long long* partial = reinterpret_cast<unsigned long long*>(base + kOffPartial);
    double2* res_part = reinterpret_cast<double2*>(base + kOffResPart);
    double2* res_out = reinterpret_cast<double2*>(base + kOffResOut);
    double* norms2 = reinterpret_cast<double*>(base + kOffNorms);
    double* ref_d = reinterpret_cast<double*>(base + kOffRef);
    int* flag = reinterpret_cast<int*>(base + kOffFlag);
    int* sstate = reinterpret_cast<int*>(base + kOffState);
    double* tol_d = reinterpret_cast<double*>(base + kOffTol);
    unsigned int* ticket = reinterpret_cast<unsigned int*>(base + kOffTicket);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long plane = (long long)H * P;

    CUtensorMap maps[2];
    for (int b = 0; b < 2; ++b)
        if (dd::make_tile_map(&maps[b], dd::Store::F32, u[b], H, W, P, C, p.block) != cudaSuccess)
            return fail(DD_ECUDA, "cuTensorMapEncodeTiled failed");

    // the error word starts clear; u0 = C f, block masks, reference norms ||b - A u0||
    SS_CK(cudaMemsetAsync(flag + 5, 0, sizeof(int), st));
    SS_CK(cudaMemsetAsync(partial, 0, sizeof(unsigned long long) * 2 * C, st));
    SS_CK(dd::launch_masked_copy(H, W, C, values, W, (long long)H * W, mask, W, u[0], P, plane, st));
    SS_CK(dd::launch_build_tmask(g, mask, W, tmask, st));
    double2 h_res[kMaxChannels];
    if (int rc = res_norms(H, W, C, u[0], P, mask, res_part, nblk, res_out, ticket, h_res, st); rc != DD_OK) return rc;
    double ref[kMaxChannels];
    for (int c = 0; c < C; ++c) ref[c] = std::sqrt(h_res[c].x);
    {
        // an empty mask leaves A singular: every block pixel is then unknown
        unsigned long long* cnt_d = reinterpret_cast<unsigned long long*>(base + kOffCount);
        unsigned long long cnt = 0, area = 0;
        SS_CK(cudaMemsetAsync(cnt_d, 0, sizeof(cnt), st));
        SS_CK(dd::launch_count_unknown(g, tmask, cnt_d, st));
        SS_CK(cudaMemcpyAsync(&cnt, cnt_d, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        SS_CK(cudaStreamSynchronize(st));
        for (int ty = 0; ty < g.nty; ++ty)
            for (int tx = 0; tx < g.ntx; ++tx)
                area += (unsigned long long)std::min(p.block, H - ty * g.s) * std::min(p.block, W - tx * g.s);
        if (cnt == area) return fail(DD_EEMPTYMASK, "empty mask");
    }
    SS_CK(cudaMemcpyAsync(ref_d, ref, sizeof(double) * C, cudaMemcpyHostToDevice, st));

    // sweeps with the device-side stop test, read back every 8 launches
    int cur = 0, done = 0;
    double target = tol;
    bool converged = false;
    const dd::SweepPair pair{{&maps[0], &maps[1]}, {u[0], u[1]}};
    for (int attempt = 0; attempt < 4 && !converged; ++attempt) {
        SS_CK(dd::launch_reset_sweep_state(sstate, flag, cur, tol_d, target, st));
        dd::SweepStop stop{partial, norms2, ref_d, tol_d, 0.0, flag, sstate, 0,
                           nullptr, flag + 5, p.test_stall_polls};
        const int start = done;
        int launched = 0;
        int hflag[3] = {0, 0, 0}, herr = 0, hstate[2] = {cur, 0};
        while (true) {
            const bool last_probe = done >= p.max_sweeps;
            const int n = last_probe ? 1 : std::min(8, p.max_sweeps - done);
            for (int i = 0; i < n; ++i) {
                stop.force_probe = last_probe ? 1 : 0;
                SS_CK(dd::launch_sweep(dd::Store::F32, g, C, plane, pair, nullptr, tmask, stop, pr,
                                       p.local_cg_iters, st, (float)p.local_rtol));
            }
            launched += n;
            SS_CK(cudaMemcpyAsync(hflag, flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
            SS_CK(cudaMemcpyAsync(&herr, flag + 5, sizeof(int), cudaMemcpyDeviceToHost, st));
            SS_CK(cudaMemcpyAsync(hstate, sstate, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
            SS_CK(cudaStreamSynchronize(st));
            if (herr != 0) return fail(DD_ETIMEOUT, "a bounded device wait for a staged tile gave up");
            if (hflag[0] == 2) return fail(DD_ENUMERIC, "non-finite residual norm");
            cur = hstate[0];
            done = start + hstate[1];
            if (hflag[0] == 1 || last_probe) break;
        }
        // verify in FP64 on the iterate that is returned
        if (int rc = res_norms(H, W, C, u[cur], P, mask, res_part, nblk, res_out, ticket, h_res, st); rc != DD_OK) return rc;
        double worst = 0.0;
        for (int c = 0; c < C; ++c) worst = std::max(worst, std::sqrt(h_res[c].x) / (ref[c] > 0.0 ? ref[c] : 1.0));
        if (!std::isfinite(worst)) return fail(DD_ENUMERIC, "non-finite residual");
        if (worst <= tol) converged = true;
        else if (hflag[0] != 1 || done >= p.max_sweeps) break;
        else target *= 0.5;
    }
    SS_CK(dd::launch_copy2d(H, W, C, u[cur], P, plane, u_out, W, (long long)H * W, st));
    SS_CK(cudaStreamSynchronize(st));
    return converged ? DD_OK : fail(DD_ENOTCONVERGED, "not converged within the sweep limit");
}
