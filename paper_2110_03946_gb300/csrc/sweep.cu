// ORAS sweep kernels (Sec. 3-4 of Kaemper & Weickert, arXiv 2110.03946).
//
// One sweep computes, for every block Omega_i of every channel, the local
// residual R_i r^n with r^n = b - A u^n, runs k conjugate-gradient steps on the
// local problem R_i A R_i^T v_i = R_i r^n (Eq. eq:ras-local-problem) with the
// optimised Robin interface condition, and adds v_i back on the block's owned
// core only (u^{n+1} = u^n + sum_i R_i^T D_i v_i, D_i 0/1).  All blocks read
// u^n and write u^{n+1} into a second buffer (additive Schwarz).
//
// GPU mapping.  Persistent CTAs take (channel, block) tiles in increasing
// order from an atomic counter, so CTAs whose local problems stop early take
// more tiles.  Thread 0 stages the next block's tile plus a one-pixel halo (and the correction
// source, if any) into shared memory with a TMA tensor copy while the CTA
// works on the current block (two buffers, one mbarrier each; every wait is
// bounded and a timeout sets an error word).  The block is then held in
// registers by NW warps: lane (lx, ly) of warp wt owns a PX x PY patch (PX
// columns as PX/2 packed FP32 pairs).  Values across patch borders move by
// warp shuffles and, between the NW warps, through shared memory.  Each CG step
// has one tile-wide reduction of three dot products: xor-butterfly warp sums
// (bitwise identical on every lane, so all break decisions are uniform) plus a
// fixed-order sum over warps.  Packed pair arithmetic (__ffma2_rn and friends,
// sm_100+) halves the issue slots.
//
// Local operator (unknown pixel p of the block):
//   (A_i v)_p = dd_p v_p - sum_{q in N(p), q in block} v_q,
//   dd_p = #{in-block neighbours} + p_R * #{in-image neighbours outside the block},
// known pixels have identity rows of A and, because u = f is held there, zero
// right-hand side, so v = 0 on them; the kernel keeps r = p = q = 0 there.
// The kernel computes q' = -(A_i p) = w (sum + nd p), nd = -dd, w = 1 - known.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "dd_internal.h"

namespace dd {

namespace {

// Residual contraction per ORAS sweep assumed before a level has two full
// sweeps of history (probe prediction only: it decides whether the next launch
// probes or sweeps, never whether the level has converged).
constexpr double kFirstContraction = 0.3;
// The residual contraction a final sweep with the looser local tolerance
// (SweepStop::final_local_rtol) is counted on: the next sweep is such a final
// sweep when its predicted input residual times this factor meets tol.
constexpr double kFinalContraction = 0.6;

constexpr unsigned FULL = 0xffffffffu;
constexpr int kWaitLimit = 1 << 22;   // bounded mbarrier polls (a TMA copy takes ~1 us)
constexpr int kDynamicRounds = 4;     // tiles per CTA (average) claimed dynamically at the end of a sweep

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ---- TMA / mbarrier primitives (PTX ISA: mbarrier, cp.async.bulk.tensor) ----------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit = kWaitLimit) {
    for (int n = 0; n < limit; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Exact, order-independent sums of non-negative FP32 values: a 128-bit
// fixed-point accumulator with the unit 2^eu.  A value's bits below the unit
// are dropped and values of 2^(eu + 104) or more saturate there; both depend on
// the value alone, so a set of values has the same sum in any order (and up to
// 2^24 values cannot overflow).  Non-finite values are flagged by the caller.
struct Fix128 {
    unsigned long long lo, hi;
};
__device__ __forceinline__ void fix_add(Fix128& acc, float v, int eu) {
    const unsigned bits = __float_as_uint(v);
    const int be = (int)((bits >> 23) & 0xffu);
    if (!(v > 0.f) || be == 0xff) return;
    unsigned long long m = (bits & 0x7fffffu) | (be != 0 ? 0x800000u : 0u);
    int sh = (be != 0 ? be : 1) - 150 - eu;   // v = m 2^(sh + eu)
    if (sh < 0) {
        if (sh <= -24) return;
        m >>= -sh;
        sh = 0;
    }
    if (sh > 80) {
        m = 0xffffffull;
        sh = 80;
    }
    const unsigned long long lo = sh < 64 ? m << sh : 0ull;
    const unsigned long long hi = sh == 0 ? 0ull : (sh < 64 ? m >> (64 - sh) : m << (sh - 64));
    acc.lo += lo;
    acc.hi += hi + (acc.lo < lo ? 1ull : 0ull);
}
__device__ __forceinline__ void fix_add(Fix128& acc, unsigned long long lo, unsigned long long hi) {
    acc.lo += lo;
    acc.hi += hi + (acc.lo < lo ? 1ull : 0ull);
}
// The accumulator unit of a channel with reference norm ref: 2^-72 ref^2, so
// sums from about 2^-72 to 2^32 times ref^2 are exact before the final rounding.
__device__ __forceinline__ int fix_unit(double ref) {
    return 2 * ilogb(ref > 0.0 && isfinite(ref) ? ref : 1.0) - 72;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Tile shape: LX x LY lanes per warp, PX x PY pixels per lane, NW warps stacked
// vertically; one block tile per CTA at a time.
template <int PX_, int PY_, int LX_, int NW_>
struct Cfg {
    static constexpr int PX = PX_, PY = PY_, LX = LX_, NW = NW_;
    static constexpr int LY = 32 / LX;
    static constexpr int BW = LX * PX;
    static constexpr int BH = NW * LY * PY;
    static constexpr int NP = PX / 2;
    static constexpr int NT = NW * 32;
    static_assert(PX % 2 == 0 && PX * PY <= 32 && BW == BH && 32 % LX == 0, "bad tile shape");
};

using Cfg16 = Cfg<2, 4, 8, 1>;     // 16 x 16 block, one warp, 8 px per lane
using Cfg32 = Cfg<4, 8, 8, 1>;     // 32 x 32 block, one warp, 32 px per lane
using Cfg32w2 = Cfg<4, 4, 8, 2>;   // 32 x 32 block, two warps of 32 x 16, 16 px per lane
using Cfg32w4 = Cfg<4, 2, 8, 4>;   // 32 x 32 block, four warps of 32 x 8, 8 px per lane
using Cfg64 = Cfg<4, 8, 16, 4>;    // 64 x 64 block, four warps of 64 x 16, 32 px per lane
using Cfg64w8 = Cfg<4, 4, 16, 8>;  // 64 x 64 block, eight warps of 64 x 8, 16 px per lane
using Cfg96 = Cfg<6, 4, 16, 12>;   // 96 x 96 block, twelve warps of 96 x 8, 24 px per lane

// Calls f(Cfg{}) for the tile layout of block side b with nw warps per block.
template <class F>
cudaError_t with_cfg(int b, int nw, F&& f) {
    switch (b) {
        case 16: return nw == 1 ? f(Cfg16{}) : cudaErrorInvalidValue;
        case 32: return nw == 1 ? f(Cfg32{}) : nw == 2 ? f(Cfg32w2{}) : nw == 4 ? f(Cfg32w4{}) : cudaErrorInvalidValue;
        case 64: return nw == 4 ? f(Cfg64{}) : nw == 8 ? f(Cfg64w8{}) : cudaErrorInvalidValue;
        case 96: return nw == 12 ? f(Cfg96{}) : cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

// Mask words of one block tile (known bits, owned bits: one word each per thread).
template <class CF>
constexpr int mask_bytes() {
    return 2 * CF::NT * 4;
}

// Shared-memory tile: block plus one-pixel halo; the TMA box starts at a
// 16-byte aligned column at or left of x0 - 1, so it is BX >= BW + 2 + (align - 1) wide.
template <class CF, typename T>
struct Box {
    static constexpr int ALIGN = 16 / (int)sizeof(T);
    static constexpr int BX = (CF::BW + 2 + ALIGN - 1 + ALIGN - 1) / ALIGN * ALIGN;
    static constexpr int BY = CF::BH + 2;
    static constexpr int BYTES = BX * BY * (int)sizeof(T);
    static constexpr int STRIDE = (BYTES + 127) / 128 * 128;   // per staged array
    static_assert(BX <= 256 && BY <= 256, "TMA box too large");
};

__device__ __forceinline__ int fdiv(int n, FastDiv f) {
    return (int)(((unsigned long long)__umulhi((uint32_t)n, f.m) + (uint32_t)n) >> f.s);
}

// Two sums over the threads of one tile in one butterfly.
template <class CF>
__device__ __forceinline__ float2 tile_sum2(float2 v, float* red_a, float* red_b, int wt, int lane) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        v.x += __shfl_xor_sync(FULL, v.x, m);
        v.y += __shfl_xor_sync(FULL, v.y, m);
    }
    if constexpr (CF::NW == 1) {
        return v;
    } else {
        if (lane == 0) {
            red_a[wt] = v.x;
            red_b[wt] = v.y;
        }
        __syncthreads();
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < CF::NW; ++w) {
            t.x += red_a[w];
            t.y += red_b[w];
        }
        return t;
    }
}

// Three sums over the threads of one tile in one butterfly (red: 3 x NW floats).
template <class CF>
__device__ __forceinline__ float3 tile_sum3(float3 v, float* red, int wt, int lane) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        v.x += __shfl_xor_sync(FULL, v.x, m);
        v.y += __shfl_xor_sync(FULL, v.y, m);
        v.z += __shfl_xor_sync(FULL, v.z, m);
    }
    if constexpr (CF::NW == 1) {
        return v;
    } else {
        if (lane == 0) {
            red[wt] = v.x;
            red[CF::NW + wt] = v.y;
            red[2 * CF::NW + wt] = v.z;
        }
        __syncthreads();
        float3 t = make_float3(0.f, 0.f, 0.f);
#pragma unroll
        for (int w = 0; w < CF::NW; ++w) {
            t.x += red[w];
            t.y += red[CF::NW + w];
            t.z += red[2 * CF::NW + w];
        }
        return t;
    }
}

// Exact sum of the 32 lanes' fixed-point accumulators (integer adds with
// carry, so the result does not depend on the order); every lane gets it.
__device__ __forceinline__ Fix128 warp_fix_sum(Fix128 f) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(FULL, f.lo, m), hi = __shfl_xor_sync(FULL, f.hi, m);
        fix_add(f, lo, hi);
    }
    return f;
}

// Add a 128-bit value exactly into a sum in global memory: the low word with
// one atomic, its carry with the high word in a second.  The number of carries
// over all adds is that of the total, so the final sum does not depend on the
// order of the adds.
__device__ __forceinline__ void fix_atomic_add(unsigned long long* dst, const Fix128& v) {
    if (v.lo == 0ull && v.hi == 0ull) return;
    const unsigned long long old = atomicAdd(dst, v.lo);
    const unsigned long long carry = (old + v.lo < old) ? 1ull : 0ull;
    if (v.hi + carry != 0ull) atomicAdd(dst + 1, v.hi + carry);
}

// The stop test of one frame's sweep (one thread, after all its tiles' sums
// are in F.acc): norms, the stop flag and the sweep state for the next launch;
// the sums and the tile count are zeroed for the next sweep.
__device__ __forceinline__ void frame_stop_test(const SweepFrame& F, bool probe, int cur) {
    __threadfence();
    int* const flag = F.flag;
    int* const state = F.state;
    const int C = F.C;
    const int sweep_index = __ldcg(state + 3);   // launches before this one
    const double tol = __ldcg(F.tol);
    double worst = 0.0, best_ratio = 1e300;
    bool bad = __ldcg(flag + 6) != 0;
    for (int c = 0; c < C; ++c) {
        const unsigned long long lo = __ldcg(F.acc + 2 * c), hi = __ldcg(F.acc + 2 * c + 1);
        F.acc[2 * c] = 0ull;
        F.acc[2 * c + 1] = 0ull;
        const double ref = F.ref[c];
        const int ec = fix_unit(ref);
        const double v = ldexp((double)hi, 64 + ec) + ldexp((double)lo, ec);
        if (!isfinite(v)) bad = true;
        const double den = ref > 0.0 ? ref : 1.0;
        worst = fmax(worst, sqrt(v) / den);
        if (sweep_index > 0) {
            const double prev = F.norms2[C + c];
            best_ratio = fmin(best_ratio, prev > 0.0 ? sqrt(v / prev) : 0.0);
        }
        F.norms2[c] = v;
        if (!probe) F.norms2[C + c] = v;
    }
    flag[2] = 0;
    flag[6] = 0;
    if (F.work != nullptr && sweep_index < kTimedLaunches) F.work[2 + sweep_index] = probe ? 0ull : 1ull;
    if (__ldcg(F.err) != 0) { flag[0] = 5; flag[1] = sweep_index; }
    else if (bad) { flag[0] = 2; flag[1] = sweep_index; }
    else if (worst <= tol) { flag[0] = 1; flag[1] = sweep_index; }
    else if (F.stall > 0.0 && sweep_index > 0 && best_ratio > F.stall) {
        flag[0] = 3;
        flag[1] = sweep_index;
    } else if (!probe) {
        // the output of this sweep becomes the current iterate; probe it next
        // if the residual ratio of this level's last two full sweeps (before its
        // second full sweep: an assumed contraction of kFirstContraction)
        // predicts that it meets tol
        const double prev_worst = F.norms2[2 * C];
        const bool history = state[1] > 0 && prev_worst > 0.0;
        const double pred = history ? worst * (worst / prev_worst) : worst * kFirstContraction;
        state[0] = cur ^ 1;
        state[1] += 1;
        // 1: probe the next iterate; 2: the next sweep is predicted to be the last
        // and takes the final local tolerance
        state[2] = (tol > 0.0 && pred <= tol) ? 1
                   : (tol > 0.0 && F.local_rtol2_final > 0.f && pred * kFinalContraction <= tol) ? 2 : 0;
    } else {
        state[2] = 0;   // the probe failed: sweep the same iterate in full
    }
    if (!probe) F.norms2[2 * C] = worst;
    state[3] = sweep_index + 1;
}

// ALN: every block starts at a column that is a multiple of 4 (stride s % 4 == 0,
// FP32 storage, 4 pixels per lane row), so a lane's 4 pixels of a row are one
// 16-byte vector in the staged tile.
// BATCH: the tiles of several frames (the list written by batch_ctl_kernel) in
// one launch; otherwise one frame, passed by value.  HASG: the frame solves
// A u = C f + (I - C) g with a source g staged beside u (has_g).
template <class CF, typename T, bool ALN, bool BATCH, bool HASG>
__global__ void __launch_bounds__(CF::NT)
oras_sweep_kernel(const __grid_constant__ SweepFrame one, const SweepFrame* __restrict__ many,
                  const int* __restrict__ list, int* __restrict__ lctl) {
    constexpr int PX = CF::PX, PY = CF::PY, LX = CF::LX, LY = CF::LY, NW = CF::NW;
    constexpr int BW = CF::BW, BH = CF::BH, NP = CF::NP, NT = CF::NT;
    using BOX = Box<CF, T>;
    constexpr int BX = BOX::BX;
    static_assert(!ALN || (PX == 4 && sizeof(T) == 4 && BX % 4 == 0), "aligned path: 4 FP32 pixels per lane row");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[3];   // [2]: never completed (the stalled-wait test hook)
    __shared__ int s_ok;
    __shared__ int s_next[2];          // next tile, by iteration parity
    __shared__ float red[3][NW];
    __shared__ float red3[2][3][NW];   // CG reductions (p,Ap), (Ap,Ap), (r,r), alternating by step parity
    __shared__ float xch[2][NW][BW];      // initial boundary rows of r
    __shared__ float xq[2][2][NW][BW];    // boundary rows of q', alternating by step parity

    const int n_act = BATCH ? __ldg(list) : 1;
    if (n_act <= 0) return;                        // uniform: no frame to sweep
    if (!BATCH && one.flag[0] != 0) return;        // uniform: converged or failed earlier
    const int total = BATCH ? __ldg(list + 1 + 2 * n_act) : one.ntiles * one.C;
    int* const ticket = BATCH ? lctl : one.flag + 3;
    int* const counter = BATCH ? lctl + 1 : one.flag + 4;
    // frame slot q of the launch: its descriptor and its tiles [begin, end)
    auto frame_at = [&](int q) -> const SweepFrame* { return BATCH ? many + __ldg(list + 1 + q) : &one; };
    auto begin_at = [&](int q) { return BATCH ? __ldg(list + 1 + n_act + q) : 0; };
    auto end_at = [&](int q) { return BATCH ? __ldg(list + 2 + n_act + q) : total; };

    const int tt = threadIdx.x;
    const int wt = tt >> 5, lane = tt & 31;
    const int lx = lane % LX, ly = lane / LX;
    const int ry0 = (wt * LY + ly) * PY, rx0 = lx * PX;
    static_assert(!(BATCH && HASG), "batched launches have no source term");
    constexpr int narr = HASG ? 2 : 1;
    constexpr int MB = mask_bytes<CF>();
    const uint32_t tx_bytes = (uint32_t)(BOX::BYTES * narr + MB);
    // TMA destinations must be 128-byte aligned: round the dynamic base up
    // (the launch reserves 128 bytes of slack for this).
    unsigned char* const smem =
        smem_raw + (((smem_addr(smem_raw) + 127u) & ~127u) - smem_addr(smem_raw));
    auto stage = [&](int buf, int which) {
        return reinterpret_cast<T*>(smem + (size_t)(buf * narr + which) * BOX::STRIDE);
    };
    // the staged tile's mask words (after the 2 x narr arrays)
    auto stage_mask = [&](int buf) {
        return reinterpret_cast<uint32_t*>(smem + (size_t)2 * narr * BOX::STRIDE + (size_t)buf * MB);
    };
    // the TMA box of a block starts at the 16-byte aligned column at or left of x0 - 1
    auto box_x = [](int x0) { return ((x0 - 1) >= 0 ? (x0 - 1) / BOX::ALIGN : -1) * BOX::ALIGN; };
    int q_st = 0;   // thread 0: frame slot of the last staged tile (a CTA's tiles increase)
    int q_map = -1;   // thread 0: the frame slot whose iterate map is cached in map_st
    const CUtensorMap* map_st = nullptr;
    auto issue = [&](int tn, int buf) {   // thread 0 only
        while (q_st + 1 < n_act && tn >= end_at(q_st)) ++q_st;
        const SweepFrame* const F = frame_at(q_st);
        if (q_map != q_st) {   // the buffer holding the frame's iterate is fixed for the launch
            map_st = __ldcg(F->state) ? &F->map_u[1] : &F->map_u[0];
            q_map = q_st;
        }
        const int local = tn - begin_at(q_st);
        const int c = fdiv(local, F->dv_tiles);
        const int tile = local - c * F->ntiles;
        const int ty = fdiv(tile, F->dv_ntx), tx = tile - ty * F->ntx;
        const int x0 = tx * F->s, y0 = ty * F->s;
        const int xs = box_x(x0);
        // (no proxy fence: the staging buffers are written only by these copies, and
        // the generic reads of a buffer's previous tile ended at the barrier
        // that closed its iteration)
        mbar_expect_tx(&mbar[buf], tx_bytes);
        tma_load_3d(stage(buf, 0), map_st, xs, y0 - 1, c, &mbar[buf]);
        if constexpr (HASG) tma_load_3d(stage(buf, 1), &F->map_g, xs, y0 - 1, c, &mbar[buf]);
        bulk_load(stage_mask(buf), F->tmask + (size_t)tile * 2 * NT, (uint32_t)MB, &mbar[buf]);
    };

    if (tt == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init(&mbar[2], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Tile order: the tiles below static_end go round-robin (CTA b takes b,
    // b + G, ...); after its last one a CTA claims further tiles from an atomic
    // counter, so CTAs whose local problems stopped early take more of the
    // tail.  Thread 0 claims one iteration ahead of the staging.  A CTA's tiles
    // come in increasing order either way (so frames and channels too).
    const int G = (int)gridDim.x;
    const int static_end = max(G, total - kDynamicRounds * G);
    auto next_of = [&](int tcur) {   // thread 0 only
        return tcur + G < static_end ? tcur + G : (int)atomicAdd(reinterpret_cast<unsigned*>(counter), 1u) + static_end;
    };
    int t = blockIdx.x;
    int claim = 0;
    if (tt == 0 && t < total) {
        issue(t, 0);
        claim = next_of(t);
    }

    const float fW = lx > 0 ? 1.f : 0.f, fE = lx < LX - 1 ? 1.f : 0.f;
    // NW == 1: a lane of the block's top (bottom) lane row has no north (south)
    // neighbour lane; its shuffled value is weighted 0
    const float2 fN2 = make_float2(ly > 0 ? 1.f : 0.f, ly > 0 ? 1.f : 0.f);
    const float2 fS2 = make_float2(ly < LY - 1 ? 1.f : 0.f, ly < LY - 1 ? 1.f : 0.f);
    // The frame being processed: its slot, descriptor and launch state (the
    // iterate buffer and whether this launch probes it), read when the CTA
    // meets the frame (before the frame's stop test can change them).
    int q_pr = -1;
    const SweepFrame* Fp = nullptr;
    int f_cur = 0, f_kcg = 0, f_tiles = 0;
    int f_probe = 0;   // (ints rather than bools for the state kept across tiles: fewer live predicates)
    float f_rtol2 = 0.f;   // the squared local tolerance of this frame's sweep
    float f_aunit = 0.f;   // local_atol^2 tol^2 / blocks: times ref_c^2, the squared absolute local stop
    float f_atol2 = 0.f;   // ... of the current channel
    // Residual sums of the input iterate per channel, exact (Fix128): lane
    // (it mod 32) holds the owned ||r||^2 of this CTA's tile it until every 32
    // tiles (or a change of channel) all lanes add their value into their own
    // accumulator at once; the lanes' accumulators are summed and added to the
    // frame's sums when the CTA leaves the channel.
    int cur_c = -1, eu = 0;
    Fix128 acc{0ull, 0ull};
    float pend = 0.f;
    int acc_bad = 0;   // the same on every lane (it follows the tile-uniform sums)
    uint32_t work_us = 0, work_u = 0;   // optional work counters (per lane)
    auto flush_channel = [&]() {   // all threads
        if (cur_c >= 0) {
            fix_add(acc, pend, eu);
            const Fix128 f = warp_fix_sum(acc);
            if (tt == 0) {
                if (acc_bad) atomicExch(Fp->flag + 6, 1);
                fix_atomic_add(Fp->acc + 2 * cur_c, f);
            }
        }
        acc = Fix128{0ull, 0ull};
        pend = 0.f;
        acc_bad = 0;
        cur_c = -1;
    };
    // leaving frame Fp: its sums, its work counters and its count of done tiles;
    // the CTA that completes the count runs the frame's stop test
    auto flush_frame = [&]() {   // all threads
        flush_channel();
        if (Fp->work != nullptr) {
            const uint32_t ws = __reduce_add_sync(FULL, work_us), wu = __reduce_add_sync(FULL, work_u);
            if (lane == 0 && wu != 0) {
                atomicAdd(Fp->work, (unsigned long long)ws);
                atomicAdd(Fp->work + 1, (unsigned long long)wu);
            }
        }
        work_us = work_u = 0;
        if constexpr (NW > 1) __syncthreads();   // every warp's work counters are in
        if (tt == 0) {
            __threadfence();
            const int prev = atomicAdd(Fp->flag + 2, f_tiles);
            if (prev + f_tiles == Fp->ntiles * Fp->C) frame_stop_test(*Fp, f_probe != 0, f_cur);
        }
        f_tiles = 0;
    };
    int it = 0;
    for (; t < total; ++it) {
        const int buf = it & 1;
        const uint32_t parity = (uint32_t)((it >> 1) & 1);
        if (tt == 0) {   // stage the next tile while this one is solved, and claim the one after
            const int tn = claim;
            s_next[buf] = tn;
            if (tn < total) {
                issue(tn, buf ^ 1);
                claim = next_of(tn);
            }
        }
        int q = q_pr < 0 ? 0 : q_pr;
        while (q + 1 < n_act && t >= end_at(q)) ++q;
        if (q != q_pr) {   // a new frame (uniform)
            if (q_pr >= 0) flush_frame();
            q_pr = q;
            Fp = frame_at(q);
            f_cur = __ldcg(Fp->state);
            const int req = __ldcg(Fp->state + 2);
            f_probe = (Fp->force_probe != 0 || req == 1) ? 1 : 0;
            f_rtol2 = req == 2 ? Fp->local_rtol2_final : Fp->local_rtol2;
            if (Fp->local_atol2 > 0.f) {
                const double tv = __ldcg(Fp->tol);
                f_aunit = tv > 0.0 ? (float)((double)Fp->local_atol2 * tv * tv / (double)Fp->ntiles) : 0.f;
            } else {
                f_aunit = 0.f;
            }
            f_kcg = f_probe ? 0 : Fp->k;
        }
        const int local = t - begin_at(q);
        const int c = fdiv(local, Fp->dv_tiles);
        const int tile = local - c * Fp->ntiles;
        const int ty = fdiv(tile, Fp->dv_ntx), tx = tile - ty * Fp->ntx;
        const int y0 = ty * Fp->s, x0 = tx * Fp->s;
        const int H = Fp->H, W = Fp->W;
        const int th = min(BH, H - y0), tw = min(BW, W - x0);
        const int cx = ALN ? 4 : x0 - box_x(x0);   // smem column of x0

        if (tt == 0) {
            const bool ok = (it == 0 && Fp->stall_polls > 0) ? mbar_wait_bounded(&mbar[2], 0u, Fp->stall_polls)
                                                             : mbar_wait_bounded(&mbar[buf], parity);
            s_ok = ok ? 1 : 0;
            if (!ok) {
                atomicExch(Fp->err, 1);
                if (BATCH) atomicExch(lctl + 2, 1);   // the whole batched launch is abandoned
            }
        }
        __syncthreads();
        if (!s_ok) break;                               // uniform
        if (tt != 0) mbar_wait_bounded(&mbar[buf], parity);   // phase already complete: returns at once
        const T* __restrict__ U = stage(buf, 0);
        const T* __restrict__ G2 = stage(buf, 1);
        const uint32_t kb = stage_mask(buf)[tt];
        const uint32_t ob = stage_mask(buf)[NT + tt];
        const float pr = Fp->p_robin;

        // ---- local operator coefficients -----------------------------------------
        float2 rpn[PY];     // -(vertical part of dd), both halves equal
        float2 cpn[NP];     // -(horizontal part of dd)
        float2 w2[PY][NP];  // 1 on unknown in-block pixels, else 0
        float2 mN[PY], mS[PY], mW[NP], mE[NP];   // 1 where the neighbour is inside the image
#pragma unroll
        for (int i = 0; i < PY; ++i) {
            const int ry = ry0 + i, y = y0 + ry;
            const float up = ry > 0 ? 1.f : (y > 0 ? pr : 0.f);
            const float dn = ry < th - 1 ? 1.f : (y < H - 1 ? pr : 0.f);
            rpn[i] = make_float2(-(up + dn), -(up + dn));
            const float n = y > 0 ? 1.f : 0.f, sv = y < H - 1 ? 1.f : 0.f;
            mN[i] = make_float2(n, n);
            mS[i] = make_float2(sv, sv);
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            float v[2], wv[2], ev[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int rx = rx0 + 2 * j + e, x = x0 + rx;
                const float lf = rx > 0 ? 1.f : (x > 0 ? pr : 0.f);
                const float rt = rx < tw - 1 ? 1.f : (x < W - 1 ? pr : 0.f);
                v[e] = -(lf + rt);
                wv[e] = x > 0 ? 1.f : 0.f;
                ev[e] = x < W - 1 ? 1.f : 0.f;
            }
            cpn[j] = make_float2(v[0], v[1]);
            mW[j] = make_float2(wv[0], wv[1]);
            mE[j] = make_float2(ev[0], ev[1]);
        }
#pragma unroll
        for (int i = 0; i < PY; ++i)
#pragma unroll
            for (int j = 0; j < NP; ++j)
                w2[i][j] = make_float2(((kb >> (i * PX + 2 * j)) & 1u) ? 0.f : 1.f,
                                       ((kb >> (i * PX + 2 * j + 1)) & 1u) ? 0.f : 1.f);

        // ---- local residual R_i (b - A u^n) and the owned residual norm ----------
        // The patch and its one-pixel ring are read from the staged tile once.
        // r_p = g_p + sum over in-image neighbours q of (u_q - u_p): each
        // difference is exact for close values, and a neighbour outside the image
        // (reflecting boundary; the staged tile holds zero there) gets weight 0.
        float2 r2[PY][NP];
        float s2 = 0.f, rr0 = 0.f;
        {
            const int o0 = (1 + ry0) * BX + cx + rx0;
            float uu[PY + 2][PX + 2];
#pragma unroll
            for (int i = 0; i < PY + 2; ++i) {
                const T* row = U + o0 + (i - 1) * BX;
                if constexpr (ALN) {   // columns 0..3 as one vector, -1 and 4 as scalars
                    const float4 q4 = *reinterpret_cast<const float4*>(row);
                    uu[i][1] = q4.x; uu[i][2] = q4.y; uu[i][3] = q4.z; uu[i][4] = q4.w;
                    const bool edge_row = i == 0 || i == PY + 1;
                    uu[i][0] = edge_row ? 0.f : to_f(row[-1]);
                    uu[i][PX + 1] = edge_row ? 0.f : to_f(row[PX]);
                } else {
#pragma unroll
                    for (int j = 0; j < PX + 2; ++j) {
                        const bool corner = (i == 0 || i == PY + 1) && (j == 0 || j == PX + 1);
                        uu[i][j] = corner ? 0.f : to_f(row[j - 1]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < PY; ++i)
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const float2 uc = make_float2(uu[i + 1][2 * j + 1], uu[i + 1][2 * j + 2]);
                    const float2 nuc = make_float2(-uc.x, -uc.y);
                    float2 acc2 = make_float2(0.f, 0.f);
                    if constexpr (HASG) acc2 = make_float2(to_f(G2[o0 + i * BX + 2 * j]), to_f(G2[o0 + i * BX + 2 * j + 1]));
                    acc2 = fma2(mN[i], add2(make_float2(uu[i][2 * j + 1], uu[i][2 * j + 2]), nuc), acc2);
                    acc2 = fma2(mS[i], add2(make_float2(uu[i + 2][2 * j + 1], uu[i + 2][2 * j + 2]), nuc), acc2);
                    acc2 = fma2(mW[j], add2(make_float2(uu[i + 1][2 * j], uu[i + 1][2 * j + 1]), nuc), acc2);
                    acc2 = fma2(mE[j], add2(make_float2(uu[i + 1][2 * j + 2], uu[i + 1][2 * j + 3]), nuc), acc2);
                    const float2 res = mul2(w2[i][j], acc2);
                    r2[i][j] = res;
                    rr0 = fmaf(res.x, res.x, fmaf(res.y, res.y, rr0));
                    const bool o_x = (ob >> (i * PX + 2 * j)) & 1u, o_y = (ob >> (i * PX + 2 * j + 1)) & 1u;
                    s2 = fmaf(o_x ? res.x : 0.f, res.x, fmaf(o_y ? res.y : 0.f, res.y, s2));
                }
        }
        // ---- k CG steps from v = 0 (Saad, the CG algorithm of Ch. 6) --------------
        float2 v2[PY][NP], p2[PY][NP], q2[PY][NP];
        float rr, rr_stop;
        float rrp = rr0;   // this thread's part of (r, r), summed again in the first CG step
        {
#pragma unroll
            for (int i = 0; i < PY; ++i)
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    v2[i][j] = make_float2(0.f, 0.f);
                    p2[i][j] = r2[i][j];
                }
            if constexpr (NW > 1) {   // boundary rows of r (= p) for the neighbouring warps
                if (ly == 0)
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        xch[0][wt][rx0 + 2 * j] = r2[0][j].x;
                        xch[0][wt][rx0 + 2 * j + 1] = r2[0][j].y;
                    }
                if (ly == LY - 1)
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        xch[1][wt][rx0 + 2 * j] = r2[PY - 1][j].x;
                        xch[1][wt][rx0 + 2 * j + 1] = r2[PY - 1][j].y;
                    }
            }
            // owned ||r||^2 and the initial (r, r) in one butterfly (a barrier when NW > 1)
            const float2 both = tile_sum2<CF>(make_float2(s2, rr0), red[0], red[1], wt, lane);
            s2 = both.x;
            rr = both.y;
        }
        // the owned residual sum of this tile into the lane-batched accumulators
        if (c != cur_c) {
            flush_channel();
            cur_c = c;
            const double refc = Fp->ref[c];
            eu = fix_unit(refc);
            f_atol2 = (float)((double)f_aunit * refc * refc);
        }
        // local stop: the relative decrease, or the absolute share of the global tolerance
        rr_stop = fmaxf(f_rtol2 * rr, f_atol2);
        ++f_tiles;
        acc_bad |= isfinite(s2) ? 0 : 1;
        if (lane == (it & 31)) pend = s2;
        if ((it & 31) == 31) {
            fix_add(acc, pend, eu);
            pend = 0.f;
        }
        // p rows of the neighbouring warps next to this warp's top / bottom row
        // (and their r rows: each warp advances its neighbours' boundary rows of r
        // and p itself, from their q rows, exactly as the neighbours do)
        float2 nbN[NP], nbS[NP], nrN[NP], nrS[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            nbN[j] = make_float2(0.f, 0.f);
            nbS[j] = make_float2(0.f, 0.f);
            if constexpr (NW > 1) {
                if (ly == 0 && wt > 0) nbN[j] = make_float2(xch[1][wt - 1][rx0 + 2 * j], xch[1][wt - 1][rx0 + 2 * j + 1]);
                if (ly == LY - 1 && wt < NW - 1)
                    nbS[j] = make_float2(xch[0][wt + 1][rx0 + 2 * j], xch[0][wt + 1][rx0 + 2 * j + 1]);
            }
            nrN[j] = nbN[j];
            nrS[j] = nbS[j];
        }
        // One tile-wide reduction per step: (p, Ap), (Ap, Ap) and this step's
        // measured (r, r) are summed together. alpha = (r, r) / (p, Ap) uses the
        // measured value; (r', r') for beta and for the local stop comes from the
        // recurrence |r - alpha Ap|^2 = alpha^2 (Ap, Ap) - (r, r), which holds
        // because (r, Ap) = (p, Ap) for A-conjugate directions. Exact CG in exact
        // arithmetic; the next step measures (r', r') again, so the recurrence
        // error does not accumulate.
        const int kcg = f_kcg;
        float rr_j = rr;   // (r, r) of the current step: measured at step 0, then by the recurrence
        int kk = 0;
        for (; kk < kcg; ++kk) {
            // converged locally (the bound also keeps the quotients below finite)
            if (!(rr_j > 1e-30f) || rr_j <= rr_stop) break;
            float pW[PY], pE[PY];
#pragma unroll
            for (int i = 0; i < PY; ++i) {
                pW[i] = __shfl_up_sync(FULL, p2[i][NP - 1].y, 1, LX);
                pE[i] = __shfl_down_sync(FULL, p2[i][0].x, 1, LX);
            }
            float2 pN[NP], pS[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                pN[j].x = __shfl_up_sync(FULL, p2[PY - 1][j].x, LX);
                pN[j].y = __shfl_up_sync(FULL, p2[PY - 1][j].y, LX);
                pS[j].x = __shfl_down_sync(FULL, p2[0][j].x, LX);
                pS[j].y = __shfl_down_sync(FULL, p2[0][j].y, LX);
            }
            if constexpr (NW > 1) {   // the block's warp boundaries: rows held by the neighbouring warps
                if (ly == 0) {
#pragma unroll
                    for (int j = 0; j < NP; ++j) pN[j] = nbN[j];
                }
                if (ly == LY - 1) {
#pragma unroll
                    for (int j = 0; j < NP; ++j) pS[j] = nbS[j];
                }
            }
            // q' = -(A_i p), with (p, q') and (q', q') on two accumulator chains each
            float2 pqa = make_float2(0.f, 0.f), pqb = make_float2(0.f, 0.f);
            float2 qqa = make_float2(0.f, 0.f), qqb = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < PY; ++i)
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    // north + south; with one warp per block the block's top and bottom
                    // lane rows weight the shuffled (wrapped) value by 0
                    float2 ns;
                    if (i > 0 && i < PY - 1) ns = add2(p2[i - 1][j], p2[i + 1][j]);
                    else if constexpr (NW > 1) ns = add2(i > 0 ? p2[i - 1][j] : pN[j], i < PY - 1 ? p2[i + 1][j] : pS[j]);
                    else if (i == 0 && PY > 1) ns = fma2(fN2, pN[j], p2[i + 1][j]);
                    else if (PY > 1) ns = fma2(fS2, pS[j], p2[i - 1][j]);
                    else ns = fma2(fN2, pN[j], mul2(fS2, pS[j]));
                    const float hx = j > 0 ? p2[i][j - 1].y + p2[i][j].y : fmaf(fW, pW[i], p2[i][j].y);
                    const float hy = j < NP - 1 ? p2[i][j].x + p2[i][j + 1].x : fmaf(fE, pE[i], p2[i][j].x);
                    const float2 h = make_float2(hx, hy);
                    const float2 sum = add2(ns, h);
                    const float2 nd = add2(rpn[i], cpn[j]);
                    const float2 q = mul2(w2[i][j], fma2(nd, p2[i][j], sum));
                    q2[i][j] = q;
                    if (i & 1) {
                        pqb = fma2(p2[i][j], q, pqb);
                        qqb = fma2(q, q, qqb);
                    } else {
                        pqa = fma2(p2[i][j], q, pqa);
                        qqa = fma2(q, q, qqa);
                    }
                }
            if constexpr (NW > 1) {   // boundary rows of q' for the neighbouring warps
                if (ly == 0)
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        xq[kk & 1][0][wt][rx0 + 2 * j] = q2[0][j].x;
                        xq[kk & 1][0][wt][rx0 + 2 * j + 1] = q2[0][j].y;
                    }
                if (ly == LY - 1)
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        xq[kk & 1][1][wt][rx0 + 2 * j] = q2[PY - 1][j].x;
                        xq[kk & 1][1][wt][rx0 + 2 * j + 1] = q2[PY - 1][j].y;
                    }
            }
            const float3 sums = tile_sum3<CF>(make_float3((pqa.x + pqa.y) + (pqb.x + pqb.y),
                                                          (qqa.x + qqa.y) + (qqb.x + qqb.y), rrp),
                                              &red3[kk & 1][0][0], wt, lane);
            const float pq = -sums.x, qq = sums.y, rr = sums.z;
            if (!(pq > 1e-30f) || !(rr > 1e-30f)) break;
            // approximate quotient (2 ulp): pq lies in [1e-30, 2^126) here, where
            // __fdividef is finite, and it shortens the step's dependency chain
            const float inv = __fdividef(1.f, pq);
            const float alpha = rr * inv;
            const float beta = fmaf(alpha, qq * inv, -1.f);   // (r', r') / (r, r)
            rr_j = beta * rr;
            const float2 a2 = make_float2(alpha, alpha), b2 = make_float2(beta, beta);
            float2 rra = make_float2(0.f, 0.f), rrb = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < PY; ++i)
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    v2[i][j] = fma2(a2, p2[i][j], v2[i][j]);
                    r2[i][j] = fma2(a2, q2[i][j], r2[i][j]);     // r - alpha A p
                    if (i & 1) rrb = fma2(r2[i][j], r2[i][j], rrb); else rra = fma2(r2[i][j], r2[i][j], rra);
                }
            rrp = (rra.x + rra.y) + (rrb.x + rrb.y);
            if (kk + 1 < kcg)
#pragma unroll
                for (int i = 0; i < PY; ++i)
#pragma unroll
                    for (int j = 0; j < NP; ++j) p2[i][j] = fma2(b2, p2[i][j], r2[i][j]);
            if constexpr (NW > 1) {   // the neighbours' rows of r and p, from their q' rows (read after the barrier)
                if (ly == 0 && wt > 0)
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        const float2 qn = make_float2(xq[kk & 1][1][wt - 1][rx0 + 2 * j], xq[kk & 1][1][wt - 1][rx0 + 2 * j + 1]);
                        nrN[j] = fma2(a2, qn, nrN[j]);
                        nbN[j] = fma2(b2, nbN[j], nrN[j]);
                    }
                if (ly == LY - 1 && wt < NW - 1)
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        const float2 qs = make_float2(xq[kk & 1][0][wt + 1][rx0 + 2 * j], xq[kk & 1][0][wt + 1][rx0 + 2 * j + 1]);
                        nrS[j] = fma2(a2, qs, nrS[j]);
                        nbS[j] = fma2(b2, nbS[j], nrS[j]);
                    }
            }
        }

        if (Fp->work != nullptr && !f_probe) {   // work actually done (the local stop shortens it)
            constexpr int LB = PX * PY;
            const uint32_t un = (uint32_t)LB - (uint32_t)__popc(kb & (LB == 32 ? 0xffffffffu : ((1u << LB) - 1u)));
            work_us += un * (uint32_t)kk;
            work_u += un;
        }

        // ---- restricted add-back on the owned core -------------------------------
        if (!f_probe) {
            T* __restrict__ uout = static_cast<T*>(Fp->u_buf[f_cur ^ 1]) + (size_t)c * Fp->plane;
            const int P = Fp->pitch;
#pragma unroll
            for (int i = 0; i < PY; ++i) {
                const int o = (1 + ry0 + i) * BX + cx + rx0;
                T* const grow = uout + (size_t)(y0 + ry0 + i) * P + (x0 + rx0);
                if constexpr (ALN) {
                    const float4 u4 = *reinterpret_cast<const float4*>(U + o);
                    const float2 lo = add2(make_float2(u4.x, u4.y), v2[i][0]);
                    const float2 hi = add2(make_float2(u4.z, u4.w), v2[i][1]);
                    const uint32_t rb = ob >> (i * PX);
                    if (rb & 1u) grow[0] = lo.x;
                    if (rb & 2u) grow[1] = lo.y;
                    if (rb & 4u) grow[2] = hi.x;
                    if (rb & 8u) grow[3] = hi.y;
                } else {
#pragma unroll
                    for (int j = 0; j < PX; ++j) {
                        if ((ob >> (i * PX + j)) & 1u) {
                            const float v = (j & 1) ? v2[i][j >> 1].y : v2[i][j >> 1].x;
                            grow[j] = from_f<T>(to_f(U[o + j]) + v);
                        }
                    }
                }
            }
        }
        if constexpr (NW > 1) __syncthreads();   // the staged tile may now be refilled
        else __syncwarp();
        t = s_next[buf];
    }
    if (tt == 0 && t < total && !s_ok) {
        // a wait gave up: before leaving, wait (bounded) for this CTA's copies
        // still in flight, the one waited for and the next tile's, if issued
        const int b = it & 1;
        mbar_wait_bounded(&mbar[b], (uint32_t)((it >> 1) & 1));
        if (s_next[b] < total) mbar_wait_bounded(&mbar[b ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
    }
    if (q_pr >= 0) flush_frame();

    // ---- the launch's completion ticket: the last CTA resets the tile counter;
    // a frame whose sweep was abandoned (a wait gave up, so its tiles never all
    // completed; in a batched launch any wait abandons every frame's sweep,
    // since the CTA that gave up leaves tiles of other frames undone) gets its
    // error word set, its sequence ended and its sums cleared
    __syncthreads();
    __shared__ int s_last;
    if (tt == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1) == G - 1;
    }
    __syncthreads();
    if (s_last && tt == 0) {
        __threadfence();
        const bool launch_failed = BATCH && __ldcg(lctl + 2) != 0;
        for (int q = 0; q < n_act; ++q) {
            const SweepFrame* const F = frame_at(q);
            if ((launch_failed || __ldcg(F->err) != 0) && __ldcg(F->flag) == 0) {
                F->err[0] = 1;
                F->flag[0] = 5;
                F->flag[1] = __ldcg(F->state + 3);
                F->flag[2] = 0;
                F->flag[6] = 0;
                for (int c = 0; c < 2 * F->C; ++c) F->acc[c] = 0ull;
            }
        }
        *ticket = 0;
        *counter = 0;
        if (BATCH) lctl[2] = 0;
    }
}

constexpr int kTmaskTPB = 256;

template <class CF>
__global__ void __launch_bounds__(kTmaskTPB)
build_tmask_kernel(const uint8_t* __restrict__ mask, int mp, uint32_t* __restrict__ tmask, int H, int W, int s,
                   int half_o, int ntx, int nty, int ntiles, unsigned long long* __restrict__ count, int vec4) {
    constexpr int PX = CF::PX, PY = CF::PY, LX = CF::LX, LY = CF::LY, NT = CF::NT;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned unknown = 0;
    if (gid < (long long)ntiles * NT) {
        const int tile = (int)(gid / NT), tt = (int)(gid - (long long)tile * NT);
        const int wt = tt >> 5, lane = tt & 31, lx = lane % LX, ly = lane / LX;
        const int ty = tile / ntx, tx = tile - ty * ntx;
        const int y0 = ty * s, x0 = tx * s;
        const int th = min(CF::BH, H - y0), tw = min(CF::BW, W - x0);
        const int oy0 = ty == 0 ? 0 : y0 + half_o, oy1 = ty == nty - 1 ? H : y0 + s + half_o;
        const int ox0 = tx == 0 ? 0 : x0 + half_o, ox1 = tx == ntx - 1 ? W : x0 + s + half_o;
        const int ry0 = (wt * LY + ly) * PY, rx0 = lx * PX;
        uint32_t kb = 0, ob = 0;
        // a row's PX = 4 mask bytes as one 32-bit load where they are in the tile and aligned
        const bool row4 = PX == 4 && vec4 && ((x0 + rx0) & 3) == 0 && rx0 + PX <= tw;
        for (int i = 0; i < PY; ++i) {
            const int y = y0 + ry0 + i;
            const bool yin = ry0 + i < th;
            uint32_t bytes = 0;
            if (row4 && yin) bytes = *reinterpret_cast<const uint32_t*>(mask + (size_t)y * mp + x0 + rx0);
            for (int j = 0; j < PX; ++j) {
                const int bit = i * PX + j;
                const int x = x0 + rx0 + j;
                const bool in = yin && (rx0 + j < tw);
                const bool known = in && (row4 ? ((bytes >> (8 * j)) & 0xffu) != 0 : mask[(size_t)y * mp + x] != 0);
                if (!in || known) kb |= 1u << bit;
                if (in && y >= oy0 && y < oy1 && x >= ox0 && x < ox1) ob |= 1u << bit;
            }
        }
        tmask[(size_t)tile * 2 * NT + tt] = kb;
        tmask[(size_t)tile * 2 * NT + NT + tt] = ob;
        constexpr int LB = PX * PY;
        unknown = (unsigned)LB - (unsigned)__popc(kb & (LB == 32 ? 0xffffffffu : ((1u << LB) - 1u)));
    }
    if (count != nullptr) {   // unknown in-tile pixels, one atomic per block (uniform per launch)
        for (int m = 16; m >= 1; m >>= 1) unknown += __shfl_xor_sync(FULL, unknown, m);
        __shared__ unsigned ws[kTmaskTPB / 32];
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = unknown;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned t = 0;
            for (int w = 0; w < kTmaskTPB / 32; ++w) t += ws[w];
            if (t) atomicAdd(count, (unsigned long long)t);
        }
    }
}

// Unknown in-block pixels summed over all blocks: each thread word has PX*PY
// pixels, known-or-outside ones have their bit set.
template <class CF>
__global__ void count_unknown_kernel(const uint32_t* __restrict__ tmask, int ntiles,
                                     unsigned long long* __restrict__ out) {
    constexpr int NT = CF::NT, NPX = CF::PX * CF::PY;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned v = 0;
    if (gid < (long long)ntiles * NT) {
        const int tile = (int)(gid / NT), tt = (int)(gid - (long long)tile * NT);
        v = NPX - __popc(tmask[(size_t)tile * 2 * NT + tt]);
    }
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(FULL, v, m);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}

template <class CF, typename T>
size_t sweep_smem_bytes(bool has_g) {
    return (size_t)Box<CF, T>::STRIDE * 2 * (has_g ? 2 : 1) + 2 * mask_bytes<CF>() + 128;
}

template <class CF, typename T, bool ALN, bool BATCH, bool HASG>
int persistent_grid() {
    // CTAs per SM from the occupancy calculator, cached per instantiation (0 on
    // a failed query: the caller reports the error); also sets the kernel's
    // dynamic shared-memory limit.
    static int slot = 0;
    if (slot == 0) {
        int dev = 0, sms = 0, per = 0;
        const size_t smem = sweep_smem_bytes<CF, T>(HASG);
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaFuncSetAttribute(oras_sweep_kernel<CF, T, ALN, BATCH, HASG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, oras_sweep_kernel<CF, T, ALN, BATCH, HASG>, CF::NT,
                                                          smem) != cudaSuccess)
            return 0;
        slot = (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
    }
    return slot;
}

// The aligned variant runs when every block starts on a multiple of 4 columns
// (stride % 4 == 0) with FP32 storage and 4 pixels per lane row.
template <class CF, typename T>
constexpr bool has_aligned_variant() {
    return CF::PX == 4 && sizeof(T) == 4;
}
template <class CF, typename T>
bool use_aligned(const TileGeom& g) {
    return has_aligned_variant<CF, T>() && g.s % 4 == 0;
}

template <class CF, typename T, bool ALN, bool HASG>
cudaError_t sweep_launch(const SweepFrame& f, cudaStream_t st) {
    const long long work = (long long)f.ntiles * f.C;
    const int resident = persistent_grid<CF, T, ALN, false, HASG>();
    if (resident == 0) return cudaGetLastError();
    const long long grid = std::min<long long>(work, resident);
    const size_t smem = sweep_smem_bytes<CF, T>(HASG);
    oras_sweep_kernel<CF, T, ALN, false, HASG><<<(unsigned)grid, CF::NT, smem, st>>>(f, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

template <class CF, typename T, bool HASG>
cudaError_t sweep_cfg_g(const SweepFrame& f, const TileGeom& g, cudaStream_t st) {
    if constexpr (has_aligned_variant<CF, T>()) {
        if (use_aligned<CF, T>(g)) return sweep_launch<CF, T, true, HASG>(f, st);
    }
    return sweep_launch<CF, T, false, HASG>(f, st);
}

template <class CF, typename T>
cudaError_t sweep_cfg(const SweepFrame& f, const TileGeom& g, cudaStream_t st) {
    return f.has_g ? sweep_cfg_g<CF, T, true>(f, g, st) : sweep_cfg_g<CF, T, false>(f, g, st);
}

template <class CF, typename T, bool HASG>
int prepare_grid_g(const TileGeom& g) {
    if constexpr (has_aligned_variant<CF, T>()) {
        if (use_aligned<CF, T>(g)) return persistent_grid<CF, T, true, false, HASG>();
    }
    return persistent_grid<CF, T, false, false, HASG>();
}

template <class CF, typename T>
int prepare_grid(const TileGeom& g, bool has_g) {
    return has_g ? prepare_grid_g<CF, T, true>(g) : prepare_grid_g<CF, T, false>(g);
}

template <class CF>
cudaError_t prepare_store(Store s, const TileGeom& g, bool has_g) {
    int n = 0;
    switch (s) {
        case Store::F32: n = prepare_grid<CF, float>(g, has_g); break;
        case Store::F16: n = prepare_grid<CF, __half>(g, has_g); break;
        case Store::BF16: n = prepare_grid<CF, __nv_bfloat16>(g, has_g); break;
    }
    return n > 0 ? cudaSuccess : cudaGetLastError();
}

template <class CF>
cudaError_t sweep_store(Store s, const SweepFrame& f, const TileGeom& g, cudaStream_t st) {
    switch (s) {
        case Store::F32: return sweep_cfg<CF, float>(f, g, st);
        case Store::F16: return sweep_cfg<CF, __half>(f, g, st);
        case Store::BF16: return sweep_cfg<CF, __nv_bfloat16>(f, g, st);
    }
    return cudaErrorInvalidValue;
}

// batched launches: FP32 storage, no source term, the resident grid
template <class CF>
int batch_grid(const TileGeom& g) {
    if constexpr (has_aligned_variant<CF, float>()) {
        if (use_aligned<CF, float>(g)) return persistent_grid<CF, float, true, true, false>();
    }
    return persistent_grid<CF, float, false, true, false>();
}

template <class CF>
cudaError_t sweep_batch_cfg(const TileGeom& g, const SweepFrame* frames, const int* list, int* bctl,
                            cudaStream_t st) {
    const int grid = batch_grid<CF>(g);
    if (grid == 0) return cudaGetLastError();
    const size_t smem = sweep_smem_bytes<CF, float>(false);
    SweepFrame none{};
    if constexpr (has_aligned_variant<CF, float>()) {
        if (use_aligned<CF, float>(g)) {
            oras_sweep_kernel<CF, float, true, true, false><<<(unsigned)grid, CF::NT, smem, st>>>(none, frames, list,
                                                                                               bctl);
            return cudaGetLastError();
        }
    }
    oras_sweep_kernel<CF, float, false, true, false><<<(unsigned)grid, CF::NT, smem, st>>>(none, frames, list, bctl);
    return cudaGetLastError();
}

// ---- batched levels: list building, resets and result records (one thread per frame or one thread) ----
__global__ void batch_ctl_kernel(const SweepFrame* __restrict__ fr, int n, int* __restrict__ list,
                                 int* __restrict__ ctl, int max_passes, cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0) return;
    const int passes = ctl[0] + 1;
    ctl[0] = passes;
    int m = 0, tiles = 0;
    if (passes <= max_passes)
        for (int f = 0; f < n; ++f) {
            const SweepFrame& F = fr[f];
            if (F.flag[0] != 0 || F.state[1] >= F.cap) continue;
            list[1 + m] = f;
            ++m;
        }
    list[0] = m;
    for (int q = 0; q < m; ++q) {
        const SweepFrame& F = fr[list[1 + q]];
        list[1 + m + q] = tiles;
        tiles += F.ntiles * F.C;
    }
    list[1 + 2 * m] = tiles;
    if (m == 0) cudaGraphSetConditional(cond, 0);
}

__global__ void batch_reset_kernel(const SweepFrame* __restrict__ fr, int n) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const SweepFrame& F = fr[f];
    for (int i = 0; i < 4; ++i) F.state[i] = 0;
    for (int i = 0; i < 5; ++i) F.flag[i] = 0;
    F.flag[6] = 0;
    *const_cast<double*>(F.tol) = F.level_tol;
}

__global__ void batch_resolve_kernel(const SweepFrame* __restrict__ fr, int n, const int* __restrict__ ctl) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const SweepFrame& F = fr[f];
    int* const out = F.resolve_out;
    out[0] = F.state[0];
    out[1] = F.state[1];
    out[2] = F.flag[0];
    out[3] = ctl[0];
}

template <class CF>
cudaError_t tmask_cfg(const TileGeom& g, const uint8_t* mask, int mp, uint32_t* tmask, cudaStream_t st,
                      unsigned long long* count) {
    const long long n = (long long)g.ntiles * CF::NT;
    const int vec4 = (reinterpret_cast<uintptr_t>(mask) & 3u) == 0 && (mp & 3) == 0;
    build_tmask_kernel<CF><<<(unsigned)((n + kTmaskTPB - 1) / kTmaskTPB), kTmaskTPB, 0, st>>>(
        mask, mp, tmask, g.H, g.W, g.s, g.half_o, g.ntx, g.nty, g.ntiles, count, vec4);
    return cudaGetLastError();
}

template <class CF>
cudaError_t count_cfg(const TileGeom& g, const uint32_t* tmask, unsigned long long* out, cudaStream_t st) {
    const long long n = (long long)g.ntiles * CF::NT;
    const int tpb = 256;
    count_unknown_kernel<CF><<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(tmask, g.ntiles, out);
    return cudaGetLastError();
}

template <class CF, typename T>
void box_dims(int* bx, int* by) {
    *bx = Box<CF, T>::BX;
    *by = Box<CF, T>::BY;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

int axis_blocks(int n, int b, int o) {
    const int s = b - o;
    const int m = n - o;
    const int cnt = m <= 0 ? 1 : (m + s - 1) / s;
    return cnt < 1 ? 1 : cnt;
}

TileGeom make_geom(int H, int W, int pitch, int b, int o, int nw) {
    TileGeom g;
    g.H = H; g.W = W; g.pitch = pitch;
    g.b = b; g.o = o; g.s = b - o; g.half_o = o / 2;
    g.nw = nw > 0 ? nw : default_tile_warps(b);
    g.ntx = axis_blocks(W, b, o);
    g.nty = axis_blocks(H, b, o);
    g.ntiles = g.ntx * g.nty;
    return g;
}

bool block_supported(int b) { return b == 16 || b == 32 || b == 64 || b == 96; }

int default_tile_warps(int b) { return b == 96 ? 12 : b == 64 ? 4 : 1; }

bool tile_warps_supported(int b, int nw) {
    return with_cfg(b, nw, [](auto) { return cudaSuccess; }) == cudaSuccess;
}

int tile_threads(int b, int nw) {
    int nt = 0;
    with_cfg(b, nw, [&](auto cfg) {
        nt = decltype(cfg)::NT;
        return cudaSuccess;
    });
    return nt;
}

size_t tmask_words(const TileGeom& g) { return (size_t)g.ntiles * 2 * tile_threads(g.b, g.nw); }

cudaError_t make_tile_map(CUtensorMap* out, Store s, const void* base, int H, int W, int pitch, int C, int b) {
    int bx = 0, by = 0;
    const cudaError_t e = with_cfg(b, default_tile_warps(b), [&](auto cfg) {
        using CF = decltype(cfg);
        switch (s) {
            case Store::F32: box_dims<CF, float>(&bx, &by); break;
            case Store::F16: box_dims<CF, __half>(&bx, &by); break;
            case Store::BF16: box_dims<CF, __nv_bfloat16>(&bx, &by); break;
        }
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    auto fn = encode_fn();
    if (fn == nullptr) return cudaErrorNotSupported;
    const size_t es = store_bytes(s);
    const CUtensorMapDataType dt = s == Store::F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : s == Store::F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)C};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)pitch * H * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(out, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_build_tmask(const TileGeom& g, const uint8_t* mask, int mp, uint32_t* tmask,
                               cudaStream_t st, unsigned long long* count) {
    return with_cfg(g.b, g.nw, [&](auto cfg) { return tmask_cfg<decltype(cfg)>(g, mask, mp, tmask, st, count); });
}

cudaError_t launch_count_unknown(const TileGeom& g, const uint32_t* tmask, unsigned long long* out,
                                 cudaStream_t st) {
    return with_cfg(g.b, g.nw, [&](auto cfg) { return count_cfg<decltype(cfg)>(g, tmask, out, st); });
}

cudaError_t prepare_sweep(Store s, const TileGeom& g, bool has_g) {
    return with_cfg(g.b, g.nw, [&](auto cfg) { return prepare_store<decltype(cfg)>(s, g, has_g); });
}

FastDiv make_fastdiv(uint32_t d) {
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    return FastDiv{(uint32_t)(((1ull << 32) * ((1ull << s) - d)) / d + 1), s};
}

namespace {

// The descriptor of one frame's sweep: geometry, buffers and stop words.
cudaError_t make_frame(SweepFrame* f, const TileGeom& g, int C, long long plane, const SweepPair& pair,
                       const CUtensorMap* map_g, const uint32_t* tmask, const SweepStop& stop, float p_robin,
                       int k, float local_rtol) {
    if (!(local_rtol >= 0.f) || !(local_rtol < 1.f)) return cudaErrorInvalidValue;
    if (stop.acc == nullptr || stop.flag == nullptr || stop.norms2 == nullptr || stop.ref == nullptr ||
        stop.state == nullptr || stop.err == nullptr || stop.tol == nullptr || stop.stall_polls < 0 ||
        pair.map[0] == nullptr || pair.map[1] == nullptr || pair.u[0] == nullptr || pair.u[1] == nullptr ||
        tmask == nullptr || C < 1 || (long long)g.ntiles * C >= (1LL << 31))
        return cudaErrorInvalidValue;
    std::memset(static_cast<void*>(f), 0, sizeof(*f));
    f->map_u[0] = *pair.map[0];
    f->map_u[1] = *pair.map[1];
    f->map_g = map_g ? *map_g : *pair.map[0];
    f->u_buf[0] = pair.u[0];
    f->u_buf[1] = pair.u[1];
    f->tmask = tmask;
    f->acc = stop.acc;
    f->norms2 = stop.norms2;
    f->ref = stop.ref;
    f->tol = stop.tol;
    f->flag = stop.flag;
    f->state = stop.state;
    f->err = stop.err;
    f->work = stop.work;
    f->stall = stop.stall;
    f->plane = plane;
    f->dv_tiles = make_fastdiv((uint32_t)g.ntiles);
    f->dv_ntx = make_fastdiv((uint32_t)g.ntx);
    f->H = g.H; f->W = g.W; f->pitch = g.pitch; f->C = C;
    f->s = g.s; f->ntx = g.ntx; f->ntiles = g.ntiles;
    f->has_g = map_g != nullptr ? 1 : 0;
    f->p_robin = p_robin;
    f->local_rtol2 = local_rtol * local_rtol;
    f->local_rtol2_final = stop.final_local_rtol > 0.f ? stop.final_local_rtol * stop.final_local_rtol : 0.f;
    f->local_atol2 = stop.local_atol > 0.f ? stop.local_atol * stop.local_atol : 0.f;
    f->k = k;
    f->stall_polls = stop.stall_polls;
    f->force_probe = stop.force_probe;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_sweep(Store s, const TileGeom& g, int C, long long plane, const SweepPair& pair,
                         const CUtensorMap* map_g, const uint32_t* tmask, const SweepStop& stop, float p_robin,
                         int k, cudaStream_t st, float local_rtol) {
    SweepFrame f;
    const cudaError_t e = make_frame(&f, g, C, plane, pair, map_g, tmask, stop, p_robin, k, local_rtol);
    if (e != cudaSuccess) return e;
    return with_cfg(g.b, g.nw, [&](auto cfg) { return sweep_store<decltype(cfg)>(s, f, g, st); });
}

void fill_sweep_frame(SweepFrame* out, const TileGeom& g, int C, long long plane, const SweepPair& pair,
                      const uint32_t* tmask, const SweepStop& stop, float p_robin, int k, float local_rtol, int cap,
                      int* resolve_out) {
    if (make_frame(out, g, C, plane, pair, nullptr, tmask, stop, p_robin, k, local_rtol) != cudaSuccess)
        std::memset(static_cast<void*>(out), 0, sizeof(*out));
    out->cap = cap;
    out->resolve_out = resolve_out;
}

cudaError_t prepare_sweep_batch(const TileGeom& g) {
    return with_cfg(g.b, g.nw, [&](auto cfg) { return batch_grid<decltype(cfg)>(g) > 0 ? cudaSuccess : cudaGetLastError(); });
}

cudaError_t launch_sweep_batch(const TileGeom& g, const SweepFrame* frames, const int* list, int* bctl,
                               cudaStream_t st) {
    if (frames == nullptr || list == nullptr || bctl == nullptr) return cudaErrorInvalidValue;
    return with_cfg(g.b, g.nw, [&](auto cfg) { return sweep_batch_cfg<decltype(cfg)>(g, frames, list, bctl, st); });
}

cudaError_t launch_batch_ctl(const SweepFrame* frames, int n, int* list, int* ctl, int max_passes,
                             cudaGraphConditionalHandle cond, cudaStream_t st) {
    if (n < 0 || n > kBatchMaxFrames) return cudaErrorInvalidValue;
    batch_ctl_kernel<<<1, 32, 0, st>>>(frames, n, list, ctl, max_passes, cond);
    return cudaGetLastError();
}

cudaError_t launch_batch_reset(const SweepFrame* frames, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    batch_reset_kernel<<<(n + 127) / 128, 128, 0, st>>>(frames, n);
    return cudaGetLastError();
}

cudaError_t launch_batch_resolve(const SweepFrame* frames, int n, const int* ctl, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    batch_resolve_kernel<<<(n + 127) / 128, 128, 0, st>>>(frames, n, ctl);
    return cudaGetLastError();
}

}  // namespace dd
