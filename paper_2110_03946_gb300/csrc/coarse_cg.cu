// Small-grid coarse solve: conjugate gradients on the coarsest level of the
// multilevel hierarchy (Sec. 4; the coarse problem is the inpainting operator
// of Sec. 2 on that grid), one CTA per channel with the whole grid resident in
// shared memory.
//
// The coarse-grid correction (DD_ML_CORRECTION) needs the solution of
//   A_c e = g,  e = 0 on coarse-known pixels,
// where A_c is the reduced operator of Eq. eq:ls on the coarse grid (5-point
// stencil with h = 1, reflecting image borders).  On a grid of at most
// kCoarseCgMaxPixels pixels the four CG vectors (e, r, p, q; FP32) and the
// mask fit in one SM's shared memory, so an iteration is a stencil pass over
// shared memory and two block-wide reductions: no grid-wide synchronisation and
// no launch per iteration.  Dot products, alpha and beta are FP64 (the CG
// recurrences stay stable to a small relative residual even on FP32 vectors).
// CG stops at ||r|| <= tol ||g|| or after max_iter iterations (every loop is
// bounded), from e = 0.
#include <cuda_runtime.h>

#include "dd_internal.h"

namespace dd {

namespace {

constexpr int kCcThreads = 1024;
constexpr int kCcWarps = kCcThreads / 32;

// sum over the block of v, returned to every thread; sh: kCcWarps doubles,
// reused only after the barrier that ends this call
__device__ __forceinline__ double cc_block_sum(double v, double* sh, double* out) {
    const int t = threadIdx.x;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    if (t < 32) {
        double s = sh[t];   // kCcWarps == 32: one value per lane, summed in a fixed order
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
        if (t == 0) *out = s;
    }
    __syncthreads();
    return *out;
}

__global__ void __launch_bounds__(kCcThreads)
coarse_cg_kernel(int H, int W, const uint8_t* __restrict__ mask, int mp, const float* __restrict__ g, int gp,
                 long long gplane, float* __restrict__ e, int ep, long long eplane, int max_iter, double tol,
                 int* __restrict__ iters_out, const int* __restrict__ skip) {
    if (skip != nullptr && *skip != 0) return;   // uniform
    extern __shared__ __align__(16) unsigned char cc_smem[];
    __shared__ double red[kCcWarps];
    __shared__ double res;
    const int N = H * W;
    float* const x = reinterpret_cast<float*>(cc_smem);
    float* const r = x + N;
    float* const p = r + N;
    float* const q = p + N;
    uint8_t* const known = reinterpret_cast<uint8_t*>(q + N);
    const int c = blockIdx.x;
    const float* __restrict__ gc = g + (long long)c * gplane;
    float* __restrict__ ec = e + (long long)c * eplane;
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;

    // e = 0; r = g on unknown pixels (0 on known ones); p = r
    double rr_part = 0.0;
    for (int y = wp; y < H; y += kCcWarps)
        for (int xx = lane; xx < W; xx += 32) {
            const int i = y * W + xx;
            const uint8_t k = mask[(long long)y * mp + xx] != 0;
            known[i] = k;
            const float rv = k ? 0.f : gc[(long long)y * gp + xx];
            x[i] = 0.f;
            r[i] = rv;
            p[i] = rv;
            rr_part += (double)rv * rv;
        }
    double rr = cc_block_sum(rr_part, red, &res);   // its barrier also publishes the arrays
    const double stop = tol * tol * rr;
    int it = 0;
    for (; it < max_iter; ++it) {
        if (!(rr > stop) || !(rr > 0.0)) break;   // uniform (every thread holds the same rr)
        // q = A_c p on unknown pixels: sum over in-image neighbours of (p_i - p_j); p = 0 on known pixels
        double pq_part = 0.0;
        for (int y = wp; y < H; y += kCcWarps)
            for (int xx = lane; xx < W; xx += 32) {
                const int i = y * W + xx;
                float qv = 0.f;
                if (!known[i]) {
                    const float pi = p[i];
                    if (xx > 0) qv += pi - p[i - 1];
                    if (xx < W - 1) qv += pi - p[i + 1];
                    if (y > 0) qv += pi - p[i - W];
                    if (y < H - 1) qv += pi - p[i + W];
                    pq_part += (double)pi * qv;
                }
                q[i] = qv;
            }
        const double pq = cc_block_sum(pq_part, red, &res);
        if (!(pq > 0.0)) break;   // uniform: p is in the null space only if r = 0
        const double alpha = rr / pq;
        const float af = (float)alpha;
        double rn_part = 0.0;
        for (int y = wp; y < H; y += kCcWarps)
            for (int xx = lane; xx < W; xx += 32) {
                const int i = y * W + xx;
                x[i] = fmaf(af, p[i], x[i]);
                const float rv = fmaf(-af, q[i], r[i]);
                r[i] = rv;
                rn_part += (double)rv * rv;
            }
        const double rr_new = cc_block_sum(rn_part, red, &res);
        const float bf = (float)(rr_new / rr);
        rr = rr_new;
        for (int y = wp; y < H; y += kCcWarps)
            for (int xx = lane; xx < W; xx += 32) {
                const int i = y * W + xx;
                p[i] = fmaf(bf, p[i], r[i]);
            }
        __syncthreads();
    }
    for (int y = wp; y < H; y += kCcWarps)
        for (int xx = lane; xx < W; xx += 32) ec[(long long)y * ep + xx] = x[y * W + xx];
    if (t == 0 && iters_out != nullptr) iters_out[c] = it;
}

}  // namespace

size_t coarse_cg_smem_bytes(int H, int W) {
    const size_t n = (size_t)H * W;
    return n * 4 * sizeof(float) + (n + 15) / 16 * 16;
}

cudaError_t prepare_coarse_cg() {
    return cudaFuncSetAttribute(coarse_cg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)coarse_cg_smem_bytes(kCoarseCgMaxPixels, 1));
}

cudaError_t launch_coarse_cg(int H, int W, int C, const uint8_t* mask, int mp, const float* g, int gp,
                             long long gplane, float* e, int ep, long long eplane, int max_iter, double tol,
                             int* iters, const int* skip, cudaStream_t st) {
    if (H < 1 || W < 1 || C < 1 || (long long)H * W > kCoarseCgMaxPixels || max_iter < 0 || !(tol >= 0.0) ||
        mask == nullptr || g == nullptr || e == nullptr || mp < W || gp < W || ep < W)
        return cudaErrorInvalidValue;
    const size_t smem = coarse_cg_smem_bytes(H, W);
    coarse_cg_kernel<<<C, kCcThreads, smem, st>>>(H, W, mask, mp, g, gp, gplane, e, ep, eplane, max_iter, tol, iters,
                                                  skip);
    return cudaGetLastError();
}

}  // namespace dd
