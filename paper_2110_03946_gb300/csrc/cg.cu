// Conjugate gradients on the whole image: the comparison solver of the paper's
// experiments (Sec. 5: CG and the multilevel CG of Bornemann & Deuflhard,
// [BD96], against which ORAS is measured).
//
// CG runs on the unknown pixels of A u = b (Sec. 2), per channel, with x held
// in the level's iterate buffer (known pixels keep u = f; r = p = q = 0 there).
// One iteration is two HBM-streaming kernels:
//   cg_apply:  p <- r + beta p (formed on the fly for the pixel and its four
//              neighbours, written to the other p buffer), q = A p, (p, q);
//   cg_update: x += alpha p, r -= alpha q, (r, r).
// Each kernel's last block (atomic ticket) reduces the per-block partials of
// every channel in a fixed order and computes alpha, or beta and the stop test
// (max over channels of sqrt((r, r)) / ||b - A u0|| <= tol), so iterations run
// back to back without the host; launches after the stop return at once.
#include <cuda_runtime.h>

#include "dd_internal.h"

namespace dd {

namespace {

constexpr int CG_TX = 32, CG_TY = 8, CG_ROWS = 8;   // a block covers 32 x 64 pixels
constexpr int CG_THREADS = CG_TX * CG_TY;

// sum over the block of v (double), result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int t = threadIdx.y * CG_TX + threadIdx.x;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (t == 0)
        for (int w = 0; w < CG_THREADS / 32; ++w) s += sh[w];
    return s;
}

// Whether this block is the last of the grid to finish (ticket in *ticket).
__device__ __forceinline__ bool last_block(int* ticket, int* s_last) {
    __threadfence();
    __syncthreads();
    const int t = threadIdx.y * CG_TX + threadIdx.x;
    if (t == 0) *s_last = atomicAdd(ticket, 1) == (int)(gridDim.x * gridDim.y * gridDim.z) - 1;
    __syncthreads();
    return *s_last != 0;
}

// Per-channel sum of the partials part[c * nblk + i] by one block, fixed order.
__device__ double channel_sum(const double* part, int c, int nblk, double* sh) {
    const int t = threadIdx.y * CG_TX + threadIdx.x;
    double v = 0.0;
    for (int i = t; i < nblk; i += CG_THREADS) v += __ldcg(part + (size_t)c * nblk + i);
    const double s = block_sum(v, sh);
    __syncthreads();
    return s;   // valid in thread 0
}

__global__ void __launch_bounds__(CG_THREADS) cg_apply_kernel(CGArgs a) {
    if (a.flag[0] != 0) return;
    const int c = blockIdx.z;
    const int x = blockIdx.x * CG_TX + threadIdx.x;
    const int yb = blockIdx.y * (CG_TY * CG_ROWS) + threadIdx.y * CG_ROWS;
    const float beta = a.first ? 0.f : (float)a.scal[2 * a.C + c];
    const long long base = (long long)c * a.plane;
    const float* __restrict__ r = a.r + base;
    const float* __restrict__ po = a.p_old + base;
    float* __restrict__ pn = a.p_new + base;
    float* __restrict__ q = a.q + base;
    const bool xin = x < a.W;
    // p = r + beta p_old for this column, rows yb-1 .. yb+CG_ROWS (0 outside the
    // image and on known pixels); horizontal neighbours come from the next lanes
    auto pval = [&](int y, int xx) -> float {
        if (y < 0 || y >= a.H || xx < 0 || xx >= a.W) return 0.f;
        const size_t o = (size_t)y * a.P + xx;
        return a.mask[(size_t)y * a.mp + xx] ? 0.f : fmaf(beta, po[o], r[o]);
    };
    float col[CG_ROWS + 2];
#pragma unroll
    for (int k = 0; k < CG_ROWS + 2; ++k) col[k] = xin ? pval(yb - 1 + k, x) : 0.f;
    float pq = 0.f;
#pragma unroll
    for (int k = 0; k < CG_ROWS; ++k) {
        const int y = yb + k;
        const float pc = col[k + 1];
        float left = __shfl_up_sync(0xffffffffu, pc, 1);
        float right = __shfl_down_sync(0xffffffffu, pc, 1);
        if (threadIdx.x == 0) left = pval(y, x - 1);
        if (threadIdx.x == CG_TX - 1) right = pval(y, x + 1);
        if (!xin || y >= a.H) continue;
        const size_t o = (size_t)y * a.P + x;
        pn[o] = pc;
        if (a.mask[(size_t)y * a.mp + x]) {
            q[o] = 0.f;
            continue;
        }
        const float deg = (float)((y > 0) + (y < a.H - 1) + (x > 0) + (x < a.W - 1));
        const float qv = fmaf(deg, pc, -((col[k] + col[k + 2]) + (left + right)));
        q[o] = qv;
        pq = fmaf(pc, qv, pq);
    }
    __shared__ double sh[CG_THREADS / 32];
    __shared__ int s_last;
    const double s = block_sum((double)pq, sh);
    const int nblk = gridDim.x * gridDim.y;
    if (threadIdx.x == 0 && threadIdx.y == 0) a.part[(size_t)c * nblk + blockIdx.y * gridDim.x + blockIdx.x] = s;
    if (!last_block(a.flag + 3, &s_last)) return;
    __threadfence();
    for (int cc = 0; cc < a.C; ++cc) {
        const double pqc = channel_sum(a.part, cc, nblk, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double rr = a.scal[cc];
            a.scal[a.C + cc] = (pqc > 0.0 && rr > 0.0) ? rr / pqc : 0.0;   // alpha
        }
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) a.flag[3] = 0;
}

__global__ void __launch_bounds__(CG_THREADS) cg_update_kernel(CGArgs a) {
    if (a.flag[0] != 0) return;
    const int c = blockIdx.z;
    const int x = blockIdx.x * CG_TX + threadIdx.x;
    const int yb = blockIdx.y * (CG_TY * CG_ROWS) + threadIdx.y * CG_ROWS;
    const float alpha = (float)a.scal[a.C + c];
    const long long base = (long long)c * a.plane;
    float* __restrict__ xv = a.x + base;
    float* __restrict__ r = a.r + base;
    const float* __restrict__ p = a.p_new + base;
    const float* __restrict__ q = a.q + base;
    float rr = 0.f;
    if (x < a.W) {
        for (int k = 0; k < CG_ROWS; ++k) {
            const int y = yb + k;
            if (y >= a.H) break;
            if (a.mask[(size_t)y * a.mp + x]) continue;
            const size_t o = (size_t)y * a.P + x;
            xv[o] = fmaf(alpha, p[o], xv[o]);
            const float rn = fmaf(-alpha, q[o], r[o]);
            r[o] = rn;
            rr = fmaf(rn, rn, rr);
        }
    }
    __shared__ double sh[CG_THREADS / 32];
    __shared__ int s_last;
    const double s = block_sum((double)rr, sh);
    const int nblk = gridDim.x * gridDim.y;
    if (threadIdx.x == 0 && threadIdx.y == 0) a.part[(size_t)c * nblk + blockIdx.y * gridDim.x + blockIdx.x] = s;
    if (!last_block(a.flag + 3, &s_last)) return;
    __threadfence();
    double worst = 0.0;
    int bad = 0;
    for (int cc = 0; cc < a.C; ++cc) {
        const double rrn = channel_sum(a.part, cc, nblk, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double rro = a.scal[cc];
            a.scal[2 * a.C + cc] = rro > 0.0 ? rrn / rro : 0.0;   // beta
            a.scal[cc] = rrn;
            if (!isfinite(rrn)) bad = 1;
            const double den = a.ref[cc] > 0.0 ? a.ref[cc] : 1.0;
            worst = fmax(worst, sqrt(rrn) / den);
        }
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        a.state[1] += 1;   // iterations applied
        if (bad) { a.flag[0] = 2; a.flag[1] = a.iter; }
        else if (worst <= a.tol) { a.flag[0] = 1; a.flag[1] = a.iter; }
        a.flag[3] = 0;
    }
}

// scal[c] = (r, r) from the residual pass, beta = 0.
__global__ void cg_init_kernel(const double2* __restrict__ res_out, double* __restrict__ scal, int C) {
    const int c = threadIdx.x;
    if (c < C) {
        scal[c] = res_out[c].x;
        scal[C + c] = 0.0;
        scal[2 * C + c] = 0.0;
    }
}

dim3 cg_grid(int H, int W, int C) {
    return dim3((W + CG_TX - 1) / CG_TX, (H + CG_TY * CG_ROWS - 1) / (CG_TY * CG_ROWS), C);
}

}  // namespace

int cg_blocks(int H, int W) {
    const dim3 g = cg_grid(H, W, 1);
    return (int)(g.x * g.y);
}

cudaError_t launch_cg_init(const double2* res_out, double* scal, int C, cudaStream_t st) {
    cg_init_kernel<<<1, 32, 0, st>>>(res_out, scal, C);
    return cudaGetLastError();
}

cudaError_t launch_cg_iteration(const CGArgs& a, cudaStream_t st) {
    if (a.C > 32) return cudaErrorInvalidValue;
    const dim3 grid = cg_grid(a.H, a.W, a.C);
    const dim3 block(CG_TX, CG_TY);
    cg_apply_kernel<<<grid, block, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cg_update_kernel<<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace dd
