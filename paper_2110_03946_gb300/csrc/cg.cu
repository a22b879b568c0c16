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
// The iteration index (and with it beta = 0 on the first iteration and the
// choice of p buffers) is read from device state, so an iteration's two
// launches are the same every time and can repeat in a graph loop.
// Each kernel's last block (atomic ticket) reduces the per-block partials of
// every channel in a fixed order and computes alpha, or beta and the stop test
// (max over channels of sqrt((r, r)) / ||b - A u0|| <= tol), so iterations run
// back to back without the host; launches after the stop return at once.
#include <cuda_runtime.h>

#include "dd_internal.h"

namespace dd {

namespace {

// A thread owns 4 consecutive pixels (one float4; the pitch is a multiple of 32
// floats) in each of CG_ROWS rows; a warp covers 128 columns, a block 128 x 64.
constexpr int CG_TX = 32, CG_TY = 8, CG_ROWS = 8, CG_VEC = 4;
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
// Called after thread 0 wrote the block's partial: its fence orders that write
// before the ticket.
__device__ __forceinline__ bool last_block(int* ticket, int* s_last) {
    const int t = threadIdx.y * CG_TX + threadIdx.x;
    if (t == 0) {
        __threadfence();
        *s_last = atomicAdd(ticket, 1) == (int)(gridDim.x * gridDim.y * gridDim.z) - 1;
    }
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

// Known pixels carry r = p = q = 0 throughout (the residual pass writes r = 0
// there and both kernels preserve it), so p = r + beta p_old needs no mask; the
// mask only zeroes q.  Columns at or beyond W are zeroed explicitly, whatever
// the pitch padding holds.
__global__ void __launch_bounds__(CG_THREADS) cg_apply_kernel(CGArgs a) {
    if (a.flag[0] != 0) return;
    const int c = blockIdx.z;
    const int x0 = (blockIdx.x * CG_TX + threadIdx.x) * CG_VEC;
    const int yb = (blockIdx.y * CG_TY + threadIdx.y) * CG_ROWS;
    const int it = __ldcg(a.state + 1);   // iterations applied before this one
    const float beta = it == 0 ? 0.f : (float)a.scal[2 * a.C + c];
    const long long base = (long long)c * a.plane;
    const float* __restrict__ r = a.r + base;
    const float* __restrict__ po = a.p[it & 1] + base;
    float* __restrict__ pn = a.p[(it + 1) & 1] + base;
    float* __restrict__ q = a.q + base;
    const bool xin = x0 < a.W;
    auto prow = [&](int y) -> float4 {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (xin && y >= 0 && y < a.H) {
            const size_t o = (size_t)y * a.P + x0;
            const float4 rv = *reinterpret_cast<const float4*>(r + o);
            const float4 pv = *reinterpret_cast<const float4*>(po + o);
            v.x = fmaf(beta, pv.x, rv.x);
            v.y = x0 + 1 < a.W ? fmaf(beta, pv.y, rv.y) : 0.f;
            v.z = x0 + 2 < a.W ? fmaf(beta, pv.z, rv.z) : 0.f;
            v.w = x0 + 3 < a.W ? fmaf(beta, pv.w, rv.w) : 0.f;
        }
        return v;
    };
    auto pone = [&](int y, int xx) -> float {
        if (y < 0 || y >= a.H || xx < 0 || xx >= a.W) return 0.f;
        const size_t o = (size_t)y * a.P + xx;
        return fmaf(beta, po[o], r[o]);
    };
    float4 col[CG_ROWS + 2];
#pragma unroll
    for (int k = 0; k < CG_ROWS + 2; ++k) col[k] = prow(yb - 1 + k);
    const float dx0 = (float)((x0 > 0) + (x0 < a.W - 1));
    const float dx1 = (float)(1 + (x0 + 1 < a.W - 1));
    const float dx2 = (float)(1 + (x0 + 2 < a.W - 1));
    const float dx3 = (float)(1 + (x0 + 3 < a.W - 1));
    float pq = 0.f;
#pragma unroll
    for (int k = 0; k < CG_ROWS; ++k) {
        const int y = yb + k;
        const float4 pc = col[k + 1], pu = col[k], pd = col[k + 2];
        float left = __shfl_up_sync(0xffffffffu, pc.w, 1);
        float right = __shfl_down_sync(0xffffffffu, pc.x, 1);
        if (threadIdx.x == 0) left = pone(y, x0 - 1);
        if (threadIdx.x == CG_TX - 1) right = pone(y, x0 + CG_VEC);
        if (!xin || y >= a.H) continue;
        const float dy = (float)((y > 0) + (y < a.H - 1));
        const unsigned char* mr = a.mask + (size_t)y * a.mp + x0;
        const bool u0 = !mr[0];
        const bool u1 = x0 + 1 < a.W && !mr[1];
        const bool u2 = x0 + 2 < a.W && !mr[2];
        const bool u3 = x0 + 3 < a.W && !mr[3];
        float4 qv;
        qv.x = u0 ? fmaf(dy + dx0, pc.x, -((pu.x + pd.x) + (left + pc.y))) : 0.f;
        qv.y = u1 ? fmaf(dy + dx1, pc.y, -((pu.y + pd.y) + (pc.x + pc.z))) : 0.f;
        qv.z = u2 ? fmaf(dy + dx2, pc.z, -((pu.z + pd.z) + (pc.y + pc.w))) : 0.f;
        qv.w = u3 ? fmaf(dy + dx3, pc.w, -((pu.w + pd.w) + (pc.z + right))) : 0.f;
        const size_t o = (size_t)y * a.P + x0;
        *reinterpret_cast<float4*>(pn + o) = pc;
        *reinterpret_cast<float4*>(q + o) = qv;
        pq = fmaf(pc.x, qv.x, pq);
        pq = fmaf(pc.y, qv.y, pq);
        pq = fmaf(pc.z, qv.z, pq);
        pq = fmaf(pc.w, qv.w, pq);
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

// x += alpha p, r -= alpha q on whole float4s: on known pixels p = q = 0 leaves
// x and r (= 0) as they are; columns at or beyond W stay out of (r, r).
__global__ void __launch_bounds__(CG_THREADS) cg_update_kernel(CGArgs a) {
    if (a.flag[0] != 0) return;
    const int c = blockIdx.z;
    const int x0 = (blockIdx.x * CG_TX + threadIdx.x) * CG_VEC;
    const int yb = (blockIdx.y * CG_TY + threadIdx.y) * CG_ROWS;
    const int it = __ldcg(a.state + 1);   // incremented by this launch's last block
    const float alpha = (float)a.scal[a.C + c];
    const long long base = (long long)c * a.plane;
    float* __restrict__ xv = a.x + base;
    float* __restrict__ r = a.r + base;
    const float* __restrict__ p = a.p[(it + 1) & 1] + base;
    const float* __restrict__ q = a.q + base;
    float rr = 0.f;
    if (x0 < a.W) {
        const bool in1 = x0 + 1 < a.W, in2 = x0 + 2 < a.W, in3 = x0 + 3 < a.W;
#pragma unroll
        for (int k = 0; k < CG_ROWS; ++k) {
            const int y = yb + k;
            if (y >= a.H) break;
            const size_t o = (size_t)y * a.P + x0;
            float4 xo = *reinterpret_cast<const float4*>(xv + o);
            float4 ro = *reinterpret_cast<const float4*>(r + o);
            const float4 pv = *reinterpret_cast<const float4*>(p + o);
            const float4 qv = *reinterpret_cast<const float4*>(q + o);
            xo.x = fmaf(alpha, pv.x, xo.x); xo.y = fmaf(alpha, pv.y, xo.y);
            xo.z = fmaf(alpha, pv.z, xo.z); xo.w = fmaf(alpha, pv.w, xo.w);
            ro.x = fmaf(-alpha, qv.x, ro.x); ro.y = fmaf(-alpha, qv.y, ro.y);
            ro.z = fmaf(-alpha, qv.z, ro.z); ro.w = fmaf(-alpha, qv.w, ro.w);
            *reinterpret_cast<float4*>(xv + o) = xo;
            *reinterpret_cast<float4*>(r + o) = ro;
            rr = fmaf(ro.x, ro.x, rr);
            rr = in1 ? fmaf(ro.y, ro.y, rr) : rr;
            rr = in2 ? fmaf(ro.z, ro.z, rr) : rr;
            rr = in3 ? fmaf(ro.w, ro.w, rr) : rr;
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
    const double tol = __ldcg(a.tol);
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
        a.state[1] = it + 1;   // iterations applied
        if (bad) { a.flag[0] = 2; a.flag[1] = it; }
        else if (worst <= tol) { a.flag[0] = 1; a.flag[1] = it; }
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
    const int cols = CG_TX * CG_VEC, rows = CG_TY * CG_ROWS;
    return dim3((W + cols - 1) / cols, (H + rows - 1) / rows, C);
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
