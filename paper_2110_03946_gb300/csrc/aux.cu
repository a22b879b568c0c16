// Auxiliary passes of the ORAS solver: data packing, the residual of the
// outer correction and its norm reductions, the
// dyadic mask/value subsampling and the coarse-to-fine prolongation of the
// multilevel method (Sec. 4 of Kaemper & Weickert, arXiv 2110.03946).
// All are HBM-bound streaming passes: one thread per pixel (or per output
// pixel), rows on the fast grid axis so warps read consecutive addresses.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cfloat>

#include "dd_internal.h"

namespace dd {

namespace {

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

constexpr int TX = 32, TY = 8;   // 2-D pass block: one warp per row segment

dim3 grid2d(int H, int W, int C) { return dim3((W + TX - 1) / TX, (H + TY - 1) / TY, C); }

__global__ void masked_copy_kernel(int H, int W, const float* __restrict__ src, int sp, long long splane,
                                   const uint8_t* __restrict__ mask, int mp, float* __restrict__ dst,
                                   int dp, long long dplane) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (x >= W || y >= H) return;
    const float v = mask[(size_t)y * mp + x] ? src[c * splane + (size_t)y * sp + x] : 0.f;
    dst[c * dplane + (size_t)y * dp + x] = v;
}

__global__ void copy2d_kernel(int H, int W, const float* __restrict__ src, int sp, long long splane,
                              float* __restrict__ dst, int dp, long long dplane) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (x >= W || y >= H) return;
    dst[c * dplane + (size_t)y * dp + x] = src[c * splane + (size_t)y * sp + x];
}

__global__ void reset_known_kernel(int H, int W, float* __restrict__ u, int up, long long uplane,
                                   const uint8_t* __restrict__ mask, int mp, const float* __restrict__ f,
                                   int fp, long long fplane) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (x >= W || y >= H) return;
    if (mask[(size_t)y * mp + x]) u[c * uplane + (size_t)y * up + x] = f[c * fplane + (size_t)y * fp + x];
}

template <typename T>
__global__ void convert_kernel(int H, int W, const float* __restrict__ src, int sp, long long splane,
                               T* __restrict__ dst, int dp, long long dplane) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (x >= W || y >= H) return;
    dst[c * dplane + (size_t)y * dp + x] = from_f<T>(src[c * splane + (size_t)y * sp + x]);
}

// ---- residual of the outer correction -----------------------------------------------
// r = b - A u on unknown pixels, i.e. r_p = sum over in-image neighbours q of
// (u_q - u_p) for an FP32 iterate u.  GB300 executes FP64 at a small fraction
// of its FP32 rate (one FP64 operation per pixel costs as much as an HBM pass
// over the frame), so the residual is formed with error-free FP32
// transformations instead: each difference u_q - u_p is split exactly into
// s + e by TwoSum (Knuth), and the four pairs are accumulated as a
// double-single number (hi, lo) with a ~48-bit significand, the accuracy FP64
// gives here.  Per-block sums of r^2 are written as doubles.
constexpr int RES_TPB = 256;
constexpr int RES_ROWS = 4;   // rows per block

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += (s, e), renormalised
__device__ __forceinline__ void ds_add(float& hi, float& lo, float s, float e) {
    float t, err;
    two_sum(hi, s, t, err);
    const float l = __fadd_rn(lo, __fadd_rn(err, e));
    hi = __fadd_rn(t, l);
    lo = __fsub_rn(l, __fsub_rn(hi, t));
}

template <typename T>
__global__ void __launch_bounds__(RES_TPB) res64_kernel(Res64Args a) {
    // block (bx, by, c) covers columns [bx*RES_TPB, +RES_TPB) and rows [by*RES_ROWS, +RES_ROWS)
    const int x = blockIdx.x * RES_TPB + threadIdx.x;
    const int c = blockIdx.z;
    const float* __restrict__ u = a.u + c * a.uplane;
    float s = 0.f, m = 0.f;
    const float sinv = a.g_out ? (float)a.scale_inv[c] : 0.f;
    if (x < a.W) {
        for (int rr = 0; rr < RES_ROWS; ++rr) {
            const int y = blockIdx.y * RES_ROWS + rr;
            if (y >= a.H) break;
            float r = 0.f;
            if (!a.mask[(size_t)y * a.mp + x]) {
                const size_t o = (size_t)y * a.up + x;
                const float uc = u[o];
                float hi = 0.f, lo = 0.f, d, e;
                if (y > 0) { two_sum(u[o - a.up], -uc, d, e); ds_add(hi, lo, d, e); }
                if (y < a.H - 1) { two_sum(u[o + a.up], -uc, d, e); ds_add(hi, lo, d, e); }
                if (x > 0) { two_sum(u[o - 1], -uc, d, e); ds_add(hi, lo, d, e); }
                if (x < a.W - 1) { two_sum(u[o + 1], -uc, d, e); ds_add(hi, lo, d, e); }
                r = __fadd_rn(hi, lo);
            }
            s = fmaf(r, r, s);
            m = fmaxf(m, fabsf(r));
            if (a.g_out) {
                T* g = static_cast<T*>(a.g_out) + c * a.gplane;
                g[(size_t)y * a.gp + x] = from_f<T>(r * sinv);
            }
        }
    }
    // fixed-order block reduction: warp butterflies, then the 8 warp results
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, k);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, k));
    }
    __shared__ float ss[RES_TPB / 32], sm[RES_TPB / 32];
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sm[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0;
        float tm = 0.f;
        for (int w = 0; w < RES_TPB / 32; ++w) {
            ts += (double)ss[w];
            tm = fmaxf(tm, sm[w]);
        }
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        a.part[(size_t)c * a.nblk + blk] = make_double2(ts, (double)tm);
    }
}

constexpr int RED_TPB = 512;

__global__ void __launch_bounds__(RED_TPB) reduce_part_kernel(const double2* __restrict__ part, int nblk,
                                                              double2* __restrict__ out) {
    const int c = blockIdx.x;
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < nblk; i += RED_TPB) {
        const double2 v = part[(size_t)c * nblk + i];
        s += v.x;
        m = fmax(m, v.y);
    }
    __shared__ double ss[RED_TPB], sm[RED_TPB];
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int h = RED_TPB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            ss[threadIdx.x] += ss[threadIdx.x + h];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = make_double2(ss[0], sm[0]);
}

// ---- multilevel ----------------------------------------------------------------------
__global__ void restrict_kernel(int H, int W, int Hc, int Wc, const uint8_t* __restrict__ mask, int mp,
                                const float* __restrict__ f, int fp, long long fplane,
                                uint8_t* __restrict__ mask_c, int mcp, float* __restrict__ f_c, int fcp,
                                long long fcplane) {
    const int X = blockIdx.x * TX + threadIdx.x, Y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (X >= Wc || Y >= Hc) return;
    int cnt = 0;
    float acc = 0.f;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int y = 2 * Y + dy, x = 2 * X + dx;
            if (y < H && x < W && mask[(size_t)y * mp + x]) {
                ++cnt;
                acc += f[c * fplane + (size_t)y * fp + x];
            }
        }
    if (c == 0) mask_c[(size_t)Y * mcp + X] = cnt > 0 ? 1 : 0;
    f_c[c * fcplane + (size_t)Y * fcp + X] = cnt > 0 ? acc / (float)cnt : 0.f;
}

__global__ void prolong_kernel(int Hc, int Wc, int H, int W, const float* __restrict__ uc, int ucp,
                               long long ucplane, const uint8_t* __restrict__ mask, int mp,
                               const float* __restrict__ f, int fp, long long fplane, float* __restrict__ u,
                               int up, long long uplane) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (x >= W || y >= H) return;
    float out;
    if (mask != nullptr && mask[(size_t)y * mp + x]) {
        out = f[c * fplane + (size_t)y * fp + x];
    } else {
        const float ty = fminf(fmaxf((y - 0.5f) * 0.5f, 0.f), (float)(Hc - 1));
        const float tx = fminf(fmaxf((x - 0.5f) * 0.5f, 0.f), (float)(Wc - 1));
        const int y0 = (int)floorf(ty), x0 = (int)floorf(tx);
        const int y1 = min(y0 + 1, Hc - 1), x1 = min(x0 + 1, Wc - 1);
        const float wy = ty - (float)y0, wx = tx - (float)x0;
        const float* p = uc + c * ucplane;
        const float top = p[(size_t)y0 * ucp + x0] * (1.f - wx) + p[(size_t)y0 * ucp + x1] * wx;
        const float bot = p[(size_t)y1 * ucp + x0] * (1.f - wx) + p[(size_t)y1 * ucp + x1] * wx;
        out = top * (1.f - wy) + bot * wy;
    }
    u[c * uplane + (size_t)y * up + x] = out;
}

template <typename T>
__global__ void correct_kernel(int H, int W, float* __restrict__ u, int up, long long uplane,
                               const T* __restrict__ e, int ep, long long eplane,
                               const uint8_t* __restrict__ mask, int mp, const double* __restrict__ scale) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (x >= W || y >= H) return;
    if (mask[(size_t)y * mp + x]) return;
    float* pu = u + c * uplane + (size_t)y * up + x;
    const double v = (double)*pu + scale[c] * (double)to_f(e[c * eplane + (size_t)y * ep + x]);
    *pu = (float)v;
}

__global__ void count_nonzero_kernel(const uint8_t* __restrict__ m, long long n,
                                     unsigned long long* __restrict__ out) {
    unsigned v = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v += m[i] != 0;
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) v += __shfl_xor_sync(0xffffffffu, v, k);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}

// ---- device-side control of a sweep sequence ------------------------------------------
// After a sweep sequence: out = {buffer holding the result, full sweeps applied, flag value}.
__global__ void resolve_kernel(const int* __restrict__ flag, const int* __restrict__ ss, const int* __restrict__ ctl,
                               int* __restrict__ out) {
    out[0] = ss[0];
    out[1] = ss[1];
    out[2] = flag[0];
    out[3] = ctl ? ctl[0] : 0;
}

__global__ void reset_sweep_state_kernel(int* __restrict__ state, int* __restrict__ flag, int cur,
                                         double* __restrict__ tol_d, double tol) {
    if (threadIdx.x < 4) {
        state[threadIdx.x] = threadIdx.x == 0 ? cur : 0;
        flag[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) *tol_d = tol;
}

__global__ void loop_ctl_kernel(const int* __restrict__ flag, const int* __restrict__ state, int* __restrict__ ctl,
                                int cap, int max_passes, cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0) return;
    const int passes = ctl[0] + 1;
    ctl[0] = passes;
    if (flag[0] != 0 || state[1] >= cap || passes >= max_passes) cudaGraphSetConditional(cond, 0);
}

__global__ void prolong_sel_kernel(int Hc, int Wc, int H, int W, const float* __restrict__ uc0,
                                   const float* __restrict__ uc1, const int* __restrict__ sel, int ucp,
                                   long long ucplane, const uint8_t* __restrict__ mask, int mp,
                                   const float* __restrict__ f, int fp, long long fplane, float* __restrict__ u,
                                   int up, long long uplane) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (x >= W || y >= H) return;
    const float* __restrict__ uc = sel[0] ? uc1 : uc0;
    float out;
    if (mask[(size_t)y * mp + x]) {
        out = f[c * fplane + (size_t)y * fp + x];
    } else {
        const float ty = fminf(fmaxf((y - 0.5f) * 0.5f, 0.f), (float)(Hc - 1));
        const float tx = fminf(fmaxf((x - 0.5f) * 0.5f, 0.f), (float)(Wc - 1));
        const int y0 = (int)floorf(ty), x0 = (int)floorf(tx);
        const int y1 = min(y0 + 1, Hc - 1), x1 = min(x0 + 1, Wc - 1);
        const float wy = ty - (float)y0, wx = tx - (float)x0;
        const float* p = uc + c * ucplane;
        const float top = p[(size_t)y0 * ucp + x0] * (1.f - wx) + p[(size_t)y0 * ucp + x1] * wx;
        const float bot = p[(size_t)y1 * ucp + x0] * (1.f - wx) + p[(size_t)y1 * ucp + x1] * wx;
        out = top * (1.f - wy) + bot * wy;
    }
    u[c * uplane + (size_t)y * up + x] = out;
}

__global__ void copy2d_sel_kernel(int H, int W, const float* __restrict__ s0, const float* __restrict__ s1,
                                  const int* __restrict__ sel, int sp, long long splane, float* __restrict__ dst,
                                  int dp, long long dplane) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (x >= W || y >= H) return;
    const float* __restrict__ src = sel[0] ? s1 : s0;
    dst[c * dplane + (size_t)y * dp + x] = src[c * splane + (size_t)y * sp + x];
}

__global__ void sqrt_sums_kernel(const double2* __restrict__ in, double* __restrict__ out, int C) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) out[c] = sqrt(in[c].x);
}

}  // namespace

cudaError_t launch_masked_copy(int H, int W, int C, const float* src, int sp, long long splane,
                               const uint8_t* mask, int mp, float* dst, int dp, long long dplane,
                               cudaStream_t st) {
    masked_copy_kernel<<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(H, W, src, sp, splane, mask, mp, dst, dp, dplane);
    return cudaGetLastError();
}

cudaError_t launch_copy2d(int H, int W, int C, const float* src, int sp, long long splane, float* dst,
                          int dp, long long dplane, cudaStream_t st) {
    copy2d_kernel<<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(H, W, src, sp, splane, dst, dp, dplane);
    return cudaGetLastError();
}

cudaError_t launch_fill_zero(Store s, void* dst, size_t n, cudaStream_t st) {
    return cudaMemsetAsync(dst, 0, n * store_bytes(s), st);
}

cudaError_t launch_reset_known(int H, int W, int C, float* u, int up, long long uplane, const uint8_t* mask,
                               int mp, const float* f, int fp, long long fplane, cudaStream_t st) {
    reset_known_kernel<<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(H, W, u, up, uplane, mask, mp, f, fp, fplane);
    return cudaGetLastError();
}

cudaError_t launch_convert(int H, int W, int C, const float* src, int sp, long long splane, void* dst,
                           Store t, int dp, long long dplane, cudaStream_t st) {
    switch (t) {
        case Store::F32:
            convert_kernel<float><<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(H, W, src, sp, splane,
                                                                             static_cast<float*>(dst), dp, dplane);
            break;
        case Store::F16:
            convert_kernel<__half><<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(H, W, src, sp, splane,
                                                                              static_cast<__half*>(dst), dp, dplane);
            break;
        case Store::BF16:
            convert_kernel<__nv_bfloat16><<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(
                H, W, src, sp, splane, static_cast<__nv_bfloat16*>(dst), dp, dplane);
            break;
    }
    return cudaGetLastError();
}

int res64_blocks(int H, int W) {
    return ((W + RES_TPB - 1) / RES_TPB) * ((H + RES_ROWS - 1) / RES_ROWS);
}

cudaError_t launch_res64(const Res64Args& a, cudaStream_t st) {
    dim3 grid((a.W + RES_TPB - 1) / RES_TPB, (a.H + RES_ROWS - 1) / RES_ROWS, a.C);
    if (a.nblk != (int)(grid.x * grid.y)) return cudaErrorInvalidValue;
    switch (a.gst) {
        case Store::F32: res64_kernel<float><<<grid, RES_TPB, 0, st>>>(a); break;
        case Store::F16: res64_kernel<__half><<<grid, RES_TPB, 0, st>>>(a); break;
        case Store::BF16: res64_kernel<__nv_bfloat16><<<grid, RES_TPB, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_part(const double2* part, int nblk, int C, double2* out, cudaStream_t st) {
    reduce_part_kernel<<<C, RED_TPB, 0, st>>>(part, nblk, out);
    return cudaGetLastError();
}

cudaError_t launch_restrict(int H, int W, int C, const uint8_t* mask, int mp, const float* f, int fp,
                            long long fplane, uint8_t* mask_c, int mcp, float* f_c, int fcp, long long fcplane,
                            cudaStream_t st) {
    const int Hc = (H + 1) / 2, Wc = (W + 1) / 2;
    restrict_kernel<<<grid2d(Hc, Wc, C), dim3(TX, TY), 0, st>>>(H, W, Hc, Wc, mask, mp, f, fp, fplane, mask_c,
                                                                mcp, f_c, fcp, fcplane);
    return cudaGetLastError();
}

cudaError_t launch_prolong(int Hc, int Wc, int H, int W, int C, const float* uc, int ucp, long long ucplane,
                           const uint8_t* mask, int mp, const float* f, int fp, long long fplane, float* u, int up,
                           long long uplane, cudaStream_t st) {
    prolong_kernel<<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(Hc, Wc, H, W, uc, ucp, ucplane, mask, mp, f, fp,
                                                             fplane, u, up, uplane);
    return cudaGetLastError();
}

cudaError_t launch_correct(int H, int W, int C, float* u, int up, long long uplane, const void* e, Store est,
                           int ep, long long eplane, const uint8_t* mask, int mp, const double* scale,
                           cudaStream_t st) {
    switch (est) {
        case Store::F32:
            correct_kernel<float><<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(
                H, W, u, up, uplane, static_cast<const float*>(e), ep, eplane, mask, mp, scale);
            break;
        case Store::F16:
            correct_kernel<__half><<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(
                H, W, u, up, uplane, static_cast<const __half*>(e), ep, eplane, mask, mp, scale);
            break;
        case Store::BF16:
            correct_kernel<__nv_bfloat16><<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(
                H, W, u, up, uplane, static_cast<const __nv_bfloat16*>(e), ep, eplane, mask, mp, scale);
            break;
    }
    return cudaGetLastError();
}

}  // namespace dd

namespace dd {

cudaError_t launch_resolve(const int* flag, const int* sweep_state, const int* ctl, int* out, cudaStream_t st) {
    resolve_kernel<<<1, 1, 0, st>>>(flag, sweep_state, ctl, out);
    return cudaGetLastError();
}

cudaError_t launch_reset_sweep_state(int* state, int* flag, int cur, double* tol_d, double tol, cudaStream_t st) {
    reset_sweep_state_kernel<<<1, 32, 0, st>>>(state, flag, cur, tol_d, tol);
    return cudaGetLastError();
}

cudaError_t launch_loop_ctl(const int* flag, const int* state, int* ctl, int cap, int max_passes,
                            cudaGraphConditionalHandle cond, cudaStream_t st) {
    loop_ctl_kernel<<<1, 32, 0, st>>>(flag, state, ctl, cap, max_passes, cond);
    return cudaGetLastError();
}

cudaError_t launch_prolong_sel(int Hc, int Wc, int H, int W, int C, const float* uc0, const float* uc1,
                               const int* sel, int ucp, long long ucplane, const uint8_t* mask, int mp,
                               const float* f, int fp, long long fplane, float* u, int up, long long uplane,
                               cudaStream_t st) {
    prolong_sel_kernel<<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(Hc, Wc, H, W, uc0, uc1, sel, ucp, ucplane, mask,
                                                                 mp, f, fp, fplane, u, up, uplane);
    return cudaGetLastError();
}

cudaError_t launch_copy2d_sel(int H, int W, int C, const float* s0, const float* s1, const int* sel, int sp,
                              long long splane, float* dst, int dp, long long dplane, cudaStream_t st) {
    copy2d_sel_kernel<<<grid2d(H, W, C), dim3(TX, TY), 0, st>>>(H, W, s0, s1, sel, sp, splane, dst, dp, dplane);
    return cudaGetLastError();
}

cudaError_t launch_sqrt_sums(const double2* in, double* out, int C, cudaStream_t st) {
    sqrt_sums_kernel<<<(C + 127) / 128, 128, 0, st>>>(in, out, C);
    return cudaGetLastError();
}

}  // namespace dd

namespace dd {

cudaError_t launch_count_nonzero(const uint8_t* m, long long n, unsigned long long* out, cudaStream_t st) {
    const long long blocks = std::min<long long>((n + 255) / 256, 1216);
    count_nonzero_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, st>>>(m, n, out);
    return cudaGetLastError();
}

}  // namespace dd
