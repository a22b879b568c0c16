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

__global__ void reset_known_kernel(int H, int W, float* __restrict__ u, int up, long long uplane,
                                   const uint8_t* __restrict__ mask, int mp, const float* __restrict__ f,
                                   int fp, long long fplane) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, c = blockIdx.z;
    if (x >= W || y >= H) return;
    if (mask[(size_t)y * mp + x]) u[c * uplane + (size_t)y * up + x] = f[c * fplane + (size_t)y * fp + x];
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
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// TwoSum on two independent lanes at once (packed FP32 adds, each rounded to
// nearest: the same operations as two_sum on each half)
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, neg2(a));
    e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
}

// (hi, lo) += (s, e), renormalised
__device__ __forceinline__ void ds_add(float& hi, float& lo, float s, float e) {
    float t, err;
    two_sum(hi, s, t, err);
    const float l = __fadd_rn(lo, __fadd_rn(err, e));
    hi = __fadd_rn(t, l);
    lo = __fsub_rn(l, __fsub_rn(hi, t));
}

// Vectorised streaming layout: a thread owns 4 consecutive columns (one
// float4 where the row is 16-byte aligned) in V_ROWS rows; a block of 32 x 8
// threads covers 128 columns x 32 rows, so a warp moves 512 contiguous bytes
// per row and each thread keeps several independent 16-byte loads in flight.
constexpr int V_TX = 32, V_TY = 8, V_ROWS = 4;
constexpr int V_TPB = V_TX * V_TY;
constexpr int V_COLS = V_TX * 4, V_BROWS = V_TY * V_ROWS;

dim3 gridv(int H, int W, int C) { return dim3((W + V_COLS - 1) / V_COLS, (H + V_BROWS - 1) / V_BROWS, C); }

// rows of pitch `pitch` elements of `elem` bytes (planes `plane` elements
// apart) from p start on 16-byte boundaries
bool vec_ok(const void* p, long long pitch, long long plane, int elem) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && (pitch * elem) % 16 == 0 && (plane * elem) % 16 == 0;
}

__device__ __forceinline__ void ld4(const float* __restrict__ row, int x0, int W, bool vec, float (&v)[4]) {
    if (vec && x0 + 3 < W) {
        const float4 t = *reinterpret_cast<const float4*>(row + x0);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = x0 + j < W ? row[x0 + j] : 0.f;
    }
}

__device__ __forceinline__ void st4(float* __restrict__ row, int x0, int W, bool vec, const float (&v)[4]) {
    if (vec && x0 + 3 < W) {
        *reinterpret_cast<float4*>(row + x0) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (x0 + j < W) row[x0 + j] = v[j];
    }
}

__device__ __forceinline__ void ldm4(const uint8_t* __restrict__ row, int x0, int W, bool vec, bool (&m)[4]) {
    if (vec && x0 + 3 < W) {
        const uchar4 t = *reinterpret_cast<const uchar4*>(row + x0);
        m[0] = t.x != 0; m[1] = t.y != 0; m[2] = t.z != 0; m[3] = t.w != 0;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j] = x0 + j < W && row[x0 + j] != 0;
    }
}

// The 4 mask bytes of columns x0 .. x0+3 (byte j for column x0 + j; 0 past W).
__device__ __forceinline__ uint32_t ldm4w(const uint8_t* __restrict__ row, int x0, int W, bool vec) {
    if (vec && x0 + 3 < W) return *reinterpret_cast<const uint32_t*>(row + x0);
    uint32_t w = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (x0 + j < W) w |= (uint32_t)row[x0 + j] << (8 * j);
    return w;
}

struct ResVec {
    bool u, m, g, cp;   // float4 / uchar4 access to u (and u1), mask, g_out (F32 only), copy_out
};

// Per pixel p, r_p = sum over in-image neighbours q of (u_q - u_p), formed
// with TwoSum so that only the final rounding to FP32 remains; r = 0 on known
// pixels.  A tile is 128 x 32 pixels: each thread owns 4 columns in 4 rows.
// Each thread accumulates r^2 (FP32) and max |r| over its pixels of a tile,
// a warp butterfly sums them, and the warp's lane 0 adds the tile's sum into
// an FP64 accumulator.
// Grid (gx, 1, C): the gx blocks of channel c walk its tiles grid-stride, one
// wave of resident blocks for the whole pass, so that the per-block work of
// fencing, taking the ticket and writing a partial is paid once per block
// rather than per tile.  Block b's partial (its warps in order) goes to
// part[c * nblk + b].  With a.out, the last block (atomic ticket) reduces each
// channel's gx partials, one warp per channel in a fixed lane order, into
// out[c] = {sum r^2, max |r|} and sqrt_out[c] = sqrt(sum).  The order of every
// sum depends only on the grid, so results repeat bit for bit on one device.
constexpr int R_ROWS = 4, R_BROWS = V_TY * R_ROWS;

dim3 grid_res(int H, int W, int C) { return dim3((W + V_COLS - 1) / V_COLS, (H + R_BROWS - 1) / R_BROWS, C); }

// Sum (and max) of n per-block partials p[0..n) by one warp, in a fixed order
// (lane-strided with four independent accumulators, then a butterfly); every
// lane gets the result.
__device__ __forceinline__ double2 warp_sum_parts(const double2* __restrict__ p, int n, int lane) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, m = 0.0;
    int i = lane;
    for (; i + 96 < n; i += 128) {
        const double2 v0 = __ldcg(p + i), v1 = __ldcg(p + i + 32), v2 = __ldcg(p + i + 64), v3 = __ldcg(p + i + 96);
        s0 += v0.x; s1 += v1.x; s2 += v2.x; s3 += v3.x;
        m = fmax(fmax(m, fmax(v0.y, v1.y)), fmax(v2.y, v3.y));
    }
    for (; i < n; i += 32) {
        const double2 v = __ldcg(p + i);
        s0 += v.x;
        m = fmax(m, v.y);
    }
    double sv = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
        sv += __shfl_xor_sync(0xffffffffu, sv, k);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, k));
    }
    return make_double2(sv, m);
}
__device__ __forceinline__ double warp_sum_parts(const double* __restrict__ p, int n, int lane) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = lane;
    for (; i + 96 < n; i += 128) {
        s0 += __ldcg(p + i);
        s1 += __ldcg(p + i + 32);
        s2 += __ldcg(p + i + 64);
        s3 += __ldcg(p + i + 96);
    }
    for (; i < n; i += 32) s0 += __ldcg(p + i);
    double sv = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, k);
    return sv;
}

template <typename T>
__global__ void __launch_bounds__(V_TPB) res64_kernel(Res64Args a, ResVec vec) {
    if (a.skip != nullptr && *a.skip != 0) return;   // uniform: no partial, no ticket
    const int c = blockIdx.z;
    const int H = a.H, W = a.W;
    const int gxt = (W + V_COLS - 1) / V_COLS, ntile = gxt * ((H + R_BROWS - 1) / R_BROWS);
    const float* __restrict__ u = ((a.sel != nullptr && a.sel[0]) ? a.u1 : a.u) + c * a.uplane;
    const float sinv = a.g_out ? (float)a.scale_inv[c] : 0.f;
    const int lane = threadIdx.x, wid = threadIdx.y;   // one warp per thread row
    double wsum = 0.0;   // lane 0: this warp's sum over the block's tiles
    float wmax = 0.f;
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int by = t / gxt, bx = t - by * gxt;
        const int x0 = (bx * V_TX + threadIdx.x) * 4;
        const int yb = (by * V_TY + threadIdx.y) * R_ROWS;
        const bool xin = x0 < W;
        // every load of the tile before any arithmetic: the rows yb-1 .. yb+R_ROWS
        // (0 outside the image), the halo columns x0-1 (lane 0) and x0+4 (lane 31)
        // and the mask bytes of the thread's rows
        float rows[R_ROWS + 2][4], hl[R_ROWS], hr[R_ROWS];
        uint32_t mk[R_ROWS];
#pragma unroll
        for (int k = 0; k < R_ROWS + 2; ++k) {
            const int y = yb - 1 + k;
            if (xin && y >= 0 && y < H) {
                ld4(u + (size_t)y * a.up, x0, W, vec.u, rows[k]);
            } else {
                rows[k][0] = rows[k][1] = rows[k][2] = rows[k][3] = 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < R_ROWS; ++k) {
            const int y = yb + k;
            const bool yin = xin && y < H;
            hl[k] = (lane == 0 && yin && x0 > 0) ? u[(size_t)y * a.up + x0 - 1] : 0.f;
            hr[k] = (lane == V_TX - 1 && yin && x0 + 4 < W) ? u[(size_t)y * a.up + x0 + 4] : 0.f;
            mk[k] = yin ? ldm4w(a.mask + (size_t)y * a.mp, x0, W, vec.m) : 0u;
        }
        float s = 0.f, mx = 0.f;
#pragma unroll
        for (int k = 0; k < R_ROWS; ++k) {
            const int y = yb + k;
            const float* rw = rows[k + 1];
            float left = __shfl_up_sync(0xffffffffu, rw[3], 1);
            float right = __shfl_down_sync(0xffffffffu, rw[0], 1);
            if (!xin || y >= H) continue;
            if (lane == 0) left = hl[k];
            if (lane == V_TX - 1) right = hr[k];
            bool known[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) known[j] = ((mk[k] >> (8 * j)) & 0xffu) != 0u;
            float r[4];
            // all four pixels away from the image border: one branch per row group
            if (y > 0 && y < H - 1 && x0 > 0 && x0 + 4 < W) {
                // (N + S) + (W + E) - 4 u_p by TwoSum steps (4 u_p is exact), the
                // rounding errors summed in FP32: ~48-bit accurate before the one
                // final rounding, as the general path below; pixels (0, 1) and
                // (2, 3) side by side in packed adds
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = 2 * h;
                    const float2 nn = make_float2(rows[k][j], rows[k][j + 1]);
                    const float2 ss2 = make_float2(rows[k + 2][j], rows[k + 2][j + 1]);
                    const float2 ww = make_float2(j > 0 ? rw[j - 1] : left, rw[j]);
                    const float2 ee = make_float2(rw[j + 1], j + 2 < 4 ? rw[j + 2] : right);
                    const float2 c4 = make_float2(-4.f * rw[j], -4.f * rw[j + 1]);
                    float2 s1, e1, s2, e2, t, e3, dd, e4;
                    two_sum2(nn, ss2, s1, e1);
                    two_sum2(ww, ee, s2, e2);
                    two_sum2(s1, s2, t, e3);
                    two_sum2(t, c4, dd, e4);
                    const float2 rv = __fadd2_rn(dd, __fadd2_rn(__fadd2_rn(e1, e2), __fadd2_rn(e3, e4)));
                    r[j] = known[j] ? 0.f : rv.x;
                    r[j + 1] = known[j + 1] ? 0.f : rv.y;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // the in-image neighbour differences u_q - u_p, each split exactly
                    // by TwoSum, accumulated double-single
                    const int x = x0 + j;
                    const float uc = rw[j];
                    float hi = 0.f, lo = 0.f, d, e;
                    if (y > 0) { two_sum(rows[k][j], -uc, d, e); ds_add(hi, lo, d, e); }
                    if (y < H - 1) { two_sum(rows[k + 2][j], -uc, d, e); ds_add(hi, lo, d, e); }
                    if (x > 0) { two_sum(j > 0 ? rw[j - 1] : left, -uc, d, e); ds_add(hi, lo, d, e); }
                    if (x < W - 1) { two_sum(j < 3 ? rw[j + 1] : right, -uc, d, e); ds_add(hi, lo, d, e); }
                    r[j] = (x < W && !known[j]) ? __fadd_rn(hi, lo) : 0.f;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                s = fmaf(r[j], r[j], s);
                mx = fmaxf(mx, fabsf(r[j]));
            }
            if (a.copy_out) st4(a.copy_out + c * a.cplane + (size_t)y * a.cp, x0, W, vec.cp, rows[k + 1]);
            if (a.g_out) {
                T* g = static_cast<T*>(a.g_out) + c * a.gplane + (size_t)y * a.gp;
                if constexpr (sizeof(T) == 4) {
                    const float gv[4] = {r[0] * sinv, r[1] * sinv, r[2] * sinv, r[3] * sinv};
                    st4(reinterpret_cast<float*>(g), x0, W, vec.g, gv);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (x0 + j < W) g[x0 + j] = from_f<T>(r[j] * sinv);
                }
            }
        }
#pragma unroll
        for (int k = 16; k >= 1; k >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, k);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, k));
        }
        if (lane == 0) {
            wsum += (double)s;
            wmax = fmaxf(wmax, mx);
        }
    }
    __shared__ double ss[V_TY];
    __shared__ float sm[V_TY];
    __shared__ int s_last;
    const int tid = threadIdx.y * V_TX + threadIdx.x;
    if (lane == 0) {
        ss[wid] = wsum;
        sm[wid] = wmax;
    }
    __syncthreads();
    if (tid == 0) {
        double ts = 0.0;
        float tm = 0.f;
        for (int w = 0; w < V_TY; ++w) {
            ts += ss[w];
            tm = fmaxf(tm, sm[w]);
        }
        a.part[(size_t)c * a.nblk + blockIdx.x] = make_double2(ts, (double)tm);
        if (a.out != nullptr) {   // the partial is visible before the ticket is taken
            __threadfence();
            s_last = atomicAdd(a.ticket, 1u) == gridDim.x * gridDim.z - 1;
        }
    }
    if (a.out == nullptr) return;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int cc = wid; cc < a.C; cc += V_TY) {
        const double2 r = warp_sum_parts(a.part + (size_t)cc * a.nblk, (int)gridDim.x, lane);
        if (lane == 0) {
            a.out[cc] = r;
            if (a.sqrt_out) a.sqrt_out[cc] = sqrt(r.x);
        }
    }
    if (tid == 0) *a.ticket = 0u;
}

// Reference norms ||b - A u0||, u0 = C f, of every level in one launch: the
// residual of u0 on an unknown pixel is the sum of its known in-image
// neighbours' values (u0 is 0 on unknown pixels), summed in FP32 (at most four
// values), squared and added per thread in FP32 and per warp and tile, then
// across tiles in FP64.  Grid (gx, levels x C): the gx blocks of segment
// (level, channel) walk its 128 x 32 tiles grid-stride (a coarse level's
// segment has fewer tiles, and its surplus blocks only take the ticket).  Block
// b writes its partial to part[seg * gx + b] if it had a tile; the last block
// (atomic ticket) sums each segment's partials, one warp per segment in a
// fixed lane order, into out[c] = {sum, 0} and sqrt_out[c].
__global__ void __launch_bounds__(V_TPB) ref_norms_kernel(RefNormArgs a) {
    const int seg = blockIdx.y;
    const int l = seg / a.C, c = seg - l * a.C;
    const RefLevel& L = a.lv[l];
    const int H = L.H, W = L.W;
    const int ntile = L.gx * L.gy;
    const float* __restrict__ u = L.f + c * L.fplane;
    const int lane = threadIdx.x, wid = threadIdx.y;
    double wsum = 0.0;
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int by = t / L.gx, bx = t - by * L.gx;
        const int x0 = (bx * V_TX + threadIdx.x) * 4;
        const int yb = (by * V_TY + threadIdx.y) * R_ROWS;
        const bool xin = x0 < W;
        // every load of the tile before any arithmetic (as in the residual pass)
        float rows[R_ROWS + 2][4], hl[R_ROWS], hr[R_ROWS];
        uint32_t mk[R_ROWS];
#pragma unroll
        for (int k = 0; k < R_ROWS + 2; ++k) {
            const int y = yb - 1 + k;
            if (xin && y >= 0 && y < H) {
                ld4(u + (size_t)y * L.fp, x0, W, true, rows[k]);
            } else {
                rows[k][0] = rows[k][1] = rows[k][2] = rows[k][3] = 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < R_ROWS; ++k) {
            const int y = yb + k;
            const bool yin = xin && y < H;
            hl[k] = (lane == 0 && yin && x0 > 0) ? u[(size_t)y * L.fp + x0 - 1] : 0.f;
            hr[k] = (lane == V_TX - 1 && yin && x0 + 4 < W) ? u[(size_t)y * L.fp + x0 + 4] : 0.f;
            mk[k] = yin ? ldm4w(L.mask + (size_t)y * L.mp, x0, W, L.mvec != 0) : 0u;
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < R_ROWS; ++k) {
            const int y = yb + k;
            const float* rw = rows[k + 1];
            float left = __shfl_up_sync(0xffffffffu, rw[3], 1);
            float right = __shfl_down_sync(0xffffffffu, rw[0], 1);
            if (!xin || y >= H) continue;
            if (lane == 0) left = hl[k];
            if (lane == V_TX - 1) right = hr[k];
            bool known[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) known[j] = ((mk[k] >> (8 * j)) & 0xffu) != 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float wv = j > 0 ? rw[j - 1] : left, ev = j < 3 ? rw[j + 1] : right;
                const float r = (x0 + j < W && !known[j]) ? (rows[k][j] + rows[k + 2][j]) + (wv + ev) : 0.f;
                s = fmaf(r, r, s);
            }
        }
#pragma unroll
        for (int k = 16; k >= 1; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
        if (lane == 0) wsum += (double)s;
    }
    __shared__ double ss[V_TY];
    __shared__ int s_last;
    const int tid = threadIdx.y * V_TX + threadIdx.x;
    if (lane == 0) ss[wid] = wsum;
    __syncthreads();
    if (tid == 0) {
        if ((int)blockIdx.x < ntile) {
            double ts = 0.0;
            for (int w = 0; w < V_TY; ++w) ts += ss[w];
            a.part[(size_t)seg * gridDim.x + blockIdx.x] = ts;
        }
        __threadfence();
        s_last = atomicAdd(a.ticket, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int q = wid; q < (int)gridDim.y; q += V_TY) {
        const int lq = q / a.C, cq = q - lq * a.C;
        const RefLevel& Q = a.lv[lq];
        const double sv = warp_sum_parts(a.part + (size_t)q * gridDim.x, min((int)gridDim.x, Q.gx * Q.gy), lane);
        if (lane == 0) {
            Q.out[cq] = make_double2(sv, 0.0);
            Q.sqrt_out[cq] = sqrt(sv);
        }
    }
    if (tid == 0) *a.ticket = 0u;
}

// ---- streaming passes (vectorised layout above) -----------------------------------------
struct CopyVec {
    bool src, dst, m;
};

// Sum of one unsigned value per thread over a block of V_TPB threads, added
// to *count by thread 0 (one atomic per block).
__device__ __forceinline__ void block_count_add(unsigned v, unsigned long long* count) {
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) v += __shfl_xor_sync(0xffffffffu, v, k);
    __shared__ unsigned ws[V_TPB / 32];
    const int tid = threadIdx.y * V_TX + threadIdx.x;
    if ((tid & 31) == 0) ws[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        unsigned t = 0;
        for (int w = 0; w < V_TPB / 32; ++w) t += ws[w];
        if (t) atomicAdd(count, (unsigned long long)t);
    }
}

// dst = mask ? src : 0 (mask may be null: plain copy); with count, the blocks
// of channel 0 add the number of known pixels to *count.
__global__ void __launch_bounds__(V_TPB) masked_copy_kernel(int H, int W, const float* __restrict__ src, int sp,
                                                            long long splane, const uint8_t* __restrict__ mask,
                                                            int mp, float* __restrict__ dst, int dp,
                                                            long long dplane, CopyVec vec,
                                                            unsigned long long* __restrict__ count) {
    const int c = blockIdx.z;
    const int x0 = (blockIdx.x * V_TX + threadIdx.x) * 4;
    const int yb = (blockIdx.y * V_TY + threadIdx.y) * V_ROWS;
    const float* __restrict__ s = src + c * splane;
    float* __restrict__ d = dst + c * dplane;
    unsigned known = 0;
    if (x0 < W) {
#pragma unroll
        for (int k = 0; k < V_ROWS; ++k) {
            const int y = yb + k;
            if (y >= H) break;
            float v[4];
            ld4(s + (size_t)y * sp, x0, W, vec.src, v);
            if (mask != nullptr) {
                bool m[4];
                ldm4(mask + (size_t)y * mp, x0, W, vec.m, m);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    v[j] = m[j] ? v[j] : 0.f;
                    known += m[j] ? 1u : 0u;
                }
            }
            st4(d + (size_t)y * dp, x0, W, vec.dst, v);
        }
    }
    if (count != nullptr && c == 0) block_count_add(known, count);   // uniform per block
}

// Bilinear cell-centred prolongation of the coarse iterate (Sec. 4) on
// unknown pixels, f on known ones (mask may be null: everywhere bilinear).
// The coarse source is sel[0] ? uc1 : uc0 (sel may be null: uc0).
// Fine pixel x sits at coarse coordinate (x - 1/2)/2, clamped to [0, Wc - 1].
// A thread's 4 columns start at an even coarse column x0/2 and need coarse
// columns x0/2 - 1 .. x0/2 + 2 with the fixed weights 1/4, 3/4 (indices
// clamped to the grid, which equals clamping the coordinate); likewise its 4
// rows need coarse rows yb/2 - 1 .. yb/2 + 2.  So each thread reads 4 x 4
// coarse values for its 16 fine pixels.
__global__ void __launch_bounds__(V_TPB) prolong_kernel(int Hc, int Wc, int H, int W, const float* __restrict__ uc0,
                                                        const float* __restrict__ uc1, const int* __restrict__ sel,
                                                        int ucp, long long ucplane, const uint8_t* __restrict__ mask,
                                                        int mp, const float* __restrict__ f, int fp, long long fplane,
                                                        float* __restrict__ u, int up, long long uplane, CopyVec vec) {
    static_assert(V_ROWS == 4, "the weight pattern covers 4 rows per thread");
    const int c = blockIdx.z;
    const int x0 = (blockIdx.x * V_TX + threadIdx.x) * 4;
    const int yb = (blockIdx.y * V_TY + threadIdx.y) * V_ROWS;
    if (x0 >= W || yb >= H) return;
    const float* __restrict__ p = ((sel != nullptr && sel[0]) ? uc1 : uc0) + c * ucplane;
    const int cx = x0 >> 1, cy = yb >> 1;
    int col[4], row[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        col[j] = min(max(cx - 1 + j, 0), Wc - 1);
        row[j] = min(max(cy - 1 + j, 0), Hc - 1);
    }
    // the mask bytes of the thread's rows first, so that the loads of the
    // known values they select and of the coarse values go out together
    uint32_t mk[V_ROWS];
#pragma unroll
    for (int k = 0; k < V_ROWS; ++k)
        mk[k] = (mask != nullptr && yb + k < H) ? ldm4w(mask + (size_t)(yb + k) * mp, x0, W, vec.m) : 0u;
    // horizontal interpolation of the 4 coarse rows onto the thread's 4 columns
    float hrow[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float* __restrict__ pr = p + (size_t)row[r] * ucp;
        const float c0 = pr[col[0]], c1 = pr[col[1]], c2 = pr[col[2]], c3 = pr[col[3]];
        hrow[r][0] = 0.25f * c0 + 0.75f * c1;
        hrow[r][1] = 0.75f * c1 + 0.25f * c2;
        hrow[r][2] = 0.25f * c1 + 0.75f * c2;
        hrow[r][3] = 0.75f * c2 + 0.25f * c3;
    }
    // the known values only where the group has a known pixel (a few per cent
    // of the groups at sparse masks)
    float fv[V_ROWS][4];
#pragma unroll
    for (int k = 0; k < V_ROWS; ++k) {
        fv[k][0] = fv[k][1] = fv[k][2] = fv[k][3] = 0.f;
        if (mk[k] != 0u) ld4(f + c * fplane + (size_t)(yb + k) * fp, x0, W, vec.src, fv[k]);
    }
#pragma unroll
    for (int k = 0; k < V_ROWS; ++k) {
        const int y = yb + k;
        if (y >= H) break;
        // rows yb, yb+1, yb+2, yb+3 sit between coarse rows (0,1), (1,2), (1,2), (2,3) of the four
        const int ra = k == 0 ? 0 : (k == 3 ? 2 : 1);
        const float wa = (k == 0 || k == 2) ? 0.25f : 0.75f;
        float out[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool known = ((mk[k] >> (8 * j)) & 0xffu) != 0u;
            out[j] = known ? fv[k][j] : (x0 + j < W ? wa * hrow[ra][j] + (1.f - wa) * hrow[ra + 1][j] : 0.f);
        }
        st4(u + c * uplane + (size_t)y * up, x0, W, vec.dst, out);
    }
}

// Dyadic restriction (Sec. 4): coarse pixel (X, Y) is known if any of its 2x2
// fine pixels is, with the mean of their known values.  A thread owns 4
// coarse columns (8 fine columns) in V_ROWS coarse rows.
__global__ void __launch_bounds__(V_TPB) restrict_kernel(int H, int W, int Hc, int Wc, const uint8_t* __restrict__ mask,
                                                         int mp, const float* __restrict__ f, int fp,
                                                         long long fplane, uint8_t* __restrict__ mask_c, int mcp,
                                                         float* __restrict__ f_c, int fcp, long long fcplane,
                                                         CopyVec vec) {
    const int c = blockIdx.z;
    const int X0 = (blockIdx.x * V_TX + threadIdx.x) * 4;
    const int Yb = (blockIdx.y * V_TY + threadIdx.y) * V_ROWS;
    if (X0 >= Wc) return;
    const float* __restrict__ fc = f + c * fplane;
#pragma unroll
    for (int k = 0; k < V_ROWS; ++k) {
        const int Y = Yb + k;
        if (Y >= Hc) break;
        float fv[2][8];
        bool mv[2][8];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int y = 2 * Y + dy;
            if (y < H) {
                float a4[4], b4[4];
                bool ma[4], mb[4];
                ld4(fc + (size_t)y * fp, 2 * X0, W, vec.src, a4);
                ld4(fc + (size_t)y * fp, 2 * X0 + 4, W, vec.src, b4);
                ldm4(mask + (size_t)y * mp, 2 * X0, W, vec.m, ma);
                ldm4(mask + (size_t)y * mp, 2 * X0 + 4, W, vec.m, mb);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    fv[dy][j] = a4[j]; fv[dy][j + 4] = b4[j];
                    mv[dy][j] = ma[j]; mv[dy][j + 4] = mb[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) { fv[dy][j] = 0.f; mv[dy][j] = false; }
            }
        }
        float out[4];
        uint8_t mo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int cnt = 0;
            float acc = 0.f;
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx)
                    if (mv[dy][2 * j + dx]) {
                        ++cnt;
                        acc += fv[dy][2 * j + dx];
                    }
            // the mean by the reciprocal of the count (1, 1/2, 1/3, 1/4: within an
            // ulp of the quotient, without the division's instruction sequence)
            const float rc = cnt == 1 ? 1.f : (cnt == 2 ? 0.5f : (cnt == 3 ? (1.f / 3.f) : 0.25f));
            out[j] = cnt > 0 ? acc * rc : 0.f;
            mo[j] = cnt > 0 ? 1 : 0;
        }
        st4(f_c + c * fcplane + (size_t)Y * fcp, X0, Wc, vec.dst, out);
        if (c == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (X0 + j < Wc) mask_c[(size_t)Y * mcp + X0 + j] = mo[j];
        }
    }
}

// ---- two-level coarse correction (DD_ML_CORRECTION) -------------------------------------
// Coarse right-hand side: g_c(X, Y) = sum of the fine values over the 2x2
// block {2Y, 2Y+1} x {2X, 2X+1} inside the image.  The h = 1 stencil on a grid
// twice as coarse represents the Laplacian times 4, so summing (4 x the mean)
// gives the coarse equation of the restricted residual.  No-op if *skip != 0.
__global__ void __launch_bounds__(V_TPB) restrict_sum_kernel(int H, int W, int Hc, int Wc,
                                                             const float* __restrict__ src, int sp, long long splane,
                                                             float* __restrict__ dst, int dp, long long dplane,
                                                             const int* __restrict__ skip, CopyVec vec) {
    if (skip != nullptr && *skip != 0) return;
    const int c = blockIdx.z;
    const int X0 = (blockIdx.x * V_TX + threadIdx.x) * 4;
    const int Yb = (blockIdx.y * V_TY + threadIdx.y) * V_ROWS;
    if (X0 >= Wc) return;
    const float* __restrict__ s = src + c * splane;
#pragma unroll
    for (int k = 0; k < V_ROWS; ++k) {
        const int Y = Yb + k;
        if (Y >= Hc) break;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int y = 2 * Y + dy;
            if (y >= H) break;
            float a4[4], b4[4];
            ld4(s + (size_t)y * sp, 2 * X0, W, vec.src, a4);
            ld4(s + (size_t)y * sp, 2 * X0 + 4, W, vec.src, b4);
            acc[0] += a4[0] + a4[1];
            acc[1] += a4[2] + a4[3];
            acc[2] += b4[0] + b4[1];
            acc[3] += b4[2] + b4[3];
        }
        st4(dst + c * dplane + (size_t)Y * dp, X0, Wc, vec.dst, acc);
    }
}

// ---- energy-optimal step of the coarse correction ---------------------------------------
// The prolonged correction d is scaled by omega = (r, d) / (d, A d) per
// channel, the step that minimises the A-norm of the error along d (A is SPD
// on the unknowns), so a correction from an approximate, non-Galerkin coarse
// problem can never increase that error.  Three streaming passes:
//   dir:   d = P e_c on unknown pixels (0 on known), written over r, and (r, d);
//   curv:  (d, A d) with (A d)_p = sum over in-image neighbours q of (d_p - d_q);
//          its last block also forms omega;
//   step:  u += omega d.
// Each pass's blocks write double partials in block order; the last block
// (atomic ticket) reduces them in a fixed order.  All are no-ops if *skip != 0.
struct DotTail {
    double* part;        // C x nblk
    int nblk;
    unsigned int* ticket;
    double* out;         // C: the reduced sums
    const double* num;   // curv only: (r, d) per channel, for omega
    double* omega;       // curv only: C
};

__device__ void dot_tail(float s, int c, const DotTail& t, int C) {
    __shared__ float ss[V_TPB / 32];
    __shared__ int s_last;
    __shared__ double rs[V_TPB];
    const int tid = threadIdx.y * V_TX + threadIdx.x;
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((tid & 31) == 0) ss[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        double ts = 0.0;
        for (int w = 0; w < V_TPB / 32; ++w) ts += (double)ss[w];
        t.part[(size_t)c * t.nblk + blockIdx.y * gridDim.x + blockIdx.x] = ts;
        __threadfence();
        s_last = atomicAdd(t.ticket, 1u) == gridDim.x * gridDim.y * gridDim.z - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int cc = 0; cc < C; ++cc) {
        double sv = 0.0;
        for (int i = tid; i < t.nblk; i += V_TPB) sv += __ldcg(t.part + (size_t)cc * t.nblk + i);
        rs[tid] = sv;
        __syncthreads();
        for (int hh = V_TPB / 2; hh > 0; hh >>= 1) {
            if (tid < hh) rs[tid] += rs[tid + hh];
            __syncthreads();
        }
        if (tid == 0) {
            t.out[cc] = rs[0];
            if (t.omega) {
                const double num = t.num[cc], den = rs[0];
                t.omega[cc] = (den > 0.0 && isfinite(num) && isfinite(den)) ? num / den : 0.0;
            }
        }
        __syncthreads();
    }
    if (tid == 0) *t.ticket = 0u;
}

// d = bilinear prolongation of (sel_c && sel_c[0] ? ec1 : ec0) on unknown fine
// pixels (0 on known), written over r; (r, d) per channel.
__global__ void __launch_bounds__(V_TPB) corr_dir_kernel(int Hc, int Wc, int H, int W, int C,
                                                         const float* __restrict__ ec0,
                                                         const float* __restrict__ ec1, const int* __restrict__ sel_c,
                                                         int ecp, long long ecplane, const uint8_t* __restrict__ mask,
                                                         int mp, float* __restrict__ rd, int rp, long long rplane,
                                                         const int* __restrict__ skip, DotTail t, CopyVec vec) {
    if (skip != nullptr && *skip != 0) return;
    const int c = blockIdx.z;
    const int x0 = (blockIdx.x * V_TX + threadIdx.x) * 4;
    const int yb = (blockIdx.y * V_TY + threadIdx.y) * V_ROWS;
    float s = 0.f;
    if (x0 < W) {
        const float* __restrict__ p = ((sel_c != nullptr && sel_c[0]) ? ec1 : ec0) + c * ecplane;
        float* __restrict__ rr = rd + c * rplane;
        int xa[4], xb[4];
        float wx[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float tx = fminf(fmaxf((x0 + j - 0.5f) * 0.5f, 0.f), (float)(Wc - 1));
            xa[j] = (int)floorf(tx);
            xb[j] = min(xa[j] + 1, Wc - 1);
            wx[j] = tx - (float)xa[j];
        }
#pragma unroll
        for (int k = 0; k < V_ROWS; ++k) {
            const int y = yb + k;
            if (y >= H) break;
            const float ty = fminf(fmaxf((y - 0.5f) * 0.5f, 0.f), (float)(Hc - 1));
            const int ya = (int)floorf(ty), yb1 = min(ya + 1, Hc - 1);
            const float wy = ty - (float)ya;
            const float* __restrict__ ra = p + (size_t)ya * ecp;
            const float* __restrict__ rb = p + (size_t)yb1 * ecp;
            bool m[4];
            ldm4(mask + (size_t)y * mp, x0, W, vec.m, m);
            float r[4], d[4];
            ld4(rr + (size_t)y * rp, x0, W, vec.dst, r);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                d[j] = 0.f;
                if (!m[j] && x0 + j < W) {
                    const float top = ra[xa[j]] * (1.f - wx[j]) + ra[xb[j]] * wx[j];
                    const float bot = rb[xa[j]] * (1.f - wx[j]) + rb[xb[j]] * wx[j];
                    d[j] = top * (1.f - wy) + bot * wy;
                }
                s = fmaf(r[j], d[j], s);
            }
            st4(rr + (size_t)y * rp, x0, W, vec.dst, d);
        }
    }
    dot_tail(s, c, t, C);
}

// (d, A d) per channel, and omega = (r, d) / (d, A d) in the last block.
__global__ void __launch_bounds__(V_TPB) corr_curv_kernel(int H, int W, int C, const float* __restrict__ dd, int dp,
                                                          long long dplane, const int* __restrict__ skip, DotTail t,
                                                          CopyVec vec) {
    if (skip != nullptr && *skip != 0) return;
    const int c = blockIdx.z;
    const int x0 = (blockIdx.x * V_TX + threadIdx.x) * 4;
    const int yb = (blockIdx.y * V_TY + threadIdx.y) * V_ROWS;
    const bool xin = x0 < W;
    const float* __restrict__ d = dd + c * dplane;
    float rows[V_ROWS + 2][4];
#pragma unroll
    for (int k = 0; k < V_ROWS + 2; ++k) {
        const int y = yb - 1 + k;
        if (xin && y >= 0 && y < H) {
            ld4(d + (size_t)y * dp, x0, W, vec.src, rows[k]);
        } else {
            rows[k][0] = rows[k][1] = rows[k][2] = rows[k][3] = 0.f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < V_ROWS; ++k) {
        const int y = yb + k;
        const float* rw = rows[k + 1];
        float left = __shfl_up_sync(0xffffffffu, rw[3], 1);
        float right = __shfl_down_sync(0xffffffffu, rw[0], 1);
        if (!xin || y >= H) continue;
        if (threadIdx.x == 0) left = x0 > 0 ? d[(size_t)y * dp + x0 - 1] : 0.f;
        if (threadIdx.x == V_TX - 1) right = x0 + 4 < W ? d[(size_t)y * dp + x0 + 4] : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + j;
            if (x >= W) continue;
            const float dc = rw[j];   // 0 on known pixels: their rows drop out
            float ad = 0.f;
            if (y > 0) ad += dc - rows[k][j];
            if (y < H - 1) ad += dc - rows[k + 2][j];
            if (x > 0) ad += dc - (j > 0 ? rw[j - 1] : left);
            if (x < W - 1) ad += dc - (j < 3 ? rw[j + 1] : right);
            s = fmaf(dc, ad, s);
        }
    }
    dot_tail(s, c, t, C);
}

// (sel_u[0] ? u1 : u0) += omega[c] d
__global__ void __launch_bounds__(V_TPB) corr_step_kernel(int H, int W, const float* __restrict__ dd, int dp,
                                                          long long dplane, const double* __restrict__ omega,
                                                          float* __restrict__ u0, float* __restrict__ u1,
                                                          const int* __restrict__ sel_u, int up, long long uplane,
                                                          const int* __restrict__ skip, CopyVec vec) {
    if (skip != nullptr && *skip != 0) return;
    const int c = blockIdx.z;
    const int x0 = (blockIdx.x * V_TX + threadIdx.x) * 4;
    const int yb = (blockIdx.y * V_TY + threadIdx.y) * V_ROWS;
    if (x0 >= W) return;
    const float w = (float)omega[c];
    const float* __restrict__ d = dd + c * dplane;
    float* __restrict__ u = (sel_u[0] ? u1 : u0) + c * uplane;
#pragma unroll
    for (int k = 0; k < V_ROWS; ++k) {
        const int y = yb + k;
        if (y >= H) break;
        float dv[4], uv[4];
        ld4(d + (size_t)y * dp, x0, W, vec.src, dv);
        ld4(u + (size_t)y * up, x0, W, vec.dst, uv);
#pragma unroll
        for (int j = 0; j < 4; ++j) uv[j] = fmaf(w, dv[j], uv[j]);
        st4(u + (size_t)y * up, x0, W, vec.dst, uv);
    }
}

// ---- multilevel ----------------------------------------------------------------------
// Four consecutive values of storage type T as floats (one 8- or 16-byte load
// where the row allows it).
template <typename T>
__device__ __forceinline__ void ld4t(const T* __restrict__ row, int x0, int W, bool vec, float (&v)[4]) {
    if (vec && x0 + 3 < W) {
        if constexpr (sizeof(T) == 4) {
            const float4 t = *reinterpret_cast<const float4*>(row + x0);
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
            const uint2 t = *reinterpret_cast<const uint2*>(row + x0);
            const T* h = reinterpret_cast<const T*>(&t);
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = to_f(h[j]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = x0 + j < W ? to_f(row[x0 + j]) : 0.f;
    }
}

// u = fl32(u + s_c e) on unknown pixels, e in storage T.  The product and the
// sum are formed by error-free FP32 transformations: s_c is split into two
// floats, s_hi e is split exactly by an FMA, and the addition to u is a TwoSum,
// so the one rounding to FP32 at the end is the only error beyond about 2^-48
// relative.  The result is that of the FP64 formula fl32(u + s_c e) except in
// rare near-tie cases, without the FP64 pipe, which is slow on this GPU.
// Vectorised layout: 4 columns x V_ROWS rows per thread.
template <typename T>
__global__ void __launch_bounds__(V_TPB) correct_kernel(int H, int W, float* __restrict__ u, int up, long long uplane,
                                                        const T* __restrict__ e0, const T* __restrict__ e1,
                                                        const int* __restrict__ sel, int ep, long long eplane,
                                                        const uint8_t* __restrict__ mask, int mp,
                                                        const double* __restrict__ scale, const int* __restrict__ skip,
                                                        CopyVec vec) {
    if (skip != nullptr && *skip != 0) return;
    const int c = blockIdx.z;
    const int x0 = (blockIdx.x * V_TX + threadIdx.x) * 4;
    const int yb = (blockIdx.y * V_TY + threadIdx.y) * V_ROWS;
    if (x0 >= W) return;
    const T* __restrict__ e = ((sel != nullptr && sel[0]) ? e1 : e0) + c * eplane;
    float* __restrict__ uc = u + c * uplane;
    const double sd = scale[c];
    const float s_hi = (float)sd, s_lo = (float)(sd - (double)s_hi);
#pragma unroll
    for (int k = 0; k < V_ROWS; ++k) {
        const int y = yb + k;
        if (y >= H) break;
        float uv[4], ev[4];
        bool m[4];
        ld4(uc + (size_t)y * up, x0, W, vec.dst, uv);
        ldm4(mask + (size_t)y * mp, x0, W, vec.m, m);
        ld4t<T>(e + (size_t)y * ep, x0, W, vec.src, ev);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float p = s_hi * ev[j];
            const float pl = fmaf(s_lo, ev[j], fmaf(s_hi, ev[j], -p));   // the product's low part
            float t, te;
            two_sum(uv[j], p, t, te);
            if (!m[j]) uv[j] = t + (te + pl);
        }
        st4(uc + (size_t)y * up, x0, W, vec.dst, uv);
    }
}

// Outer control of the device-driven correction loop (one thread), after the
// FP64-accurate residual of u (res_out[c] = {sum r^2, max |r|}).  ctl: [0]
// corrections applied, [1] inner sweeps applied, [2] outcome (0 running,
// 1 converged, 2 limit reached, 3 NaN/Inf, 4 a bounded wait gave up: *err != 0),
// [3] outer passes, [4] inner loop
// passes, [5] skip (the rest of this pass does nothing).  First the previous
// inner solve is added up (inner_state[1] full sweeps, inner_ctl[0] passes);
// then either the loop ends (condition cleared) or the next correction's
// scales are set: scale = max |r|, scale_inv = 1 / scale, inner_ref =
// ||r|| / scale (the inner solve's reference norm).
__global__ void ref_outer_ctl_kernel(const double2* __restrict__ res_out, const double* __restrict__ ref, int C,
                                     const double* __restrict__ tol, int max_corr, int max_sweeps,
                                     const int* __restrict__ inner_state, const int* __restrict__ inner_ctl,
                                     const int* __restrict__ err, int* __restrict__ ctl, double* __restrict__ scale,
                                     double* __restrict__ scale_inv, double* __restrict__ inner_ref,
                                     cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0) return;
    const int passes = ctl[3] + 1;
    ctl[3] = passes;
    if (ctl[0] > 0) {
        ctl[1] += inner_state[1];
        ctl[4] += inner_ctl[0];
    }
    double worst = 0.0;
    bool bad = false;
    for (int c = 0; c < C; ++c) {
        const double s = res_out[c].x;
        if (!isfinite(s)) bad = true;
        const double den = ref[c] > 0.0 ? ref[c] : 1.0;
        worst = fmax(worst, sqrt(s) / den);
    }
    int done = 0;
    if (*err != 0) done = 4;
    else if (bad) done = 3;
    else if (worst <= *tol) done = 1;
    else if (ctl[0] >= max_corr || ctl[1] >= max_sweeps || passes > max_corr + 1) done = 2;
    if (done == 0) {
        for (int c = 0; c < C; ++c) {
            const double sc = res_out[c].y > 0.0 ? res_out[c].y : 1.0;
            scale[c] = sc;
            scale_inv[c] = 1.0 / sc;
            inner_ref[c] = sqrt(res_out[c].x) / sc;
        }
        ctl[0] += 1;
    }
    ctl[2] = done;
    ctl[5] = done != 0;
    if (done != 0) cudaGraphSetConditional(cond, 0);
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
                                         double* __restrict__ tol_d, double tol, const int* __restrict__ skip_if) {
    const bool skip = skip_if != nullptr && *skip_if != 0;
    if (threadIdx.x < 4) state[threadIdx.x] = threadIdx.x == 0 ? cur : 0;
    if (threadIdx.x < 5) flag[threadIdx.x] = (threadIdx.x == 0 && skip) ? 4 : 0;   // 4: sequence skipped
    if (threadIdx.x == 6) flag[6] = 0;
    if (threadIdx.x == 0) *tol_d = tol;
}

// Entry of a device loop: pass counter to 0 and the loop's condition to 1.  A
// graph resets conditions to their default only when it is launched, so a
// loop nested in another loop's body is re-armed here on every entry.
__global__ void loop_begin_kernel(int* __restrict__ ctl, cudaGraphConditionalHandle cond) {
    if (threadIdx.x < 4) ctl[threadIdx.x] = 0;
    if (threadIdx.x == 0) cudaGraphSetConditional(cond, 1);
}

// The decision, after a fine sweep, whether the coarse-grid correction follows
// it (returns 1 to skip it).  gate: [0] skip this pass's correction, [1]
// corrections off (trigger 0) or paused (trigger > 0), [2] corrections
// applied, [3] full fine sweeps seen at the last decision, [4] the last full
// pass was corrected, [5] the trigger has fired, [6] gate launches (counted by
// corr_gate_kernel), [7] consecutive slow passes.  prev[0]: the fine residual w at the last full pass
// (w = norms2[2C], the worst relative residual of the latest full sweep's
// input, i.e. of the previous pass's output); prev[1]: the contraction of the
// slow pass that fired the trigger (or resumed the corrections).
//  - A probe pass (state[1], the count of full sweeps, did not grow) changed
//    no iterate: no correction, no history.
//  - trigger > 0: a pass that reduced w by less than trigger while w is still
//    above kTriggerMargin tol is slow (the residual is dominated by a smooth
//    mode that the sweeps contract slowly; close to tol a correction cannot
//    pay).  No pass is corrected until the second slow pass in a row, which
//    sets [5]; the later passes are corrected.  trigger = 0: every pass is
//    corrected.
//  - A corrected pass that reduced w by less than kGateRatio (after a trigger:
//    by less than the slow pass's own contraction, if that is larger) switches
//    corrections off: for good with trigger 0 (with the non-symmetric ORAS
//    smoother the corrected iteration can grow slowly where plain ORAS
//    converges), and with a trigger only until a plain pass is slow again (a
//    smooth correction can remove error without moving the residual much).
constexpr double kGateRatio = 0.7;
constexpr double kTriggerMargin = 4.0;

__device__ int corr_gate_decide(const int* __restrict__ flag, const double* __restrict__ norms2, int C,
                                const int* __restrict__ state, int* __restrict__ gate, double* __restrict__ prev,
                                double trigger, const double* __restrict__ tol) {
    int skip = flag[0] != 0 || (trigger <= 0.0 && gate[1] != 0);
    if (!skip) {
        const int nfull = state[1];
        if (nfull == gate[3]) {
            skip = 1;   // a probe
        } else {
            gate[3] = nfull;
            const double w = norms2[2 * C], wp = prev[0];
            const bool slow = trigger > 0.0 && wp > 0.0 && w > trigger * wp && w > kTriggerMargin * tol[0];
            gate[7] = slow ? gate[7] + 1 : 0;
            if (trigger > 0.0 && gate[5] == 0) {   // plain passes until the second slow one in a row
                if (gate[7] >= 2) {
                    gate[5] = 1;
                    prev[1] = w / wp;
                }
                skip = 1;
            } else if (gate[1] != 0) {             // paused: resume after a slow plain pass
                if (slow) {
                    gate[1] = 0;
                    prev[1] = w / wp;
                } else {
                    skip = 1;
                }
            } else if (wp > 0.0 && gate[4] != 0 && !(w <= fmax(kGateRatio, prev[1]) * wp)) {
                gate[1] = 1;
                skip = 1;
            }
            prev[0] = w;
            gate[4] = skip ? 0 : 1;
        }
    }
    gate[0] = skip;
    if (!skip) gate[2] += 1;
    return skip;
}

// The gate ahead of the correction kernels, which read gate[0].
__global__ void corr_gate_kernel(const int* __restrict__ flag, const double* __restrict__ norms2, int C,
                                 const int* __restrict__ state, int* __restrict__ gate, double* __restrict__ prev,
                                 double trigger, const double* __restrict__ tol) {
    if (threadIdx.x != 0) return;
    gate[6] += 1;
    (void)corr_gate_decide(flag, norms2, C, state, gate, prev, trigger, tol);
}

__global__ void loop_ctl_kernel(const int* __restrict__ flag, const int* __restrict__ state, int* __restrict__ ctl,
                                int cap, int max_passes, cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0) return;
    const int passes = ctl[0] + 1;
    ctl[0] = passes;
    if (flag[0] != 0 || state[1] >= cap || passes >= max_passes) cudaGraphSetConditional(cond, 0);
}

// Loop control of the plain phase of a fine level with a correction trigger
// (body: sweep -> this kernel): the loop also ends once the trigger fires, and
// the corrected phase's loop (loop_begin_corrected_kernel) takes over.
__global__ void loop_ctl_trigger_kernel(const int* __restrict__ flag, const int* __restrict__ state,
                                        int* __restrict__ ctl, int cap, int max_passes,
                                        cudaGraphConditionalHandle cond, const double* __restrict__ norms2, int C,
                                        int* __restrict__ gate, double* __restrict__ prev, double trigger,
                                        const double* __restrict__ tol) {
    if (threadIdx.x != 0) return;
    (void)corr_gate_decide(flag, norms2, C, state, gate, prev, trigger, tol);
    const int passes = ctl[0] + 1;
    ctl[0] = passes;
    if (flag[0] != 0 || state[1] >= cap || passes >= max_passes || gate[5] != 0) cudaGraphSetConditional(cond, 0);
}

// Entry of the corrected phase's loop: it runs only if the trigger fired and
// the level is still iterating; the pass counter continues from the plain
// phase, so both phases together stay within max_passes.
__global__ void loop_begin_corrected_kernel(const int* __restrict__ ctl, const int* __restrict__ flag,
                                            const int* __restrict__ state, const int* __restrict__ gate, int cap,
                                            int max_passes, cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0) return;
    const bool go = gate[5] != 0 && flag[0] == 0 && state[1] < cap && ctl[0] < max_passes;
    cudaGraphSetConditional(cond, go ? 1u : 0u);
}

}  // namespace

cudaError_t launch_masked_copy(int H, int W, int C, const float* src, int sp, long long splane,
                               const uint8_t* mask, int mp, float* dst, int dp, long long dplane,
                               cudaStream_t st, unsigned long long* count) {
    const CopyVec v{vec_ok(src, sp, splane, 4), vec_ok(dst, dp, dplane, 4), vec_ok(mask, mp, 0, 1)};
    masked_copy_kernel<<<gridv(H, W, C), dim3(V_TX, V_TY), 0, st>>>(H, W, src, sp, splane, mask, mp, dst, dp,
                                                                    dplane, v, count);
    return cudaGetLastError();
}

cudaError_t launch_copy2d(int H, int W, int C, const float* src, int sp, long long splane, float* dst,
                          int dp, long long dplane, cudaStream_t st) {
    const CopyVec v{vec_ok(src, sp, splane, 4), vec_ok(dst, dp, dplane, 4), false};
    masked_copy_kernel<<<gridv(H, W, C), dim3(V_TX, V_TY), 0, st>>>(H, W, src, sp, splane, nullptr, 0, dst, dp,
                                                                    dplane, v, nullptr);
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

int res64_blocks(int H, int W) {
    const dim3 g = grid_res(H, W, 1);
    return (int)(g.x * g.y);
}

// One wave of resident blocks of a V_TPB-thread kernel on the current device
// (0 if the device cannot be queried).
template <typename K>
int wave_blocks(K kernel) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, V_TPB, 0) != cudaSuccess)
        return 0;
    return sms * std::max(per, 1);
}

// Blocks per channel (or per segment) of a grid-stride pass over `tiles`
// tiles with `groups` channels: about one wave in all, at least one block per
// group, at most one per tile.
int stride_blocks(int wave, int groups, int tiles) { return std::max(1, std::min(tiles, wave / std::max(groups, 1))); }

cudaError_t launch_res64(const Res64Args& a, cudaStream_t st) {
    const dim3 tiles = grid_res(a.H, a.W, 1);
    if (a.nblk < (int)(tiles.x * tiles.y)) return cudaErrorInvalidValue;
    const int wave = wave_blocks(res64_kernel<float>);
    if (wave <= 0) return cudaErrorInvalidDevice;
    const dim3 grid(stride_blocks(wave, a.C, (int)(tiles.x * tiles.y)), 1, a.C);
    if (a.out != nullptr && a.ticket == nullptr) return cudaErrorInvalidValue;
    if (a.sel != nullptr && a.u1 == nullptr) return cudaErrorInvalidValue;
    ResVec v;
    v.u = vec_ok(a.u, a.up, a.uplane, 4) && (a.u1 == nullptr || vec_ok(a.u1, a.up, a.uplane, 4));
    v.cp = a.copy_out != nullptr && vec_ok(a.copy_out, a.cp, a.cplane, 4);
    v.m = vec_ok(a.mask, a.mp, 0, 1);
    v.g = a.g_out != nullptr && a.gst == Store::F32 && vec_ok(a.g_out, a.gp, a.gplane, 4);
    const dim3 block(V_TX, V_TY);
    switch (a.gst) {
        case Store::F32: res64_kernel<float><<<grid, block, 0, st>>>(a, v); break;
        case Store::F16: res64_kernel<__half><<<grid, block, 0, st>>>(a, v); break;
        case Store::BF16: res64_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(a, v); break;
    }
    return cudaGetLastError();
}

int ref_norm_part_words(int H, int W, int nl) { return nl * res64_blocks(H, W); }

cudaError_t launch_ref_norms(RefNormArgs a, cudaStream_t st) {
    if (a.nl < 1 || a.nl > kRefMaxLevels || a.C < 1 || a.part == nullptr || a.ticket == nullptr)
        return cudaErrorInvalidValue;
    for (int l = 0; l < a.nl; ++l) {
        RefLevel& L = a.lv[l];
        const dim3 g = grid_res(L.H, L.W, 1);
        L.gx = (int)g.x;
        L.gy = (int)g.y;
        L.mvec = vec_ok(L.mask, L.mp, 0, 1) ? 1 : 0;
        if (!vec_ok(L.f, L.fp, L.fplane, 4) || L.out == nullptr || L.sqrt_out == nullptr) return cudaErrorInvalidValue;
    }
    const int wave = wave_blocks(ref_norms_kernel);
    if (wave <= 0) return cudaErrorInvalidDevice;
    // the blocks per segment suit the finest level, whose segments hold most tiles
    const int gx = stride_blocks(wave, a.C, a.lv[0].gx * a.lv[0].gy);
    if ((long long)gx * a.nl * a.C > a.part_capacity) return cudaErrorInvalidValue;
    ref_norms_kernel<<<dim3(gx, a.nl * a.C), dim3(V_TX, V_TY), 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_restrict(int H, int W, int C, const uint8_t* mask, int mp, const float* f, int fp,
                            long long fplane, uint8_t* mask_c, int mcp, float* f_c, int fcp, long long fcplane,
                            cudaStream_t st) {
    const int Hc = (H + 1) / 2, Wc = (W + 1) / 2;
    const CopyVec v{vec_ok(f, fp, fplane, 4), vec_ok(f_c, fcp, fcplane, 4), vec_ok(mask, mp, 0, 1)};
    restrict_kernel<<<gridv(Hc, Wc, C), dim3(V_TX, V_TY), 0, st>>>(H, W, Hc, Wc, mask, mp, f, fp, fplane, mask_c,
                                                                   mcp, f_c, fcp, fcplane, v);
    return cudaGetLastError();
}

cudaError_t launch_prolong(int Hc, int Wc, int H, int W, int C, const float* uc, int ucp, long long ucplane,
                           const uint8_t* mask, int mp, const float* f, int fp, long long fplane, float* u, int up,
                           long long uplane, cudaStream_t st) {
    const CopyVec v{mask != nullptr && vec_ok(f, fp, fplane, 4), vec_ok(u, up, uplane, 4),
                    mask != nullptr && vec_ok(mask, mp, 0, 1)};
    prolong_kernel<<<gridv(H, W, C), dim3(V_TX, V_TY), 0, st>>>(Hc, Wc, H, W, uc, uc, nullptr, ucp, ucplane, mask,
                                                                mp, f, fp, fplane, u, up, uplane, v);
    return cudaGetLastError();
}

cudaError_t launch_correct(int H, int W, int C, float* u, int up, long long uplane, const void* e, Store est,
                           int ep, long long eplane, const uint8_t* mask, int mp, const double* scale,
                           cudaStream_t st, const void* e1, const int* sel, const int* skip) {
    if (e1 == nullptr) e1 = e;
    const int es = (int)store_bytes(est);
    // e rows as 4-element vectors: 16 bytes (FP32) or 8 bytes (FP16 / BF16)
    auto evec = [&](const void* p) {
        return (reinterpret_cast<uintptr_t>(p) & (uintptr_t)(4 * es - 1)) == 0 && ((long long)ep * es) % (4 * es) == 0 &&
               (eplane * es) % (4 * es) == 0;
    };
    const CopyVec v{evec(e) && evec(e1), vec_ok(u, up, uplane, 4), vec_ok(mask, mp, 0, 1)};
    const dim3 grid = gridv(H, W, C), block(V_TX, V_TY);
    switch (est) {
        case Store::F32:
            correct_kernel<float><<<grid, block, 0, st>>>(H, W, u, up, uplane, static_cast<const float*>(e),
                                                          static_cast<const float*>(e1), sel, ep, eplane, mask, mp,
                                                          scale, skip, v);
            break;
        case Store::F16:
            correct_kernel<__half><<<grid, block, 0, st>>>(H, W, u, up, uplane, static_cast<const __half*>(e),
                                                           static_cast<const __half*>(e1), sel, ep, eplane, mask, mp,
                                                           scale, skip, v);
            break;
        case Store::BF16:
            correct_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(
                H, W, u, up, uplane, static_cast<const __nv_bfloat16*>(e), static_cast<const __nv_bfloat16*>(e1), sel,
                ep, eplane, mask, mp, scale, skip, v);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ref_outer_ctl(const double2* res_out, const double* ref, int C, const double* tol, int max_corr,
                                 int max_sweeps, const int* inner_state, const int* inner_ctl, const int* err,
                                 int* ctl, double* scale, double* scale_inv, double* inner_ref,
                                 cudaGraphConditionalHandle cond, cudaStream_t st) {
    ref_outer_ctl_kernel<<<1, 32, 0, st>>>(res_out, ref, C, tol, max_corr, max_sweeps, inner_state, inner_ctl, err,
                                           ctl, scale, scale_inv, inner_ref, cond);
    return cudaGetLastError();
}

}  // namespace dd

namespace dd {

cudaError_t launch_resolve(const int* flag, const int* sweep_state, const int* ctl, int* out, cudaStream_t st) {
    resolve_kernel<<<1, 1, 0, st>>>(flag, sweep_state, ctl, out);
    return cudaGetLastError();
}

cudaError_t launch_reset_sweep_state(int* state, int* flag, int cur, double* tol_d, double tol, cudaStream_t st,
                                     const int* skip_if) {
    reset_sweep_state_kernel<<<1, 32, 0, st>>>(state, flag, cur, tol_d, tol, skip_if);
    return cudaGetLastError();
}

cudaError_t launch_restrict_sum(int H, int W, int C, const float* src, int sp, long long splane, float* dst, int dp,
                                long long dplane, const int* skip, cudaStream_t st) {
    const int Hc = (H + 1) / 2, Wc = (W + 1) / 2;
    const CopyVec v{vec_ok(src, sp, splane, 4), vec_ok(dst, dp, dplane, 4), false};
    restrict_sum_kernel<<<gridv(Hc, Wc, C), dim3(V_TX, V_TY), 0, st>>>(H, W, Hc, Wc, src, sp, splane, dst, dp, dplane,
                                                                       skip, v);
    return cudaGetLastError();
}

cudaError_t launch_corr_gate(const int* flag, const double* norms2, int C, const int* state, int* gate, double* prev,
                             double trigger, const double* tol, cudaStream_t st) {
    corr_gate_kernel<<<1, 32, 0, st>>>(flag, norms2, C, state, gate, prev, trigger, tol);
    return cudaGetLastError();
}

cudaError_t launch_corr_dir(int Hc, int Wc, int H, int W, int C, const float* ec0, const float* ec1, const int* sel_c,
                            int ecp, long long ecplane, const uint8_t* mask, int mp, float* rd, int rp,
                            long long rplane, const int* skip, double* part, int nblk, unsigned int* ticket,
                            double* out, cudaStream_t st) {
    const dim3 grid = gridv(H, W, C);
    if (nblk != (int)(grid.x * grid.y)) return cudaErrorInvalidValue;
    const CopyVec v{false, vec_ok(rd, rp, rplane, 4), vec_ok(mask, mp, 0, 1)};
    const DotTail t{part, nblk, ticket, out, nullptr, nullptr};
    corr_dir_kernel<<<grid, dim3(V_TX, V_TY), 0, st>>>(Hc, Wc, H, W, C, ec0, ec1, sel_c, ecp, ecplane, mask, mp, rd, rp,
                                                       rplane, skip, t, v);
    return cudaGetLastError();
}

cudaError_t launch_corr_curv(int H, int W, int C, const float* d, int dp, long long dplane, const int* skip,
                             double* part, int nblk, unsigned int* ticket, double* out, const double* num,
                             double* omega, cudaStream_t st) {
    const dim3 grid = gridv(H, W, C);
    if (nblk != (int)(grid.x * grid.y)) return cudaErrorInvalidValue;
    const CopyVec v{vec_ok(d, dp, dplane, 4), false, false};
    const DotTail t{part, nblk, ticket, out, num, omega};
    corr_curv_kernel<<<grid, dim3(V_TX, V_TY), 0, st>>>(H, W, C, d, dp, dplane, skip, t, v);
    return cudaGetLastError();
}

cudaError_t launch_corr_step(int H, int W, int C, const float* d, int dp, long long dplane, const double* omega,
                             float* u0, float* u1, const int* sel_u, int up, long long uplane, const int* skip,
                             cudaStream_t st) {
    const CopyVec v{vec_ok(d, dp, dplane, 4), vec_ok(u0, up, uplane, 4) && vec_ok(u1, up, uplane, 4), false};
    corr_step_kernel<<<gridv(H, W, C), dim3(V_TX, V_TY), 0, st>>>(H, W, d, dp, dplane, omega, u0, u1, sel_u, up,
                                                                  uplane, skip, v);
    return cudaGetLastError();
}

const void* loop_begin_kernel_fn() { return reinterpret_cast<const void*>(&loop_begin_kernel); }

cudaError_t launch_loop_ctl(const int* flag, const int* state, int* ctl, int cap, int max_passes,
                            cudaGraphConditionalHandle cond, cudaStream_t st) {
    loop_ctl_kernel<<<1, 32, 0, st>>>(flag, state, ctl, cap, max_passes, cond);
    return cudaGetLastError();
}

cudaError_t launch_loop_ctl_trigger(const int* flag, const int* state, int* ctl, int cap, int max_passes,
                                    cudaGraphConditionalHandle cond, const double* norms2, int C, int* gate,
                                    double* prev, double trigger, const double* tol, cudaStream_t st) {
    loop_ctl_trigger_kernel<<<1, 32, 0, st>>>(flag, state, ctl, cap, max_passes, cond, norms2, C, gate, prev,
                                              trigger, tol);
    return cudaGetLastError();
}

const void* loop_begin_corrected_kernel_fn() { return reinterpret_cast<const void*>(&loop_begin_corrected_kernel); }

cudaError_t launch_prolong_sel(int Hc, int Wc, int H, int W, int C, const float* uc0, const float* uc1,
                               const int* sel, int ucp, long long ucplane, const uint8_t* mask, int mp,
                               const float* f, int fp, long long fplane, float* u, int up, long long uplane,
                               cudaStream_t st) {
    const CopyVec v{vec_ok(f, fp, fplane, 4), vec_ok(u, up, uplane, 4), vec_ok(mask, mp, 0, 1)};
    prolong_kernel<<<gridv(H, W, C), dim3(V_TX, V_TY), 0, st>>>(Hc, Wc, H, W, uc0, uc1, sel, ucp, ucplane, mask,
                                                                mp, f, fp, fplane, u, up, uplane, v);
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
