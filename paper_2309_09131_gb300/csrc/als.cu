// als.cu -- K7/K8: one CP-ALS iteration (Algorithm 1) on the GPU.
//
// Algorithm 1 writes each factor update as an spMTTKRP followed by a column
// normalisation; the least-squares solve between the two is the Kolda-Bader
// update Y_n <- M_n (hadamard_{w != n} Y_w^T Y_w)^{-1}.  Per mode n, in order
// 0..N-1 (Gauss-Seidel, each update sees the newest factors):
//   1. M_n: one fused spMTTKRP + remap pass (K2 + K4), L_n -> L_{n+1};
//   2. V = hadamard_{w != n} G_w in FP64 (R x R);
//   3. V = L D L^T and W = V^{-1} in FP64 (R/8 blocks, one column of W per
//      warp); a pivot that is not positive ends the step with
//      FLYCOO_ERR_NOT_SPD;
//   4. Y = M_n W with W in FP64 and the sums carried in double-float (below),
//      and the column sums of squares of Y in FP64;
//   5. lambda_r = column 2-norm (FP64); Y_n = Y / lambda in FP64, rounded to
//      FP32, then to BF16 when the factors are stored in BF16;
//   6. G_n = Y_n^T Y_n from the stored factor.
// The long sums of steps 4 and 6 (over I_n rows or R terms) are carried as
// double-float pairs (hi, lo) of FP32 values: each product a*b is split
// exactly into p + e with an FMA (e = fma(a, b, -p)), p is added to hi with
// Knuth's two-sum, and the rounding errors go to lo.  A pair keeps about 46
// significant bits, so the Gram matrices and M_n W come out with FP64-level
// accuracy at FP32 rates (FP64 runs at a small fraction of the FP32 rate on
// this GPU).  Every operation of a pair uses the _rn intrinsics, which the
// compiler never contracts into FMAs.  Chunk sums of pairs are accumulated in
// FP64, and the blocks' partials are added in a fixed order.  After the last
// mode
//   fit = 1 - sqrt(||X||^2 + ||Xhat||^2 - 2 <X, Xhat>) / ||X||,
//   ||Xhat||^2 = lambda^T (hadamard_w G_w) lambda,
//   <X, Xhat>  = sum_r lambda_r sum_i M_{N-1}[i,r] Y_{N-1}[i,r].
// Every reduction has a fixed order, so an iteration is bitwise reproducible.
#include "internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

namespace flycoo {
namespace {

constexpr int kAlsThreads = 256;

// (hi, lo) += a * (bhi + blo): the product a * bhi is split exactly into
// p + e, p joins hi by two-sum, and the rounding terms (with a * blo) join lo
__device__ __forceinline__ void df_fma(float &hi, float &lo, float a, float bhi, float blo) {
    const float p = __fmul_rn(a, bhi);
    const float e = __fmaf_rn(a, bhi, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, __fmaf_rn(a, blo, e)));
}

// (hi, lo) += a * b
__device__ __forceinline__ void df_fma(float &hi, float &lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, e));
}

template <bool BF16> __device__ __forceinline__ float load_factor(const void *Y, u64 i) {
    if constexpr (BF16) return __bfloat162float(static_cast<const __nv_bfloat16 *>(Y)[i]);
    else return static_cast<const float *>(Y)[i];
}

__device__ __forceinline__ void block_rows(u64 I, u64 &lo, u64 &hi) {
    const u64 per = (I + gridDim.x - 1) / gridDim.x;
    lo = min((u64)blockIdx.x * per, I);
    hi = min(lo + per, I);
}

// Gram partials: partials[b][a*R + c] = sum over the rows of block b of Y[i,a] Y[i,c].
// A block stages chunks of rows (32 KB of FP32) in shared memory with 16-byte
// loads.  Thread t of row group g owns the B x B tile at (a0, c0) and sums the
// products of the group's rows of the chunk as double-float pairs; the chunk
// sums are accumulated in FP64, and the groups' partials are added in group
// order.
template <int R> struct GramCfg {
    static constexpr int B = (R >= 32) ? 4 : 2;      // register tile per thread
    static constexpr int TB = R / B;                 // tiles per matrix row
    static constexpr int TPG = TB * TB;              // threads per row group
    static constexpr int NG = kAlsThreads / TPG;     // row groups
    static constexpr int ROWS = 8192 / R;            // rows per chunk (32 KB of FP32)
    static_assert(NG >= 1 && NG * R * R * 8 <= ROWS * R * 4, "group partials must fit the chunk buffer");
};

template <int R, bool BF16>
__global__ void __launch_bounds__(kAlsThreads) gram_partial_kernel(const void *Y, u64 I, double *partials) {
    using C = GramCfg<R>;
    constexpr int B = C::B, NG = C::NG, ROWS = C::ROWS;
    __shared__ __align__(16) float rows[ROWS * R];
    u64 lo, hi;
    block_rows(I, lo, hi);
    const int g = threadIdx.x / C::TPG, tig = threadIdx.x % C::TPG;
    const int a0 = (tig / C::TB) * B, c0 = (tig % C::TB) * B;
    double acc[B][B];
#pragma unroll
    for (int x = 0; x < B; ++x)
#pragma unroll
        for (int y = 0; y < B; ++y) acc[x][y] = 0.0;
    for (u64 r0 = lo; r0 < hi; r0 += ROWS) {
        const int nr = (int)min((u64)ROWS, hi - r0);
        __syncthreads();
        if constexpr (BF16) {
            const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(Y) + r0 * R);
            for (int e = threadIdx.x; e < nr * R / 8; e += kAlsThreads) {
                const uint4 v = src[e];
                const u32 wv[4] = {v.x, v.y, v.z, v.w};
                float4 *dst = reinterpret_cast<float4 *>(rows + e * 8);
                dst[0] = make_float4(__uint_as_float(wv[0] << 16), __uint_as_float(wv[0] & 0xffff0000u),
                                     __uint_as_float(wv[1] << 16), __uint_as_float(wv[1] & 0xffff0000u));
                dst[1] = make_float4(__uint_as_float(wv[2] << 16), __uint_as_float(wv[2] & 0xffff0000u),
                                     __uint_as_float(wv[3] << 16), __uint_as_float(wv[3] & 0xffff0000u));
            }
        } else {
            const float4 *src = reinterpret_cast<const float4 *>(static_cast<const float *>(Y) + r0 * R);
            for (int e = threadIdx.x; e < nr * R / 4; e += kAlsThreads) reinterpret_cast<float4 *>(rows)[e] = src[e];
        }
        __syncthreads();
        float hi[B][B], lo[B][B];
#pragma unroll
        for (int x = 0; x < B; ++x)
#pragma unroll
            for (int y = 0; y < B; ++y) hi[x][y] = lo[x][y] = 0.f;
        for (int i = g; i < nr; i += NG) {
            float va[B], vc[B];
#pragma unroll
            for (int x = 0; x < B; ++x) {
                va[x] = rows[i * R + a0 + x];
                vc[x] = rows[i * R + c0 + x];
            }
#pragma unroll
            for (int x = 0; x < B; ++x)
#pragma unroll
                for (int y = 0; y < B; ++y) df_fma(hi[x][y], lo[x][y], va[x], vc[y]);
        }
#pragma unroll
        for (int x = 0; x < B; ++x)
#pragma unroll
            for (int y = 0; y < B; ++y) acc[x][y] += (double)hi[x][y] + (double)lo[x][y];
    }
    __syncthreads();
    double *gp = reinterpret_cast<double *>(rows); // [NG][R*R]
#pragma unroll
    for (int x = 0; x < B; ++x)
#pragma unroll
        for (int y = 0; y < B; ++y) gp[g * R * R + (a0 + x) * R + c0 + y] = acc[x][y];
    __syncthreads();
    for (int e = threadIdx.x; e < R * R; e += kAlsThreads) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < NG; ++q) t += gp[q * R * R + e];
        partials[(size_t)blockIdx.x * R * R + e] = t;
    }
}

// out[e] = sum over b < nblocks of partials[b * len + e] (sqrt of it with
// take_sqrt), in a fixed order: warp q of a block sums b = q, q + 8, ... for 32
// consecutive e, then the 8 warp sums are added in warp order.  Skipped when
// *status is set.
__global__ void __launch_bounds__(256) reduce_partials_kernel(const double *partials, int nblocks, int len,
                                                              double *out, int take_sqrt, const u32 *status) {
    __shared__ double part[8][32];
    if (status && *status) return;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (e < len)
        for (int b = wq; b < nblocks; b += 8) s += partials[(size_t)b * len + e];
    part[wq][lane] = s;
    __syncthreads();
    if (wq == 0 && e < len) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += part[q][lane];
        out[e] = take_sqrt ? sqrt(t) : t;
    }
}

// FP64 is a narrow pipe on this GPU, so a serial chain of FP64 divisions is
// slow.  1/d: an FP32 estimate refined by two Newton-Raphson steps
// r <- r + r (1 - d r); each step squares the relative error (2^-23 -> 2^-46
// -> FP64 rounding).  Outside the range where the FP32 estimate is accurate the
// plain division is used.
__device__ __forceinline__ double recip_f64(double d) {
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / d;
    double r = (double)__frcp_rn((float)d);
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

constexpr int kInvWarps = 8; // columns of the inverse per block, one per warp

// W = V^{-1} for V = hadamard_{w != n} G_w (R x R, symmetric), in FP64, by the
// factorisation V = L D L^T (L unit lower triangular, D diagonal): a
// positive-definite V has every pivot d_k > 0, and a pivot <= 0 sets *status.
// Each block factors V itself (R^3/6 FMAs) and then solves kInvWarps columns
// c of W, one per warp, lanes owning rows i = lane and lane + 32:
//   L z = e_c,   y = D^{-1} z,   L^T w = y,   W[:, c] = w.
// Shared memory: V (R x R) and the pivot reciprocals (R).  After the loop the
// strictly lower triangle of V holds L and the strictly upper one L^T.
__global__ void __launch_bounds__(kInvWarps * 32)
    ldl_inverse_kernel(const double *G, int N, int n, int R, double *W, u32 *status) {
    extern __shared__ double inv_smem[];
    double *V = inv_smem, *dinv = inv_smem + R * R;
    __shared__ int bad;
    if (*status) return; // an earlier mode failed: leave the rest untouched
    const int RR = R * R;
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        double v = 1.0;
        for (int w = 0; w < N; ++w)
            if (w != n) v *= G[(size_t)w * RR + e];
        V[e] = v;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < R; ++k) {
        if (threadIdx.x == 0) {
            const double d = V[k * R + k];
            if (!(d > 0.0)) bad = 1;
            else dinv[k] = recip_f64(d);
        }
        __syncthreads();
        if (bad) break;
        const double r = dinv[k];
        // rows i > k: V[i][j] -= V[i][k] L[j][k] for k < j <= i, with
        // L[j][k] = V[j][k] / d_k, and L[i][k] stored at V[k][i] (upper); the
        // update reads column k below the diagonal and writes neither it nor row k
        const int t = R - k - 1;
        for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
            const int i = k + 1 + e / t, j = k + 1 + e % t;
            if (j <= i) V[i * R + j] -= V[i * R + k] * (V[j * R + k] * r);
        }
        for (int i = k + 1 + threadIdx.x; i < R; i += blockDim.x) V[k * R + i] = V[i * R + k] * r;
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0 && blockIdx.x == 0) *status = 1u;
        return;
    }
    // lower triangle: L[i][k] = V[k][i] (copy the scaled values down)
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        const int i = e / R, k = e % R;
        if (k < i) V[i * R + k] = V[k * R + i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kInvWarps + (threadIdx.x >> 5);
    if (c >= R) return;
    const int i0 = lane, i1 = lane + 32; // rows of this lane (R <= 64)
    const bool has0 = i0 < R, has1 = i1 < R;
    // forward: z_i -= L[i][q] z_q for i > q, q = c .. R-2 (z_q = 0 for q < c)
    double z0 = (i0 == c) ? 1.0 : 0.0, z1 = (i1 == c) ? 1.0 : 0.0;
    for (int q = c; q < R - 1; ++q) {
        const double zq = __shfl_sync(0xffffffffu, q < 32 ? z0 : z1, q & 31);
        if (has0 && i0 > q) z0 -= V[q * R + i0] * zq; // V[q][i] = L[i][q] (upper copy)
        if (has1 && i1 > q) z1 -= V[q * R + i1] * zq;
    }
    if (has0) z0 *= dinv[i0];
    if (has1) z1 *= dinv[i1];
    // backward: w_i -= L[q][i] w_q for i < q, q = R-1 .. 1
    for (int q = R - 1; q > 0; --q) {
        const double wq = __shfl_sync(0xffffffffu, q < 32 ? z0 : z1, q & 31);
        if (has0 && i0 < q) z0 -= V[q * R + i0] * wq; // V[q][i] = L[q][i] (lower)
        if (has1 && i1 < q) z1 -= V[q * R + i1] * wq;
    }
    if (has0) W[i0 * R + c] = z0;
    if (has1) W[i1 * R + c] = z1;
}

// Y = M W with W = V^{-1} in FP64.  W is split into FP32 pairs
// (hi, lo) = (fl32(w), fl32(w - hi)) in shared memory; tiles of M (8 KB) are
// staged in shared memory; thread t computes column c = t % R of the tile's
// rows t/R, t/R + 256/R, ..., each as a double-float sum over a of
// M[i,a] * (hi + lo)[a,c] (about 46 significant bits), and stores the pair.
// Per-block column sums of squares of the pairs' values in FP64.
template <int R>
__global__ void __launch_bounds__(kAlsThreads)
    als_apply_kernel(const float *M, const double *W, float2 *Y, u64 I, double *colsq, const u32 *status) {
    constexpr int ROWS = 2048 / R;
    constexpr int rstep = kAlsThreads / R;
    __shared__ __align__(16) float mt[ROWS * R];
    __shared__ float2 wp[R * R];
    __shared__ double part[kAlsThreads];
    if (*status) return;
    for (int e = threadIdx.x; e < R * R; e += kAlsThreads) {
        const double w = W[e];
        const float whi = __double2float_rn(w);
        wp[e] = make_float2(whi, __double2float_rn(w - (double)whi));
    }
    const int c = threadIdx.x % R, rsub = threadIdx.x / R;
    u64 lo, hi;
    block_rows(I, lo, hi);
    double sq = 0.0;
    for (u64 r0 = lo; r0 < hi; r0 += ROWS) {
        const int nr = (int)min((u64)ROWS, hi - r0);
        __syncthreads();
        const float4 *src = reinterpret_cast<const float4 *>(M + r0 * R);
        for (int e = threadIdx.x; e < nr * R / 4; e += kAlsThreads) reinterpret_cast<float4 *>(mt)[e] = src[e];
        __syncthreads();
        for (int i = rsub; i < nr; i += rstep) {
            const float *m = mt + i * R;
            float yh = 0.f, yl = 0.f;
#pragma unroll 8
            for (int a = 0; a < R; ++a) {
                const float2 w = wp[a * R + c];
                df_fma(yh, yl, m[a], w.x, w.y);
            }
            Y[(r0 + i) * R + c] = make_float2(yh, yl);
            const double y = (double)yh + (double)yl;
            sq = fma(y, y, sq);
        }
    }
    part[threadIdx.x] = sq;
    __syncthreads();
    if (threadIdx.x < R) {
        double t = 0.0;
        for (int q = 0; q < rstep; ++q) t += part[q * R + threadIdx.x];
        colsq[(size_t)blockIdx.x * R + threadIdx.x] = t;
    }
}

// factor = Y * (1 / lambda) in FP64 (Y from its double-float pairs), rounded
// to FP32, then to BF16 when stored so; with M set, also the per-block
// partials of sum_i M[i,r] factor[i,r].  Thread t handles the four columns
// 4q..4q+3, q = t % (R/4), of every (256/(R/4))-th row, with 16-byte loads.
template <int R, bool BF16>
__global__ void __launch_bounds__(kAlsThreads)
    normalize_store_kernel(const float2 *Yt, const double *lambda, void *Yout, u64 I, const float *M, double *inner,
                           const u32 *status) {
    constexpr int Q = R / 4;
    constexpr int rstep = kAlsThreads / Q;
    __shared__ double part[4][kAlsThreads];
    if (*status) return;
    const int q = threadIdx.x % Q, rsub = threadIdx.x / Q;
    double inv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double lam = lambda[4 * q + j];
        inv[j] = lam > 0.0 ? 1.0 / lam : 1.0;
    }
    u64 lo, hi;
    block_rows(I, lo, hi);
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (u64 i = lo + rsub; i < hi; i += rstep) {
        const float4 ya = reinterpret_cast<const float4 *>(Yt)[(i * Q + q) * 2];
        const float4 yb = reinterpret_cast<const float4 *>(Yt)[(i * Q + q) * 2 + 1];
        const double y[4] = {(double)ya.x + (double)ya.y, (double)ya.z + (double)ya.w, (double)yb.x + (double)yb.y,
                             (double)yb.z + (double)yb.w};
        float v[4] = {__double2float_rn(y[0] * inv[0]), __double2float_rn(y[1] * inv[1]),
                      __double2float_rn(y[2] * inv[2]), __double2float_rn(y[3] * inv[3])};
        if constexpr (BF16) {
            __nv_bfloat16 b[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                b[j] = __float2bfloat16_rn(v[j]);
                v[j] = __bfloat162float(b[j]);
            }
            uint2 packed;
            packed.x = (u32)__bfloat16_as_ushort(b[0]) | ((u32)__bfloat16_as_ushort(b[1]) << 16);
            packed.y = (u32)__bfloat16_as_ushort(b[2]) | ((u32)__bfloat16_as_ushort(b[3]) << 16);
            reinterpret_cast<uint2 *>(Yout)[i * Q + q] = packed;
        } else {
            reinterpret_cast<float4 *>(Yout)[i * Q + q] = make_float4(v[0], v[1], v[2], v[3]);
        }
        if (M) {
            const float4 m = reinterpret_cast<const float4 *>(M)[i * Q + q];
            s[0] += (double)m.x * (double)v[0];
            s[1] += (double)m.y * (double)v[1];
            s[2] += (double)m.z * (double)v[2];
            s[3] += (double)m.w * (double)v[3];
        }
    }
    if (inner) {
#pragma unroll
        for (int j = 0; j < 4; ++j) part[j][threadIdx.x] = s[j];
        __syncthreads();
        if (threadIdx.x < R) {
            const int cq = threadIdx.x / 4, cj = threadIdx.x % 4;
            double t = 0.0;
            for (int r = 0; r < rstep; ++r) t += part[cj][r * Q + cq];
            inner[(size_t)blockIdx.x * R + threadIdx.x] = t;
        }
    }
}

template <int R>
void launch_normalize_t(bool bf, const float2 *Yt, const double *lambda, void *Yout, u64 I, const float *M,
                        double *inner, const u32 *status, int nblk, cudaStream_t s) {
    if (bf) normalize_store_kernel<R, true><<<nblk, kAlsThreads, 0, s>>>(Yt, lambda, Yout, I, M, inner, status);
    else normalize_store_kernel<R, false><<<nblk, kAlsThreads, 0, s>>>(Yt, lambda, Yout, I, M, inner, status);
}

void launch_normalize(int R, bool bf, const float2 *Yt, const double *lambda, void *Yout, u64 I, const float *M,
                      double *inner, const u32 *status, int nblk, cudaStream_t s) {
    switch (R) {
    case 16: launch_normalize_t<16>(bf, Yt, lambda, Yout, I, M, inner, status, nblk, s); break;
    case 32: launch_normalize_t<32>(bf, Yt, lambda, Yout, I, M, inner, status, nblk, s); break;
    default: launch_normalize_t<64>(bf, Yt, lambda, Yout, I, M, inner, status, nblk, s); break;
    }
}

// sum of part[0 .. kAlsThreads) in a fixed order: each warp adds its 8-value
// strip serially, then thread 0 adds the 32 strip sums in order
__device__ double block_sum_fixed(double *part) {
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kAlsThreads / 32; ++q) t += part[threadIdx.x * (kAlsThreads / 32) + q];
        part[threadIdx.x * (kAlsThreads / 32)] = t;
    }
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < 32; ++q) t += part[q * (kAlsThreads / 32)];
    return t; // valid in thread 0
}

// fit from ||X||^2, the Gram matrices, lambda and the <X, Xhat> partials.  One block.
__global__ void __launch_bounds__(kAlsThreads) fit_kernel(const double *G, int N, int R, const double *lambda,
                                                          const double *inner, int nblocks, const double *normx2,
                                                          double *fit) {
    __shared__ double part[2][kAlsThreads];
    double xh = 0.0, xi = 0.0;
    for (int e = threadIdx.x; e < R * R; e += kAlsThreads) {
        double v = 1.0;
        for (int w = 0; w < N; ++w) v *= G[(size_t)w * R * R + e];
        xh += lambda[e / R] * v * lambda[e % R];
    }
    for (int e = threadIdx.x; e < nblocks * R; e += kAlsThreads) xi += lambda[e % R] * inner[e];
    part[0][threadIdx.x] = xh;
    part[1][threadIdx.x] = xi;
    const double sxh = block_sum_fixed(part[0]);
    const double sxi = block_sum_fixed(part[1]);
    if (threadIdx.x == 0) {
        const double x2 = *normx2;
        const double resid2 = fmax(x2 + sxh - 2.0 * sxi, 0.0);
        *fit = 1.0 - sqrt(resid2) / sqrt(x2);
    }
}

// per-block partials of ||X||^2 = sum of squared nonzero values (FP64)
__global__ void __launch_bounds__(kAlsThreads)
    value_sq_kernel(const u32 *elem, int ew, int N, u64 nnz, double *partials) {
    __shared__ double part[kAlsThreads];
    u64 lo, hi;
    block_rows(nnz, lo, hi);
    double s = 0.0;
    for (u64 p = lo + threadIdx.x; p < hi; p += kAlsThreads) {
        const double v = (double)__uint_as_float(elem[p * (u64)ew + N]);
        s += v * v;
    }
    part[threadIdx.x] = s;
    const double t = block_sum_fixed(part);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

template <int R>
void launch_gram_t(const void *Y, bool bf16, u64 I, double *gpart, int nblk, cudaStream_t s) {
    if (bf16) gram_partial_kernel<R, true><<<nblk, kAlsThreads, 0, s>>>(Y, I, gpart);
    else gram_partial_kernel<R, false><<<nblk, kAlsThreads, 0, s>>>(Y, I, gpart);
}

flycoo_status gram(const void *Y, bool bf16, u64 I, int R, double *G, double *gpart, int nblk, cudaStream_t s) {
    switch (R) {
    case 16: launch_gram_t<16>(Y, bf16, I, gpart, nblk, s); break;
    case 32: launch_gram_t<32>(Y, bf16, I, gpart, nblk, s); break;
    default: launch_gram_t<64>(Y, bf16, I, gpart, nblk, s); break;
    }
    reduce_partials_kernel<<<(R * R + 31) / 32, 256, 0, s>>>(gpart, nblk, R * R, G, 0, nullptr);
    FLY_TRY_CUDA(cudaGetLastError());
    return FLYCOO_OK;
}

void launch_apply(int R, const float *M, const double *W, float2 *Y, u64 I, double *colsq, const u32 *status,
                  int nblk, cudaStream_t s) {
    switch (R) {
    case 16: als_apply_kernel<16><<<nblk, kAlsThreads, 0, s>>>(M, W, Y, I, colsq, status); break;
    case 32: als_apply_kernel<32><<<nblk, kAlsThreads, 0, s>>>(M, W, Y, I, colsq, status); break;
    default: als_apply_kernel<64><<<nblk, kAlsThreads, 0, s>>>(M, W, Y, I, colsq, status); break;
    }
}

} // namespace

flycoo_status als_step(Tensor &t, void *const *F, flycoo_dtype fdt, int R, int iters, double *d_lambda,
                       double *h_fits, cudaStream_t s, const char *who) {
    const int N = t.N;
    const bool bf = fdt == FLYCOO_BF16;
    AlsWork &w = t.als;
    u64 maxI = 0;
    for (int n = 0; n < N; ++n) maxI = std::max<u64>(maxI, t.dims[n]);
    const int nblk = 4 * t.sm_count;
    if (w.rows < maxI || w.nblk != nblk) {
        FLY_TRY(w.M.alloc(maxI * kMaxRank * sizeof(float)));
        FLY_TRY(w.Y.alloc(maxI * kMaxRank * sizeof(float2)));
        FLY_TRY(w.G.alloc((size_t)FLYCOO_MAX_MODES * kMaxRank * kMaxRank * sizeof(double)));
        FLY_TRY(w.gpart.alloc((size_t)nblk * kMaxRank * kMaxRank * sizeof(double)));
        FLY_TRY(w.W.alloc(kMaxRank * kMaxRank * sizeof(double)));
        FLY_TRY(w.colsq.alloc((size_t)nblk * kMaxRank * sizeof(double)));
        FLY_TRY(w.inner.alloc((size_t)nblk * kMaxRank * sizeof(double)));
        FLY_TRY(w.scal.alloc((size_t)(nblk + 4) * sizeof(double)));
        w.rows = maxI;
        w.nblk = nblk;
        w.normx2_valid = false;
    }
    if (w.fits.bytes < (size_t)iters * sizeof(double)) FLY_TRY(w.fits.alloc((size_t)iters * sizeof(double)));
    double *G = w.G.as<double>();
    double *scal = w.scal.as<double>(); // [0] ||X||^2, [1] fit, [2] status word, [4..] partials
    u32 *status = reinterpret_cast<u32 *>(scal + 2);
    // the sweep starts in L_0; ||X||^2 is summed in that order, so the result
    // does not depend on the layout the tensor was left in
    while (t.layout != 0) {
        FLY_TRY(launch_remap_step(t, t.layout, t.elem[t.cur].p, t.elem[1 - t.cur].p, s));
        t.cur = 1 - t.cur;
        t.remap_since_sync = true;
        t.layout = (t.layout + 1) % N;
    }
    if (!w.normx2_valid) {
        if (t.nnz) {
            value_sq_kernel<<<nblk, kAlsThreads, 0, s>>>(t.elem[t.cur].as<u32>(), t.elem_words, N, t.nnz, scal + 4);
            reduce_partials_kernel<<<1, 256, 0, s>>>(scal + 4, nblk, 1, scal, 0, nullptr);
            FLY_TRY_CUDA(cudaGetLastError());
        } else {
            FLY_TRY_CUDA(cudaMemsetAsync(scal, 0, sizeof(double), s));
        }
        FLY_TRY_CUDA(cudaMemcpyAsync(&w.normx2, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        FLY_TRY_CUDA(cudaStreamSynchronize(s));
        w.normx2_valid = true;
    }
    if (!(w.normx2 > 0.0)) {
        set_error("%s: the tensor has no nonzero value (||X|| = 0, fit undefined)", who);
        return FLYCOO_ERR_INVALID_ARG;
    }
    const size_t RR = (size_t)R * R;
    // the Gram matrices of the factors as given; later iterations of this call
    // reuse the ones computed after each update
    for (int n = 0; n < N; ++n) FLY_TRY(gram(F[n], bf, t.dims[n], R, G + n * RR, w.gpart.as<double>(), nblk, s));
    FLY_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(u32), s));
    double *fits = w.fits.as<double>();
    for (int it = 0; it < iters; ++it) {
        for (int n = 0; n < N; ++n) {
            const u64 I = t.dims[n];
            FLY_TRY(run_pass(t, n, F, fdt, R, w.M.as<float>(), nullptr, nullptr, s));
            ldl_inverse_kernel<<<(R + kInvWarps - 1) / kInvWarps, kInvWarps * 32, (RR + R) * sizeof(double), s>>>(
                G, N, n, R, w.W.as<double>(), status);
            launch_apply(R, w.M.as<float>(), w.W.as<double>(), w.Y.as<float2>(), I, w.colsq.as<double>(), status,
                         nblk, s);
            reduce_partials_kernel<<<(R + 31) / 32, 256, 0, s>>>(w.colsq.as<double>(), nblk, R, d_lambda, 1, status);
            const bool last = n == N - 1;
            float *Mlast = last ? w.M.as<float>() : nullptr;
            double *inner = last ? w.inner.as<double>() : nullptr;
            launch_normalize(R, bf, w.Y.as<float2>(), d_lambda, F[n], I, Mlast, inner, status, nblk, s);
            FLY_TRY_CUDA(cudaGetLastError());
            FLY_TRY(gram(F[n], bf, I, R, G + n * RR, w.gpart.as<double>(), nblk, s));
        }
        fit_kernel<<<1, kAlsThreads, 0, s>>>(G, N, R, d_lambda, w.inner.as<double>(), nblk, scal, fits + it);
        FLY_TRY_CUDA(cudaGetLastError());
    }
    double res[3];
    FLY_TRY_CUDA(cudaMemcpyAsync(res, scal, sizeof(res), cudaMemcpyDeviceToHost, s));
    if (h_fits)
        FLY_TRY_CUDA(cudaMemcpyAsync(h_fits, fits, (size_t)iters * sizeof(double), cudaMemcpyDeviceToHost, s));
    FLY_TRY(check_error_word(t, s, who));
    u32 st;
    memcpy(&st, &res[2], sizeof(st));
    if (st) {
        set_error("%s: a normal-equation matrix (hadamard of Gram matrices) is not positive definite; the modes "
                  "before it were updated, the others are unchanged",
                  who);
        return FLYCOO_ERR_NOT_SPD;
    }
    return FLYCOO_OK;
}

} // namespace flycoo
