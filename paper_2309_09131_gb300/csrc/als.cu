// als.cu -- K7/K8: one CP-ALS iteration (Algorithm 1) on the GPU.
//
// Algorithm 1 writes each factor update as an spMTTKRP followed by a column
// normalisation; the least-squares solve between the two is the Kolda-Bader
// update Y_n <- M_n (hadamard_{w != n} Y_w^T Y_w)^{-1}.  Per mode n, in order
// 0..N-1 (Gauss-Seidel, each update sees the newest factors):
//   1. M_n: one fused spMTTKRP + remap pass (K2 + K4), L_n -> L_{n+1};
//   2. V = hadamard_{w != n} G_w in FP64 (R x R);
//   3. Cholesky V = L L^T and W = V^{-1} in FP64, one block; a pivot that is
//      not positive ends the step with FLYCOO_ERR_NOT_SPD;
//   4. Y = M_n W in FP32 (W rounded to FP32) and the column sums of squares;
//   5. lambda_r = column 2-norm (FP64); Y_n = Y / lambda rounded to FP32, then
//      to BF16 when the factors are stored in BF16;
//   6. G_n = Y_n^T Y_n from the stored factor.
// Gram matrices: FP32 products summed over 32 rows, those sums accumulated in
// FP64 per block and the blocks summed in a fixed order.  After the last mode
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
constexpr int kGramRows = 32; // rows whose products are summed in FP32

template <bool BF16> __device__ __forceinline__ float load_factor(const void *Y, u64 i) {
    if constexpr (BF16) return __bfloat162float(static_cast<const __nv_bfloat16 *>(Y)[i]);
    else return static_cast<const float *>(Y)[i];
}

__device__ __forceinline__ void block_rows(u64 I, u64 &lo, u64 &hi) {
    const u64 per = (I + gridDim.x - 1) / gridDim.x;
    lo = min((u64)blockIdx.x * per, I);
    hi = min(lo + per, I);
}

// partials[b][a*R + c] = sum over the rows of block b of Y[i,a] Y[i,c].
// Thread t owns the B x B sub-block at rows (t/16)*B, columns (t%16)*B, B = R/16.
template <int R, bool BF16>
__global__ void __launch_bounds__(kAlsThreads) gram_partial_kernel(const void *Y, u64 I, double *partials) {
    constexpr int B = R / 16;
    __shared__ float rows[kGramRows * R];
    u64 lo, hi;
    block_rows(I, lo, hi);
    const int a0 = (threadIdx.x / 16) * B, c0 = (threadIdx.x % 16) * B;
    double acc[B][B];
#pragma unroll
    for (int x = 0; x < B; ++x)
#pragma unroll
        for (int y = 0; y < B; ++y) acc[x][y] = 0.0;
    for (u64 r0 = lo; r0 < hi; r0 += kGramRows) {
        const int nr = (int)min((u64)kGramRows, hi - r0);
        __syncthreads();
        for (int e = threadIdx.x; e < nr * R; e += kAlsThreads) rows[e] = load_factor<BF16>(Y, r0 * R + e);
        __syncthreads();
        float s[B][B];
#pragma unroll
        for (int x = 0; x < B; ++x)
#pragma unroll
            for (int y = 0; y < B; ++y) s[x][y] = 0.f;
        for (int i = 0; i < nr; ++i) {
            float va[B], vc[B];
#pragma unroll
            for (int x = 0; x < B; ++x) {
                va[x] = rows[i * R + a0 + x];
                vc[x] = rows[i * R + c0 + x];
            }
#pragma unroll
            for (int x = 0; x < B; ++x)
#pragma unroll
                for (int y = 0; y < B; ++y) s[x][y] = fmaf(va[x], vc[y], s[x][y]);
        }
#pragma unroll
        for (int x = 0; x < B; ++x)
#pragma unroll
            for (int y = 0; y < B; ++y) acc[x][y] += (double)s[x][y];
    }
    double *o = partials + (size_t)blockIdx.x * R * R;
#pragma unroll
    for (int x = 0; x < B; ++x)
#pragma unroll
        for (int y = 0; y < B; ++y) o[(a0 + x) * R + c0 + y] = acc[x][y];
}

// out[e] = sum_b partials[b][e], blocks in order
__global__ void sum_partials_kernel(const double *partials, int nblocks, int len, double *out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * len + e];
        out[e] = s;
    }
}

// V = hadamard_{w != n} G_w; V = L L^T (lower triangle of V overwritten by L);
// W = V^{-1} by one forward and one backward substitution per column of I.
// One block, 2 R^2 doubles of dynamic shared memory.  *status = 1 when a pivot
// is not positive.
__global__ void __launch_bounds__(kAlsThreads)
    chol_inverse_kernel(const double *G, int N, int n, int R, float *W, u32 *status) {
    extern __shared__ double chol_smem[];
    double *V = chol_smem, *Z = chol_smem + R * R;
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
            else V[k * R + k] = sqrt(d);
        }
        __syncthreads();
        if (bad) break;
        const double lkk = V[k * R + k];
        for (int i = k + 1 + threadIdx.x; i < R; i += blockDim.x) V[i * R + k] /= lkk;
        __syncthreads();
        // trailing update of the lower triangle: V[i][j] -= L[i][k] L[j][k], k < j <= i
        for (int e = threadIdx.x; e < RR; e += blockDim.x) {
            const int i = e / R, j = e % R;
            if (j > k && i >= j) V[i * R + j] -= V[i * R + k] * V[j * R + k];
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) *status = 1u;
        return;
    }
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        for (int i = 0; i < R; ++i) { // L z = e_c
            double s = (i == c) ? 1.0 : 0.0;
            for (int q = 0; q < i; ++q) s -= V[i * R + q] * Z[q * R + c];
            Z[i * R + c] = s / V[i * R + i];
        }
        for (int i = R - 1; i >= 0; --i) { // L^T w = z
            double s = Z[i * R + c];
            for (int q = i + 1; q < R; ++q) s -= V[q * R + i] * Z[q * R + c];
            Z[i * R + c] = s / V[i * R + i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < RR; e += blockDim.x) W[e] = (float)Z[e];
}

// Y = M W in FP32; thread t computes column c = t % R of rows lo + t/R, stepping
// by 256/R, with column c of W in registers.  Per-block column sums of squares.
template <int R>
__global__ void __launch_bounds__(kAlsThreads)
    als_apply_kernel(const float *M, const float *W, float *Y, u64 I, double *colsq, const u32 *status) {
    __shared__ double part[kAlsThreads];
    if (*status) return;
    constexpr int rstep = kAlsThreads / R;
    const int c = threadIdx.x % R, rsub = threadIdx.x / R;
    float w[R];
#pragma unroll
    for (int a = 0; a < R; ++a) w[a] = W[a * R + c];
    u64 lo, hi;
    block_rows(I, lo, hi);
    double sq = 0.0;
    for (u64 i = lo + rsub; i < hi; i += rstep) {
        const float4 *m = reinterpret_cast<const float4 *>(M + i * R);
        float y = 0.f;
#pragma unroll
        for (int a4 = 0; a4 < R / 4; ++a4) {
            const float4 v = m[a4];
            y = fmaf(v.x, w[4 * a4 + 0], y);
            y = fmaf(v.y, w[4 * a4 + 1], y);
            y = fmaf(v.z, w[4 * a4 + 2], y);
            y = fmaf(v.w, w[4 * a4 + 3], y);
        }
        Y[i * R + c] = y;
        sq += (double)y * (double)y;
    }
    part[threadIdx.x] = sq;
    __syncthreads();
    if (threadIdx.x < R) {
        double s = 0.0;
        for (int q = 0; q < rstep; ++q) s += part[q * R + threadIdx.x];
        colsq[(size_t)blockIdx.x * R + threadIdx.x] = s;
    }
}

__global__ void norms_kernel(const double *colsq, int nblocks, int R, double *lambda, const u32 *status) {
    const int r = threadIdx.x;
    if (r >= R || *status) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += colsq[(size_t)b * R + r];
    lambda[r] = sqrt(s);
}

// factor = Y / lambda (FP64 divide, rounded to FP32, then to BF16 when stored
// so); with M set, also the per-block partials of sum_i M[i,r] factor[i,r]
template <bool BF16>
__global__ void __launch_bounds__(kAlsThreads)
    normalize_store_kernel(const float *Yt, const double *lambda, void *Yout, u64 I, int R, const float *M,
                           double *inner, const u32 *status) {
    __shared__ double part[kAlsThreads];
    if (*status) return;
    const int rstep = kAlsThreads / R;
    const int c = threadIdx.x % R, rsub = threadIdx.x / R;
    const double lam = lambda[c];
    const double div = lam > 0.0 ? lam : 1.0;
    u64 lo, hi;
    block_rows(I, lo, hi);
    double s = 0.0;
    for (u64 i = lo + rsub; i < hi; i += rstep) {
        float stored = (float)((double)Yt[i * R + c] / div);
        if constexpr (BF16) {
            const __nv_bfloat16 b = __float2bfloat16_rn(stored);
            static_cast<__nv_bfloat16 *>(Yout)[i * R + c] = b;
            stored = __bfloat162float(b);
        } else {
            static_cast<float *>(Yout)[i * R + c] = stored;
        }
        if (M) s += (double)M[i * R + c] * (double)stored;
    }
    if (inner) {
        part[threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.x < R) {
            double t = 0.0;
            for (int q = 0; q < rstep; ++q) t += part[q * R + threadIdx.x];
            inner[(size_t)blockIdx.x * R + threadIdx.x] = t;
        }
    }
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
    __syncthreads();
    if (threadIdx.x == 0) {
        double sxh = 0.0, sxi = 0.0;
        for (int q = 0; q < kAlsThreads; ++q) {
            sxh += part[0][q];
            sxi += part[1][q];
        }
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
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kAlsThreads; ++q) t += part[q];
        partials[blockIdx.x] = t;
    }
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
    sum_partials_kernel<<<(R * R + 255) / 256, 256, 0, s>>>(gpart, nblk, R * R, G);
    FLY_TRY_CUDA(cudaGetLastError());
    return FLYCOO_OK;
}

void launch_apply(int R, const float *M, const float *W, float *Y, u64 I, double *colsq, const u32 *status,
                  int nblk, cudaStream_t s) {
    switch (R) {
    case 16: als_apply_kernel<16><<<nblk, kAlsThreads, 0, s>>>(M, W, Y, I, colsq, status); break;
    case 32: als_apply_kernel<32><<<nblk, kAlsThreads, 0, s>>>(M, W, Y, I, colsq, status); break;
    default: als_apply_kernel<64><<<nblk, kAlsThreads, 0, s>>>(M, W, Y, I, colsq, status); break;
    }
}

} // namespace

flycoo_status als_step(Tensor &t, void *const *F, flycoo_dtype fdt, int R, double *d_lambda, double *h_fit,
                       cudaStream_t s) {
    const int N = t.N;
    const bool bf = fdt == FLYCOO_BF16;
    AlsWork &w = t.als;
    u64 maxI = 0;
    for (int n = 0; n < N; ++n) maxI = std::max<u64>(maxI, t.dims[n]);
    const int nblk = 2 * t.sm_count;
    if (w.rows < maxI || w.nblk != nblk) {
        FLY_TRY_CUDA(cudaFuncSetAttribute(chol_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          2 * kMaxRank * kMaxRank * (int)sizeof(double)));
        FLY_TRY(w.M.alloc(maxI * kMaxRank * sizeof(float)));
        FLY_TRY(w.Y.alloc(maxI * kMaxRank * sizeof(float)));
        FLY_TRY(w.G.alloc((size_t)FLYCOO_MAX_MODES * kMaxRank * kMaxRank * sizeof(double)));
        FLY_TRY(w.gpart.alloc((size_t)nblk * kMaxRank * kMaxRank * sizeof(double)));
        FLY_TRY(w.W.alloc(kMaxRank * kMaxRank * sizeof(float)));
        FLY_TRY(w.colsq.alloc((size_t)nblk * kMaxRank * sizeof(double)));
        FLY_TRY(w.inner.alloc((size_t)nblk * kMaxRank * sizeof(double)));
        FLY_TRY(w.scal.alloc((size_t)(nblk + 4) * sizeof(double)));
        w.rows = maxI;
        w.nblk = nblk;
        w.normx2_valid = false;
    }
    double *G = w.G.as<double>();
    double *scal = w.scal.as<double>(); // [0] ||X||^2, [1] fit, [2] status word, [4..] partials
    u32 *status = reinterpret_cast<u32 *>(scal + 2);
    // the sweep starts in L_0; ||X||^2 is summed in that order, so the result
    // does not depend on the layout the tensor was left in
    while (t.layout != 0) {
        FLY_TRY(launch_remap_step(t, t.layout, t.elem[t.cur].p, t.elem[1 - t.cur].p, s));
        t.cur = 1 - t.cur;
        t.layout = (t.layout + 1) % N;
    }
    if (!w.normx2_valid) {
        if (t.nnz) {
            value_sq_kernel<<<nblk, kAlsThreads, 0, s>>>(t.elem[t.cur].as<u32>(), t.elem_words, N, t.nnz, scal + 4);
            sum_partials_kernel<<<1, 32, 0, s>>>(scal + 4, nblk, 1, scal);
            FLY_TRY_CUDA(cudaGetLastError());
        } else {
            FLY_TRY_CUDA(cudaMemsetAsync(scal, 0, sizeof(double), s));
        }
        FLY_TRY_CUDA(cudaMemcpyAsync(&w.normx2, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        FLY_TRY_CUDA(cudaStreamSynchronize(s));
        w.normx2_valid = true;
    }
    if (!(w.normx2 > 0.0)) {
        set_error("flycoo_cp_als_step: the tensor has no nonzero value (||X|| = 0, fit undefined)");
        return FLYCOO_ERR_INVALID_ARG;
    }
    const size_t RR = (size_t)R * R;
    for (int n = 0; n < N; ++n) FLY_TRY(gram(F[n], bf, t.dims[n], R, G + n * RR, w.gpart.as<double>(), nblk, s));
    FLY_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(u32), s));
    for (int n = 0; n < N; ++n) {
        const u64 I = t.dims[n];
        FLY_TRY(run_pass(t, n, F, fdt, R, w.M.as<float>(), nullptr, nullptr, s));
        chol_inverse_kernel<<<1, kAlsThreads, 2 * RR * sizeof(double), s>>>(G, N, n, R, w.W.as<float>(), status);
        launch_apply(R, w.M.as<float>(), w.W.as<float>(), w.Y.as<float>(), I, w.colsq.as<double>(), status, nblk,
                     s);
        norms_kernel<<<1, kMaxRank, 0, s>>>(w.colsq.as<double>(), nblk, R, d_lambda, status);
        const bool last = n == N - 1;
        float *Mlast = last ? w.M.as<float>() : nullptr;
        double *inner = last ? w.inner.as<double>() : nullptr;
        if (bf)
            normalize_store_kernel<true><<<nblk, kAlsThreads, 0, s>>>(w.Y.as<float>(), d_lambda, F[n], I, R, Mlast,
                                                                     inner, status);
        else
            normalize_store_kernel<false><<<nblk, kAlsThreads, 0, s>>>(w.Y.as<float>(), d_lambda, F[n], I, R, Mlast,
                                                                      inner, status);
        FLY_TRY_CUDA(cudaGetLastError());
        FLY_TRY(gram(F[n], bf, I, R, G + n * RR, w.gpart.as<double>(), nblk, s));
    }
    fit_kernel<<<1, kAlsThreads, 0, s>>>(G, N, R, d_lambda, w.inner.as<double>(), nblk, scal, scal + 1);
    FLY_TRY_CUDA(cudaGetLastError());
    double res[3];
    FLY_TRY_CUDA(cudaMemcpyAsync(res, scal, sizeof(res), cudaMemcpyDeviceToHost, s));
    FLY_TRY_CUDA(cudaStreamSynchronize(s));
    u32 st;
    memcpy(&st, &res[2], sizeof(st));
    if (st) {
        set_error("flycoo_cp_als_step: a normal-equation matrix (hadamard of Gram matrices) is not positive "
                  "definite; the modes before it were updated, the others are unchanged");
        return FLYCOO_ERR_NOT_SPD;
    }
    if (h_fit) *h_fit = res[1];
    return FLYCOO_OK;
}

} // namespace flycoo
