// grad.cu -- the gradient of spMTTKRP with respect to the nonzero values.
//
// The elementwise update of Section IV (Eq. 4) adds val(x) * prod_{w != n}
// Y_w[c_w(x), :] to row c_n(x) of M_n, so M_n is linear in every value, and
// for an upstream gradient G = d loss / d M_n
//   d loss / d val(x) = sum_r G[c_n(x), r] prod_{w != n} Y_w[c_w(x), r],
// the CP model value of x (Eq. 1) with Y_n replaced by G.  The kernel below
// computes it for every nonzero of layout L_0 and writes it at the nonzero's
// position in the caller's COO input.
#include "internal.cuh"

namespace flycoo {
namespace {

struct FactorPtrs {
    const void *p[FLYCOO_MAX_MODES];
};

template <bool BF16>
__device__ __forceinline__ void widen_chunk(const uint4 &v, float *f) {
    if constexpr (BF16) {
        const u32 w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            f[2 * q] = __uint_as_float(w[q] << 16);
            f[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
        }
    } else {
        f[0] = __uint_as_float(v.x);
        f[1] = __uint_as_float(v.y);
        f[2] = __uint_as_float(v.z);
        f[3] = __uint_as_float(v.w);
    }
}

// Groups of L = R / CV lanes, one nonzero per group: lane k loads the k-th 16
// bytes of each of the N rows (F[w] row c_w for every mode w, G in place of the
// output mode's factor), multiplies them elementwise in FP32 and sums its CV
// products; the group's partial sums are added by a fixed xor-shuffle tree.
// In L_0 word w of a stored nonzero is c_w.  dvals[orig[p]] receives the
// result of position p.
template <int R, bool BF16>
__global__ void __launch_bounds__(256) value_grad_kernel(const u32 *__restrict__ elem, int ew, int N, u64 nnz,
                                                         const u32 *__restrict__ orig, const FactorPtrs F,
                                                         float *__restrict__ dvals) {
    constexpr int CV = BF16 ? 8 : 4;
    constexpr int L = R / CV;
    constexpr int GPW = 32 / L;
    static_assert(L >= 1 && L <= 32 && 32 % L == 0, "rank not supported");
    const int lane = threadIdx.x & 31;
    const int k = lane % L;
    const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 base = warp * GPW; base < nnz; base += nwarps * GPW) {
        const u64 p = base + lane / L;
        const bool valid = p < nnz;
        float prod[CV];
#pragma unroll
        for (int v = 0; v < CV; ++v) prod[v] = 1.f;
        if (valid) {
            const u32 *e = elem + p * (u64)ew;
            for (int w = 0; w < N; ++w) {
                const uint4 *row = static_cast<const uint4 *>(F.p[w]) + (u64)e[w] * (R / CV);
                float f[CV];
                widen_chunk<BF16>(__ldg(row + k), f);
#pragma unroll
                for (int v = 0; v < CV; ++v) prod[v] *= f[v];
            }
        }
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < CV; ++v) s += prod[v];
#pragma unroll
        for (int off = L / 2; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (valid && k == 0) dvals[orig[p]] = s;
    }
}

template <int R>
void launch_vg(bool bf, const Tensor &t, const FactorPtrs &F, float *d_gvals, cudaStream_t s) {
    const unsigned grid = (unsigned)(4 * t.sm_count);
    if (bf)
        value_grad_kernel<R, true><<<grid, 256, 0, s>>>(t.elem[t.cur].as<u32>(), t.elem_words, t.N, t.nnz,
                                                       t.orig.as<u32>(), F, d_gvals);
    else
        value_grad_kernel<R, false><<<grid, 256, 0, s>>>(t.elem[t.cur].as<u32>(), t.elem_words, t.N, t.nnz,
                                                        t.orig.as<u32>(), F, d_gvals);
}

} // namespace

flycoo_status launch_value_grad(const Tensor &t, int mode, const void *const *Y, const void *G, flycoo_dtype fdt,
                                int R, float *d_gvals, cudaStream_t s) {
    if (t.layout != 0) {
        set_error("internal: the value gradient runs in layout L_0 (the tensor is in L_%d)", t.layout);
        return FLYCOO_ERR_LAYOUT;
    }
    if (t.nnz == 0) return FLYCOO_OK;
    FactorPtrs F{};
    for (int w = 0; w < t.N; ++w) F.p[w] = (w == mode) ? G : Y[w];
    const bool bf = fdt == FLYCOO_BF16;
    switch (R) {
    case 16: launch_vg<16>(bf, t, F, d_gvals, s); break;
    case 32: launch_vg<32>(bf, t, F, d_gvals, s); break;
    case 64: launch_vg<64>(bf, t, F, d_gvals, s); break;
    default:
        set_error("rank %d not built (16, 32 or 64)", R);
        return FLYCOO_ERR_UNSUPPORTED;
    }
    FLY_TRY_CUDA(cudaGetLastError());
    return FLYCOO_OK;
}

} // namespace flycoo
