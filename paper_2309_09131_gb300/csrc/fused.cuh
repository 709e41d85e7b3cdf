// fused.cuh -- K2: spMTTKRP of one mode with the dynamic remap fused into the
// same pass (Algorithm 2, one value of n), and K4: the fixed-order sum of the
// partial rows that straddle shard boundaries.
//
// Work decomposition.  The tensor is in layout L_n: nonzeros ordered by the
// output index c_n, in shards of at most g consecutive nonzeros (Section
// III-A).  Thread block b walks the shards that Algorithm 3 put in bin b.
// Inside a shard, each group of L lanes owns one contiguous slice of the
// shard; its lanes split the rank dimension (16 bytes of every factor row per
// lane, so a row gather is one coalesced vector load per lane).  A group
// streams its slice in batches: the L lanes load the batch's nonzeros (and
// their slots in L_{n+1}), store each nonzero at its slot of the next layout
// (the fused remap), and stage the batch in shared memory.  Every lane then
// reads each staged nonzero, gathers the N-1 input factor rows, forms
// val * (Hadamard product) in FP32 and adds it to a running row sum held in
// registers.  Rows are contiguous in L_n, so a row sum is complete when the
// output index changes, unless the row touches the start or end of the slice.
//
// Ownership and determinism (no atomics).  A row strictly inside one slice is
// stored by that slice's group.  The first and last row of each slice are
// combined with the neighbouring slices in slice order after a block barrier;
// a row strictly inside the shard is then stored by the group whose slice it
// starts in.  The first and last row of each shard go to a per-shard partial
// buffer, and K4 sums those partials in shard order.  Each output row is
// written exactly once, by exactly one thread group, and the summation order
// depends only on the layout and the launch shape.  Rows that no nonzero
// touches are written as zeros by whoever owns the gap before them.
#pragma once

#include "internal.cuh"

namespace flycoo {

template <int N, int R, bool BF16>
struct FusedCfg {
    static constexpr int VEC = BF16 ? 8 : 4;       // factor values per 16-byte load
    static constexpr int L = R / VEC;              // lanes per group
    static constexpr int GPW = 32 / L;             // groups per warp
    static constexpr int WARPS = 8;
    static constexpr int THREADS = WARPS * 32;
    static constexpr int G = WARPS * GPW;          // groups per block
    static constexpr int EW = (N + 1 <= 4) ? 4 : 8; // 32-bit words per stored nonzero
    static constexpr int EQ = EW / 4;              // 16-byte chunks per stored nonzero
    static constexpr int BATCH = 8;                // nonzeros staged per group and batch
    static constexpr int SUB = (N <= 3) ? 4 : 2;   // nonzeros whose gathers are in flight together
    static constexpr size_t SMEM = (size_t)G * BATCH * EQ * 16 + 2 * (size_t)G * R * 4 + 3 * (size_t)G * 4;
    static_assert(R % VEC == 0 && L >= 1 && L <= 32 && 32 % L == 0, "rank not supported");
};

template <bool BF16>
__device__ __forceinline__ void widen(const uint4 &v, float *f) {
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

template <int VEC>
__device__ __forceinline__ void store_vec(float *dst, const float *v) {
#pragma unroll
    for (int q = 0; q < VEC / 4; ++q)
        reinterpret_cast<float4 *>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

template <int VEC>
__device__ __forceinline__ void load_vec(const float *src, float *v) {
#pragma unroll
    for (int q = 0; q < VEC / 4; ++q) {
        const float4 x = reinterpret_cast<const float4 *>(src)[q];
        v[4 * q] = x.x;
        v[4 * q + 1] = x.y;
        v[4 * q + 2] = x.z;
        v[4 * q + 3] = x.w;
    }
}

template <int VEC>
__device__ __forceinline__ void store_zero(float *dst) {
#pragma unroll
    for (int q = 0; q < VEC / 4; ++q) reinterpret_cast<float4 *>(dst)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int N, int R, bool BF16>
__global__ void __launch_bounds__(256) fused_mttkrp_remap_kernel(const FusedArgs a) {
    using C = FusedCfg<N, R, BF16>;
    constexpr int VEC = C::VEC;
    constexpr int RV = R / VEC; // 16-byte chunks per factor row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint4 *stage = reinterpret_cast<uint4 *>(smem_raw);
    float *hacc = reinterpret_cast<float *>(stage + C::G * C::BATCH * C::EQ);
    float *tacc = hacc + C::G * R;
    u32 *hrow = reinterpret_cast<u32 *>(tacc + C::G * R);
    u32 *trow = hrow + C::G;
    u32 *multi = trow + C::G;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int k = lane % C::L;
    const int grp = warp * C::GPW + lane / C::L;
    const bool remap = a.elem_out != nullptr;
    const uint4 *__restrict__ ein = static_cast<const uint4 *>(a.elem_in);
    uint4 *__restrict__ eout = static_cast<uint4 *>(a.elem_out);
    const u32 *__restrict__ next = a.next;
    float *__restrict__ out = a.out;
    const uint4 *Yp[N - 1];
#pragma unroll
    for (int t = 0; t < N - 1; ++t) Yp[t] = static_cast<const uint4 *>(a.Y[t]) + k;
    uint4 *my_stage = stage + grp * C::BATCH * C::EQ;
    float *my_hacc = hacc + grp * R + k * VEC;
    float *my_tacc = tacc + grp * R + k * VEC;

    const u32 it_end = a.bin_ptr[blockIdx.x + 1];
    for (u32 it = a.bin_ptr[blockIdx.x]; it < it_end; ++it) {
        const u32 s = a.bin_items[it];
        const u32 start = a.shard_ptr[s];
        const u32 len = a.shard_ptr[s + 1] - start;
        const u32 chunk = (len + C::G - 1) / C::G;
        const u32 geff = (len + chunk - 1) / chunk;
        const u32 lo = start + min((u32)grp * chunk, len);
        const u32 hi = start + min((u32)(grp + 1) * chunk, len);
        const u32 first_row = a.first_row[s];
        const u32 last_row = a.last_row[s];

        // empty rows before this shard (and after the last shard)
        {
            const u32 z0 = (s == 0) ? 0u : a.last_row[s - 1] + 1u;
            for (u32 r = z0 + grp; r < first_row; r += C::G) store_zero<VEC>(out + (size_t)r * R + k * VEC);
            if (s + 1 == a.S)
                for (u32 r = last_row + 1u + grp; r < a.I_out; r += C::G)
                    store_zero<VEC>(out + (size_t)r * R + k * VEC);
        }

        float acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
        u32 cur = kInvalidRow;
        bool first = true;

        for (u32 b0 = 0; b0 < chunk; b0 += C::BATCH) {
            // stage the batch; the fused remap stores each nonzero at its next slot
            for (int j = k; j < C::BATCH; j += C::L) {
                const u32 p = lo + b0 + j;
                uint4 e[C::EQ];
                if (p < hi) {
#pragma unroll
                    for (int q = 0; q < C::EQ; ++q) e[q] = __ldcs(ein + (size_t)p * C::EQ + q);
                    if (remap) {
                        const u32 d = __ldcs(next + p);
                        u32 w[C::EW], r[C::EW];
#pragma unroll
                        for (int q = 0; q < C::EQ; ++q) {
                            w[4 * q] = e[q].x;
                            w[4 * q + 1] = e[q].y;
                            w[4 * q + 2] = e[q].z;
                            w[4 * q + 3] = e[q].w;
                        }
#pragma unroll
                        for (int t = 0; t < C::EW; ++t) r[t] = (t < N) ? w[(t + 1) % N] : w[t];
#pragma unroll
                        for (int q = 0; q < C::EQ; ++q)
                            eout[(size_t)d * C::EQ + q] = make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < C::EQ; ++q) e[q] = make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int q = 0; q < C::EQ; ++q) my_stage[j * C::EQ + q] = e[q];
            }
            __syncwarp();
#pragma unroll
            for (int j0 = 0; j0 < C::BATCH; j0 += C::SUB) {
                uint4 raw[C::SUB][N - 1];
                u32 row[C::SUB];
                float val[C::SUB];
#pragma unroll
                for (int j = 0; j < C::SUB; ++j) {
                    u32 w[C::EW];
#pragma unroll
                    for (int q = 0; q < C::EQ; ++q) {
                        const uint4 x = my_stage[(j0 + j) * C::EQ + q];
                        w[4 * q] = x.x;
                        w[4 * q + 1] = x.y;
                        w[4 * q + 2] = x.z;
                        w[4 * q + 3] = x.w;
                    }
                    row[j] = w[0];
                    val[j] = __uint_as_float(w[N]);
#pragma unroll
                    for (int t = 1; t < N; ++t) raw[j][t - 1] = __ldg(Yp[t - 1] + (size_t)w[t] * RV);
                }
#pragma unroll
                for (int j = 0; j < C::SUB; ++j) {
                    if (lo + b0 + j0 + j < hi) {
                        float prod[VEC];
                        widen<BF16>(raw[j][0], prod);
#pragma unroll
                        for (int t = 1; t < N - 1; ++t) {
                            float f[VEC];
                            widen<BF16>(raw[j][t], f);
#pragma unroll
                            for (int v = 0; v < VEC; ++v) prod[v] *= f[v];
                        }
                        if (row[j] != cur) {
                            if (cur != kInvalidRow) {
                                if (first) {
                                    store_vec<VEC>(my_hacc, acc);
                                    if (k == 0) hrow[grp] = cur;
                                    first = false;
                                } else {
                                    store_vec<VEC>(out + (size_t)cur * R + k * VEC, acc);
                                }
                                for (u32 r = cur + 1u; r < row[j]; ++r)
                                    store_zero<VEC>(out + (size_t)r * R + k * VEC);
                            }
                            cur = row[j];
#pragma unroll
                            for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
                        }
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[v] = fmaf(val[j], prod[v], acc[v]);
                    }
                }
            }
            __syncwarp();
        }

        // slice summary: a single run goes to the head slot, else the last run to the tail slot
        if ((u32)grp < geff) {
            if (first) {
                store_vec<VEC>(my_hacc, acc);
                if (k == 0) {
                    hrow[grp] = cur;
                    multi[grp] = 0u;
                }
            } else {
                store_vec<VEC>(my_tacc, acc);
                if (k == 0) {
                    trow[grp] = cur;
                    multi[grp] = 1u;
                }
            }
        }
        __syncthreads();

        if ((u32)grp < geff) {
            const u32 h = hrow[grp];
            const bool mg = multi[grp] != 0u;
            const u32 prev_last = (grp == 0) ? kInvalidRow : (multi[grp - 1] ? trow[grp - 1] : hrow[grp - 1]);
            // sum a run that starts in this slice over the following slices, in order;
            // returns true if it reaches the end of the shard
            auto extend = [&](u32 r, float *sum) -> bool {
                for (u32 q = grp + 1; q < geff; ++q) {
                    if (hrow[q] != r) return false;
                    float x[VEC];
                    load_vec<VEC>(hacc + q * R + k * VEC, x);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) sum[v] += x[v];
                    if (multi[q]) return false;
                }
                return true;
            };
            auto emit = [&](u32 r, const float *sum, bool is_start, bool reach_end) {
                if (is_start) store_vec<VEC>(a.p_head + (size_t)s * R + k * VEC, sum);
                else if (reach_end) store_vec<VEC>(a.p_tail + (size_t)s * R + k * VEC, sum);
                else store_vec<VEC>(out + (size_t)r * R + k * VEC, sum);
            };
            if (grp == 0 || prev_last != h) {
                float sum[VEC];
                load_vec<VEC>(my_hacc, sum);
                const bool reach_end = mg ? false : extend(h, sum);
                emit(h, sum, grp == 0, reach_end);
            }
            if (mg) {
                const u32 tr = trow[grp];
                float sum[VEC];
                load_vec<VEC>(my_tacc, sum);
                const bool reach_end = extend(tr, sum);
                emit(tr, sum, false, reach_end);
            }
            if (grp > 0)
                for (u32 r = prev_last + 1u; r < h; ++r) store_zero<VEC>(out + (size_t)r * R + k * VEC);
        }
        __syncthreads();
    }
}

// K4: one warp per boundary row; sums the shard partials in shard order.
template <int R>
__global__ void __launch_bounds__(256) boundary_fixup_kernel(const FixupArgs a) {
    constexpr int PER = (R + 31) / 32;
    const u32 w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= a.nb) return;
    const u32 row = a.bnd[3 * (size_t)w];
    const u32 s_lo = a.bnd[3 * (size_t)w + 1];
    const u32 s_hi = a.bnd[3 * (size_t)w + 2];
    const float *first = (a.first_row[s_lo] == row) ? a.p_head : a.p_tail;
    float sum[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int r = lane + 32 * i;
        sum[i] = (r < R) ? first[(size_t)s_lo * R + r] : 0.f;
    }
#pragma unroll 4
    for (u32 s = s_lo + 1; s <= s_hi; ++s) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int r = lane + 32 * i;
            if (r < R) sum[i] += a.p_head[(size_t)s * R + r];
        }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int r = lane + 32 * i;
        if (r < R) a.out[(size_t)row * R + r] = sum[i];
    }
}

template <int N, int R, bool BF16>
flycoo_status launch_fused_t(const FusedArgs &a, cudaStream_t s) {
    using C = FusedCfg<N, R, BF16>;
    auto kern = fused_mttkrp_remap_kernel<N, R, BF16>;
    if (C::SMEM > 48 * 1024)
        FLY_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    kern<<<a.bins, C::THREADS, C::SMEM, s>>>(a);
    FLY_TRY_CUDA(cudaGetLastError());
    return FLYCOO_OK;
}

template <int N>
flycoo_status launch_fused_dispatch(int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s) {
    const bool bf = dt == FLYCOO_BF16;
    switch (R) {
    case 16: return bf ? launch_fused_t<N, 16, true>(a, s) : launch_fused_t<N, 16, false>(a, s);
    case 32: return bf ? launch_fused_t<N, 32, true>(a, s) : launch_fused_t<N, 32, false>(a, s);
    case 64: return bf ? launch_fused_t<N, 64, true>(a, s) : launch_fused_t<N, 64, false>(a, s);
    default: break;
    }
    set_error("rank %d not built (16, 32 or 64)", R);
    return FLYCOO_ERR_UNSUPPORTED;
}

} // namespace flycoo
