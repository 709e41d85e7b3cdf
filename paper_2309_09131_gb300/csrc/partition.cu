// partition.cu -- K1: FLYCOO preprocessing on the GPU (Section III-A; the
// preprocessing stages of Section V-J) plus the standalone remap step.
//
// The layout L_n orders the nonzeros by their super-shard ids
// (ss_n, ss_{n-1}, ..., ss_{n+1}, input position), ss_w = c_w div m_w.  Under
// this cyclic key, L_{n+1} is exactly L_n stably sorted by ss_{n+1} alone, and
// L_0 is the input order stably sorted by ss_1, ss_2, ..., ss_{N-1} and
// finally ss_0.  K1 therefore runs 2N-1 stable sorts, each a few 8-bit LSD
// radix passes (histogram, exclusive scan, stable scatter).  The tensor is
// stored in exactly this order.  Separately, for every stage tile of both
// sizes, K1 records the tile's compute order: the permutation that sorts the
// tile stably by output index, so the fused kernel finds each row of a tile
// contiguous without moving the stored nonzeros.  Every step is integer work
// with no atomics on the data path, so the layouts, pointers, remap
// permutations and compute orders are bit-exact and deterministic.  There is
// no spin-wait anywhere: the scan is a plain reduce-then-scan.
#include "internal.cuh"

#include <algorithm>

namespace flycoo {

// ===========================================================================
// exclusive scan of uint32 (reduce -> scan block sums -> downsweep)
// ===========================================================================
namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ u32 block_exclusive_scan(u32 v, u32 *warp_sums, u32 *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        u32 y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        u32 w = (lane < kScanThreads / 32) ? warp_sums[lane] : 0u;
        u32 z = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            u32 y = __shfl_up_sync(0xffffffffu, z, d);
            if (lane >= d) z += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = z - w;
        if (lane == kScanThreads / 32 - 1) *total = z;
    }
    __syncthreads();
    return x - v + warp_sums[warp];
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const u32 *in, u64 n, u32 *sums) {
    __shared__ u32 ws[kScanThreads / 32];
    __shared__ u32 tot;
    const u64 base = (u64)blockIdx.x * kScanTile + (u64)threadIdx.x * kScanItems;
    u32 s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    block_exclusive_scan(s, ws, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single block, loops over the block sums in tiles, carrying the running total
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(u32 *sums, u64 nb) {
    __shared__ u32 ws[kScanThreads / 32];
    __shared__ u32 tot;
    u32 carry = 0;
    for (u64 t0 = 0; t0 < nb; t0 += kScanTile) {
        const u64 base = t0 + (u64)threadIdx.x * kScanItems;
        u32 v[kScanItems];
        u32 s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = (base + i < nb) ? sums[base + i] : 0u;
            s += v[i];
        }
        u32 off = block_exclusive_scan(s, ws, &tot) + carry;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (base + i < nb) sums[base + i] = off;
            off += v[i];
        }
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads)
    scan_down_kernel(const u32 *in, u32 *out, u64 n, const u32 *offs) {
    __shared__ u32 ws[kScanThreads / 32];
    __shared__ u32 tot;
    const u64 base = (u64)blockIdx.x * kScanTile + (u64)threadIdx.x * kScanItems;
    u32 v[kScanItems];
    u32 s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    u32 off = block_exclusive_scan(s, ws, &tot) + offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = off;
        off += v[i];
    }
}
} // namespace

u64 scan_scratch_words(u64 n) { return (n + kScanTile - 1) / kScanTile + 1; }

flycoo_status exclusive_scan_u32(const u32 *in, u32 *out, u64 n, u32 *scratch, cudaStream_t s) {
    if (n == 0) return FLYCOO_OK;
    const u64 nb = (n + kScanTile - 1) / kScanTile;
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, scratch);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(scratch, nb);
    scan_down_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, scratch);
    FLY_TRY_CUDA(cudaGetLastError());
    return FLYCOO_OK;
}

// ===========================================================================
// stable LSD radix sort of (key, value) uint32 pairs, 8 bits per pass
// ===========================================================================
namespace {
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;                          // 32-element rounds per warp
constexpr int kRsTile = kRsThreads * kRsRounds;        // 4096 elements per block

__global__ void __launch_bounds__(kRsThreads)
    rs_hist_kernel(const u32 *keys, u64 n, int shift, u32 *counts, u64 ntiles) {
    __shared__ u32 h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const u64 base = (u64)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        const u64 p = base + i;
        if (p < n) atomicAdd(&h[(keys[p] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(u64)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: ranks follow input order (warp order, then round, then lane).
__global__ void __launch_bounds__(kRsThreads)
    rs_scatter_kernel(const u32 *keys, const u32 *vals, u64 n, int shift, const u32 *offs,
                      u64 ntiles, u32 *keys_out, u32 *vals_out) {
    __shared__ u32 cnt[kRsWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u64 base = (u64)blockIdx.x * kRsTile + (u64)warp * (32 * kRsRounds);
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    u32 k[kRsRounds], v[kRsRounds];
#pragma unroll
    for (int t = 0; t < kRsRounds; ++t) {
        const u64 p = base + (u64)t * 32 + lane;
        k[t] = (p < n) ? keys[p] : 0u;
        v[t] = (p < n) ? vals[p] : 0u;
    }
    const unsigned lt_mask = (1u << lane) - 1u;
    // pass 1: per-warp digit counts
#pragma unroll
    for (int t = 0; t < kRsRounds; ++t) {
        const u64 p = base + (u64)t * 32 + lane;
        const bool valid = p < n;
        const u32 d = valid ? ((k[t] >> shift) & 255u) : (256u + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lt_mask) == 0) cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: global offset of this tile, then the warps in order
    {
        const int d = threadIdx.x; // kRsThreads == 256 digits
        u32 run = offs[(u64)d * ntiles + blockIdx.x];
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            const u32 c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    // pass 2: rank and scatter
#pragma unroll
    for (int t = 0; t < kRsRounds; ++t) {
        const u64 p = base + (u64)t * 32 + lane;
        const bool valid = p < n;
        const u32 d = valid ? ((k[t] >> shift) & 255u) : (256u + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        u32 pos = 0;
        if (valid) pos = cnt[warp][d] + __popc(peers & lt_mask);
        __syncwarp();
        if (valid && (peers & lt_mask) == 0) cnt[warp][d] += __popc(peers);
        __syncwarp();
        if (valid) {
            keys_out[pos] = k[t];
            vals_out[pos] = v[t];
        }
    }
}

// stable sort of (keys, vals) by the low `bits` bits of keys; results end up in
// (*keys, *vals) (the buffers may be swapped with the temporaries)
flycoo_status stable_sort_pairs(u32 **keys, u32 **vals, u32 **ktmp, u32 **vtmp, u32 *counts,
                                u32 *scan_tmp, u64 n, int bits, cudaStream_t s) {
    if (n == 0) return FLYCOO_OK;
    const u64 ntiles = (n + kRsTile - 1) / kRsTile;
    for (int shift = 0; shift < bits; shift += 8) {
        rs_hist_kernel<<<(unsigned)ntiles, kRsThreads, 0, s>>>(*keys, n, shift, counts, ntiles);
        FLY_TRY(exclusive_scan_u32(counts, counts, 256 * ntiles, scan_tmp, s));
        rs_scatter_kernel<<<(unsigned)ntiles, kRsThreads, 0, s>>>(*keys, *vals, n, shift, counts,
                                                                  ntiles, *ktmp, *vtmp);
        FLY_TRY_CUDA(cudaGetLastError());
        std::swap(*keys, *ktmp);
        std::swap(*vals, *vtmp);
    }
    return FLYCOO_OK;
}

// ===========================================================================
// small K1 kernels
// ===========================================================================
struct Dims {
    u32 d[FLYCOO_MAX_MODES];
};

__global__ void check_index_kernel(const u32 *idx, u64 nnz, int N, Dims dims, u32 *err) {
    const u64 total = nnz * (u64)N;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (u64)gridDim.x * blockDim.x) {
        const int w = (int)(i / nnz);
        if (idx[i] >= dims.d[w]) atomicOr(err, 1u);
    }
}

__global__ void iota_kernel(u32 *a, u64 n) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
        a[i] = (u32)i;
}

__global__ void gather_kernel(const u32 *src, const u32 *perm, u32 *dst, u64 n) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

// super-shard id of each element of a permuted order: dst[i] = src[perm[i]] / m
__global__ void gather_div_kernel(const u32 *src, const u32 *perm, u32 *dst, u64 n, u32 m) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]] / m;
}

// Z-Morton code of the other modes' super-shard ids of element perm[i], for
// output mode `mode`: bit levels from the most significant down, modes
// mode+1, ..., mode-1 at each level, the id of mode w taking width[w] bits;
// word 0 = the low 32 bits of the code, word 1 = the high 32 bits
__global__ void morton_key_kernel(const u32 *idx, u64 nnz, int N, int mode, Dims m, Dims width, int maxw,
                                  const u32 *perm, u32 *keys, int word) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (u64)gridDim.x * blockDim.x) {
        const u32 e = perm[i];
        u64 code = 0;
        for (int level = maxw - 1; level >= 0; --level)
            for (int t = 1; t < N; ++t) {
                const int w = (mode + t) % N;
                if (level < (int)width.d[w]) code = (code << 1) | ((idx[(u64)w * nnz + e] / m.d[w] >> level) & 1u);
            }
        keys[i] = word ? (u32)(code >> 32) : (u32)code;
    }
}

__global__ void inverse_kernel(const u32 *perm, u32 *inv, u64 n) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
        inv[perm[i]] = (u32)i;
}

// ptr[r] = first position whose key is >= r (keys sorted ascending), r in [0, I]
__global__ void row_ptr_kernel(const u32 *rows, u64 n, u64 I, u32 *row_ptr) {
    for (u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x; p <= n; p += (u64)gridDim.x * blockDim.x) {
        const int64_t prev = (p == 0) ? -1 : (int64_t)rows[p - 1];
        const int64_t cur = (p == n) ? (int64_t)I : (int64_t)rows[p];
        for (int64_t r = prev + 1; r <= cur; ++r) row_ptr[r] = (u32)p;
    }
}

// element of layout L_0: slot t holds c_t, word N holds the value bits
__global__ void build_elems_kernel(const u32 *idx, const float *vals, const u32 *perm, u64 nnz, int N,
                                   int ew, u32 *elem) {
    for (u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (u64)gridDim.x * blockDim.x) {
        const u32 e = perm[p];
        u32 *o = elem + p * (u64)ew;
        for (int t = 0; t < ew; ++t) {
            u32 w = 0;
            if (t < N) w = idx[(u64)t * nnz + e];
            else if (t == N) w = __float_as_uint(vals[e]);
            o[t] = w;
        }
    }
}

template <int EW>
__global__ void remap_step_kernel(const uint4 *__restrict__ in, uint4 *__restrict__ out,
                                  const u32 *__restrict__ next, u64 nnz, int N) {
    for (u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (u64)gridDim.x * blockDim.x) {
        u32 w[EW];
#pragma unroll
        for (int q = 0; q < EW / 4; ++q) {
            const uint4 v = __ldcs(in + p * (EW / 4) + q);
            w[4 * q + 0] = v.x;
            w[4 * q + 1] = v.y;
            w[4 * q + 2] = v.z;
            w[4 * q + 3] = v.w;
        }
        u32 r[EW];
#pragma unroll
        for (int t = 0; t < EW; ++t) r[t] = w[t];
        // rotate the coordinate slots by one: slot t of L_{n+1} is slot t+1 of L_n
        for (int t = 0; t < N; ++t) r[t] = w[(t + 1) % N];
        const u64 d = __ldcs(next + p);
#pragma unroll
        for (int q = 0; q < EW / 4; ++q)
            out[d * (EW / 4) + q] = make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    }
}

__global__ void export_layout_kernel(const u32 *elem, int ew, int N, int layout, u64 nnz, u32 *idx_out,
                                     float *vals_out) {
    for (u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (u64)gridDim.x * blockDim.x) {
        const u32 *e = elem + p * (u64)ew;
        for (int w = 0; w < N; ++w) idx_out[(u64)w * nnz + p] = e[(w - layout + N) % N];
        vals_out[p] = __uint_as_float(e[N]);
    }
}

// Compute order of the stage tiles: for the tile [start, start + len) of a
// layout, perm_out[start + p] = the tile-local index of the nonzero that comes
// p-th when the tile is sorted stably by output index.  One block per tile:
// per-warp row counts, a scan, then stable ranks from __match_any_sync.
__global__ void __launch_bounds__(256)
    tile_order_kernel(const u32 *pi_in, const u32 *tile_ptr, const u32 *coord, u32 m, uint16_t *perm_out) {
    constexpr int W = 8;
    constexpr int M = (int)kMaxSuperShardRows;
    __shared__ u32 cnt[W][M];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 start = tile_ptr[blockIdx.x];
    const u32 len = tile_ptr[blockIdx.x + 1] - start;
    for (int i = threadIdx.x; i < W * M; i += blockDim.x) (&cnt[0][0])[i] = 0u;
    const u32 row_base = (coord[pi_in[start]] / m) * m;
    __syncthreads();
    const u32 per = (len + W - 1) / W;
    const u32 lo = min((u32)warp * per, len), hi = min(lo + per, len);
    const unsigned lt = (1u << lane) - 1u;
    for (u32 b0 = lo; b0 < hi; b0 += 32) {
        const u32 i = b0 + lane;
        const bool v = i < hi;
        const u32 lr = v ? min(coord[pi_in[start + i]] - row_base, (u32)M - 1u) : 0x10000u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, lr);
        if (v && (peers & lt) == 0) cnt[warp][lr] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // warp 0 turns the counts into start offsets: lane l owns the PER rows
    // l*PER .. l*PER + PER-1, warps in order inside a row
    constexpr int PER = M / 32;
    static_assert(M >= 32 && M % 32 == 0, "the row scan gives each lane M / 32 rows");
    if (warp == 0) {
        u32 tot[PER], run = 0;
        for (int c = 0; c < PER; ++c) {
            u32 t = 0;
            for (int w = 0; w < W; ++w) t += cnt[w][lane * PER + c];
            tot[c] = t;
            run += t;
        }
        u32 incl = run;
        for (int d = 1; d < 32; d <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        u32 base = incl - run;
        for (int c = 0; c < PER; ++c) {
            u32 o = base;
            for (int w = 0; w < W; ++w) {
                const u32 x = cnt[w][lane * PER + c];
                cnt[w][lane * PER + c] = o;
                o += x;
            }
            base += tot[c];
        }
    }
    __syncthreads();
    for (u32 b0 = lo; b0 < hi; b0 += 32) {
        const u32 i = b0 + lane;
        const bool v = i < hi;
        const u32 e = v ? pi_in[start + i] : 0u;
        const u32 lr = v ? min(coord[e] - row_base, (u32)M - 1u) : 0x10000u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, lr);
        u32 pos = 0;
        if (v) pos = cnt[warp][lr] + __popc(peers & lt);
        __syncwarp();
        if (v && (peers & lt) == 0) cnt[warp][lr] += __popc(peers);
        __syncwarp();
        if (v && pos < len) perm_out[start + pos] = (uint16_t)i;
    }
}

inline unsigned grid_for(u64 n, int threads = 256) {
    u64 b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1u << 20)) b = (1u << 20);
    return (unsigned)b;
}

int bits_for(u64 I) {
    int b = 0;
    while (b < 32 && (1ull << b) < I) ++b;
    return b;
}
} // namespace

// ===========================================================================
// K1 driver
// ===========================================================================
flycoo_status build_flycoo(Tensor &t, const u32 *d_idx, const float *d_vals,
                           std::vector<std::vector<u32>> &ss_ptr_host, cudaStream_t s) {
    const int N = t.N;
    const u64 nnz = t.nnz;
    ss_ptr_host.assign(N, {});
    if (t.order == FLYCOO_ORDER_MORTON) {
        for (int n = 0; n < N; ++n) {
            int total = 0;
            for (int q = 1; q < N; ++q) {
                const int w = (n + q) % N;
                const u64 kw = (t.dims[w] + t.mode[w].m - 1) / t.mode[w].m;
                int b = 0;
                while (b < 32 && (1ull << b) <= kw - 1) ++b;
                total += std::max(b, 1);
            }
            if (total > 64) {
                set_error("flycoo_create: the Z-Morton code of mode %d needs %d bits (at most 64)", n, total);
                return FLYCOO_ERR_INVALID_ARG;
            }
        }
    }
    // 1. coordinate range check
    DevBuf err;
    FLY_TRY(err.alloc(sizeof(u32)));
    FLY_TRY_CUDA(cudaMemsetAsync(err.p, 0, sizeof(u32), s));
    Dims dims{};
    for (int w = 0; w < N; ++w) dims.d[w] = (u32)t.dims[w];
    if (nnz) {
        check_index_kernel<<<grid_for(nnz * N), 256, 0, s>>>(d_idx, nnz, N, dims, err.as<u32>());
        FLY_TRY_CUDA(cudaGetLastError());
    }
    u32 h_err = 0;
    FLY_TRY_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(u32), cudaMemcpyDeviceToHost, s));
    FLY_TRY_CUDA(cudaStreamSynchronize(s));
    if (h_err) {
        set_error("flycoo_create: a coordinate is >= its mode size");
        return FLYCOO_ERR_INDEX_RANGE;
    }

    // 2. layouts by chained stable sorts
    const u64 ntiles = (nnz + kRsTile - 1) / kRsTile;
    DevBuf b_keys, b_vals, b_ktmp, b_vtmp, b_counts, b_scan;
    FLY_TRY(b_keys.alloc(nnz * 4));
    FLY_TRY(b_vals.alloc(nnz * 4));
    FLY_TRY(b_ktmp.alloc(nnz * 4));
    FLY_TRY(b_vtmp.alloc(nnz * 4));
    FLY_TRY(b_counts.alloc(256 * ntiles * 4));
    u64 scan_words = scan_scratch_words(std::max<u64>(256 * ntiles, 1));
    FLY_TRY(b_scan.alloc(scan_words * 4));
    std::vector<DevBuf> pi(N);
    for (int n = 0; n < N; ++n) FLY_TRY(pi[n].alloc(nnz * 4));

    u32 *keys = b_keys.as<u32>(), *vals = b_vals.as<u32>();
    u32 *ktmp = b_ktmp.as<u32>(), *vtmp = b_vtmp.as<u32>();
    const unsigned grid = grid_for(nnz);
    if (nnz) iota_kernel<<<grid, 256, 0, s>>>(vals, nnz);
    // super-shard ids: ss_w = c_w div m_w, k_w = ceil(I_w / m_w) of them
    std::vector<u64> kss(N);
    for (int w = 0; w < N; ++w) kss[w] = (t.dims[w] + t.mode[w].m - 1) / t.mode[w].m;
    std::vector<DevBuf> rp(N);
    auto sort_by_mode = [&](int w) -> flycoo_status {
        if (nnz) gather_div_kernel<<<grid, 256, 0, s>>>(d_idx + (u64)w * nnz, vals, keys, nnz, (u32)t.mode[w].m);
        FLY_TRY_CUDA(cudaGetLastError());
        return stable_sort_pairs(&keys, &vals, &ktmp, &vtmp, b_counts.as<u32>(), b_scan.as<u32>(), nnz,
                                 bits_for(kss[w]), s);
    };
    auto finish_mode = [&](int n) -> flycoo_status {
        // vals = pi_n, keys = super-shard ids of mode n in L_n order
        FLY_TRY_CUDA(cudaMemcpyAsync(pi[n].p, vals, nnz * 4, cudaMemcpyDeviceToDevice, s));
        FLY_TRY(rp[n].alloc((kss[n] + 1) * 4));
        row_ptr_kernel<<<grid_for(nnz + 1), 256, 0, s>>>(keys, nnz, kss[n], rp[n].as<u32>());
        FLY_TRY_CUDA(cudaGetLastError());
        return FLYCOO_OK;
    };
    if (t.order == FLYCOO_ORDER_KEY) {
        for (int w = 1; w < N; ++w) FLY_TRY(sort_by_mode(w));
        FLY_TRY(sort_by_mode(0));
        FLY_TRY(finish_mode(0));
        for (int n = 1; n < N; ++n) {
            FLY_TRY(sort_by_mode(n));
            FLY_TRY(finish_mode(n));
        }
    } else {
        // Z-Morton variant: each layout on its own, from the input order, by
        // stable sorts on the code's low word, its high word, then ss_n
        Dims mw{}, width{};
        for (int w = 0; w < N; ++w) {
            mw.d[w] = (u32)t.mode[w].m;
            int b = 0;
            while (b < 32 && (1ull << b) <= kss[w] - 1) ++b;
            width.d[w] = (u32)std::max(b, 1);
        }
        for (int n = 0; n < N; ++n) {
            int total = 0, maxw = 0;
            for (int q = 1; q < N; ++q) {
                total += (int)width.d[(n + q) % N];
                maxw = std::max(maxw, (int)width.d[(n + q) % N]);
            }
            if (nnz) iota_kernel<<<grid, 256, 0, s>>>(vals, nnz);
            for (int word = 0; word < 2 && word * 32 < total; ++word) {
                if (nnz)
                    morton_key_kernel<<<grid, 256, 0, s>>>(d_idx, nnz, N, n, mw, width, maxw, vals, keys, word);
                FLY_TRY_CUDA(cudaGetLastError());
                FLY_TRY(stable_sort_pairs(&keys, &vals, &ktmp, &vtmp, b_counts.as<u32>(), b_scan.as<u32>(), nnz,
                                          std::min(32, total - 32 * word), s));
            }
            FLY_TRY(sort_by_mode(n));
            FLY_TRY(finish_mode(n));
        }
    }

    // 3. host: super-shard pointers -> shards, tiles, schedules (Section III-A, Algorithm 3)
    for (int n = 0; n < N; ++n) {
        ss_ptr_host[n].resize(kss[n] + 1);
        FLY_TRY_CUDA(cudaMemcpyAsync(ss_ptr_host[n].data(), rp[n].p, (kss[n] + 1) * 4,
                                     cudaMemcpyDeviceToHost, s));
    }
    FLY_TRY_CUDA(cudaStreamSynchronize(s));
    for (int n = 0; n < N; ++n) FLY_TRY(partition_mode(t, n, ss_ptr_host[n], s));

    // 4. compute order of every stage tile of both sizes (stable sort by output index)
    for (int n = 0; n < N; ++n)
        for (int z = 0; z < 2; ++z) {
            // +32 bytes: tile loads round the order range out to 16-byte boundaries
            FLY_TRY(t.mode[n].d_perm[z].alloc(nnz * 2 + 32));
            FLY_TRY_CUDA(cudaMemsetAsync(t.mode[n].d_perm[z].p, 0, nnz * 2 + 32, s));
            const std::vector<u32> &tp = t.mode[n].tile_ptr[z];
            if (!nnz) continue;
            DevBuf d_tp;
            FLY_TRY(d_tp.alloc(tp.size() * 4));
            FLY_TRY_CUDA(cudaMemcpyAsync(d_tp.p, tp.data(), tp.size() * 4, cudaMemcpyHostToDevice, s));
            tile_order_kernel<<<(unsigned)(tp.size() - 1), 256, 0, s>>>(
                pi[n].as<u32>(), d_tp.as<u32>(), d_idx + (u64)n * nnz, (u32)t.mode[n].m,
                t.mode[n].d_perm[z].as<uint16_t>());
            FLY_TRY_CUDA(cudaGetLastError());
            FLY_TRY_CUDA(cudaStreamSynchronize(s)); // d_tp goes out of scope
        }

    // 5. remap permutations: next_n[p] = pos_{n+1}[pi_n[p]]
    {
        u32 *pos = ktmp; // scratch
        for (int n = 0; n < N; ++n) {
            const int m = (n + 1) % N;
            // +16 bytes: tile loads round the slot range out to 16-byte boundaries
            FLY_TRY(t.mode[n].d_next.alloc(nnz * 4 + 16));
            if (nnz) {
                inverse_kernel<<<grid, 256, 0, s>>>(pi[m].as<u32>(), pos, nnz);
                gather_kernel<<<grid, 256, 0, s>>>(pos, pi[n].as<u32>(), t.mode[n].d_next.as<u32>(), nnz);
                FLY_TRY_CUDA(cudaGetLastError());
            }
        }
    }

    // 6. element buffers, tensor stored in L_0
    const u64 eb = (u64)t.elem_words * 4;
    FLY_TRY(t.elem[0].alloc(nnz * eb));
    FLY_TRY(t.elem[1].alloc(nnz * eb));
    if (nnz) {
        build_elems_kernel<<<grid, 256, 0, s>>>(d_idx, d_vals, pi[0].as<u32>(), nnz, N, t.elem_words,
                                                t.elem[0].as<u32>());
        FLY_TRY_CUDA(cudaGetLastError());
    }
    t.cur = 0;
    t.layout = 0;
    FLY_TRY_CUDA(cudaStreamSynchronize(s));
    // the input position of every nonzero of L_0 stays with the handle (the
    // value gradient is written in input order)
    t.orig.swap(pi[0]);
    return FLYCOO_OK;
}

flycoo_status launch_remap_step(const Tensor &t, int n, const void *in, void *out, cudaStream_t s) {
    if (t.nnz == 0) return FLYCOO_OK;
    const u32 *next = t.mode[n].d_next.as<u32>();
    if (t.elem_words == 4)
        remap_step_kernel<4><<<grid_for(t.nnz), 256, 0, s>>>((const uint4 *)in, (uint4 *)out, next, t.nnz, t.N);
    else
        remap_step_kernel<8><<<grid_for(t.nnz), 256, 0, s>>>((const uint4 *)in, (uint4 *)out, next, t.nnz, t.N);
    FLY_TRY_CUDA(cudaGetLastError());
    return FLYCOO_OK;
}

flycoo_status launch_export_layout(const Tensor &t, const void *elem, u32 *idx_out, float *vals_out,
                                   cudaStream_t s) {
    if (t.nnz == 0) return FLYCOO_OK;
    export_layout_kernel<<<grid_for(t.nnz), 256, 0, s>>>((const u32 *)elem, t.elem_words, t.N, t.layout,
                                                         t.nnz, idx_out, vals_out);
    FLY_TRY_CUDA(cudaGetLastError());
    return FLYCOO_OK;
}

} // namespace flycoo
