// fused.cuh -- K2: spMTTKRP of one mode with the dynamic remap fused into the
// same pass (Algorithm 2, one value of n), and K4: the fixed-order sum of the
// row blocks of super-shards that the schedule splits into several segments.
//
// Layout.  The tensor is in layout L_n: nonzeros ordered by the key of
// super-shard ids (ss_n, ss_{n-1}, ..., ss_{n+1}, input position) with
// ss_w = c_w div m_w, cut into shards of at most g consecutive nonzeros
// (Section III-A).  Under this key L_{n+1} is L_n stably sorted by ss_{n+1},
// so the nonzeros of a tile that share (ss_{n-1}, ..., ss_{n+1}) land in one
// contiguous run of L_{n+1}: the remap stores of a warp are mostly coalesced.
//
// Work decomposition.  Thread block b walks the stage tiles of the shards that
// Algorithm 3 put in bin b (runs of 1024 positions from a shard start when
// three such blocks fit on an SM, else 512).  A shard's super-shard owns m_n
// output rows, which the block accumulates in shared memory (the paper keeps
// them in cache, Eq. 3), across all shards of that super-shard that follow
// each other in the bin (a segment).  One thread streams the tiles with 1-D
// TMA bulk copies into a two-stage shared buffer on mbarriers, two tiles
// ahead: the nonzeros and the tile's compute order (a precomputed u16
// permutation that sorts the tile stably by output index); it prefetches the
// nonzeros' slots in L_{n+1} into L2 and publishes each tile's 16-byte
// descriptor with it.  For each tile:
//
//  1. remap: every thread stores a few of the tile's nonzeros at their slots of
//     L_{n+1} (the Store of Algorithm 2's remap step), in one burst, in
//     layout order;
//  2. compute: each group of L lanes takes a fixed slice of the tile in its
//     compute order, where a row's nonzeros are contiguous; its lanes split
//     the rank dimension (16 or 32 bytes of a factor row per lane).  Per nonzero it
//     gathers the N-1 input factor rows and adds val * Hadamard product (FP32)
//     to a running row sum in registers.  A run of one row that lies inside
//     the slice is added to its shared-memory accumulator by the group alone;
//  3. combine: a run that crosses a slice edge is summed after the block
//     barrier, in slice order, by the group where it starts; when no run
//     crosses an edge this step and its barrier are skipped.
//
// At the end of a segment the accumulator rows go straight to the output when
// the super-shard has no other segment, else to the segment's row block, and
// the accumulator is zeroed; K4 then sums the blocks of a super-shard in a
// fixed order.  Every accumulator row is updated by one thread group at a
// time, in an order fixed by the layout and the launch shape, so results are
// bitwise reproducible; no atomics touch the data.  Rows without nonzeros come
// out as zeros.
//
// Every wait on an mbarrier is bounded; a block whose wait gives up sets the
// error word, lets its copies in flight land (bounded) and returns.
#pragma once

#include "internal.cuh"

#include <type_traits>

namespace flycoo {

// warps whose groups all have full slices skip the clamps and weights (1)
#ifndef FLYCOO_FULL_FAST
#define FLYCOO_FULL_FAST 1
#endif
// unroll factor of a full tile's compute steps
#ifndef FLYCOO_FULL_UNROLL
#define FLYCOO_FULL_UNROLL 2
#endif
constexpr int kFullUnroll = FLYCOO_FULL_UNROLL;
// warps of a thread block of the fused kernel
#ifndef FLYCOO_WARPS
#define FLYCOO_WARPS 8
#endif
// registers of gathered factor data a lane may hold per compute step
#ifndef FLYCOO_LOAD_REGS
#define FLYCOO_LOAD_REGS 32
#endif

// 16-byte loads of one factor row per lane for FP32 factors: a lane takes
// FLYCOO_FP32_CHUNKS chunks of 4 values, chunk c from the c-th part of the row,
// so every load instruction of a warp still covers whole sectors.  One chunk is
// the default: with two, a warp's load instruction touches twice as many rows
// (lines), which costs more in L1 than the shared per-nonzero work saves.
#ifndef FLYCOO_FP32_CHUNKS
#define FLYCOO_FP32_CHUNKS 1
#endif
// the same for R = 64, where a row is two lines and two chunks per lane still
// keep each warp load at four lines
#ifndef FLYCOO_FP32_CHUNKS_R64
#define FLYCOO_FP32_CHUNKS_R64 2
#endif

// FP32 factors at R >= 32: each lane loads 32 bytes of a row in one
// instruction (a group of R/8 lanes covers a row), so a warp's gather serves
// twice as many nonzeros as with 16-byte loads at the same one line per row
#ifndef FLYCOO_WIDE_FP32
#define FLYCOO_WIDE_FP32 1
#endif

template <int N, int R, bool BF16>
struct FusedCfg {
    static constexpr int LB = (!BF16 && FLYCOO_WIDE_FP32 && R >= 32) ? 32 : 16; // bytes per lane load
    static constexpr int CW = LB / 4;               // 32-bit words per load
    static constexpr int CV = BF16 ? 2 * CW : CW;   // factor values per load
    static constexpr int CPL = (LB == 32 || BF16 || N >= 5) ? 1
                               : (R >= 64 ? FLYCOO_FP32_CHUNKS_R64 : FLYCOO_FP32_CHUNKS);
    static constexpr int VEC = CPL * CV;            // factor values per lane
    static constexpr int L = R / VEC;               // lanes per group
    static constexpr int GPW = 32 / L;              // groups per warp
    static constexpr int WARPS = FLYCOO_WARPS;
    static constexpr int THREADS = WARPS * 32;
    static constexpr int G = WARPS * GPW;           // groups per block
    static constexpr int EW = (N + 1 <= 4) ? 4 : 8; // 32-bit words per stored nonzero
    static constexpr int EQ = EW / 4;               // 16-byte chunks per stored nonzero
    static constexpr int EB = EW * 4;               // bytes per stored nonzero
    static constexpr int M = R > kMaxRank ? (int)kMaxRowsAtRank128 : (int)kMaxSuperShardRows; // accumulator rows
    // shared memory: two stages (nonzeros and the compute order; the order
    // load is rounded out to 16-byte boundaries, at most cap + 8 entries), the
    // row accumulators and the slice summaries.  The remap slots are not staged:
    // they are prefetched into L2 with the tile and read once from there.
    static constexpr size_t PERM_OFF(size_t cap) { return cap * EB; }
    static constexpr size_t stage_bytes(size_t cap) { return PERM_OFF(cap) + (cap + 8) * 2; }
    static constexpr size_t ACC = (size_t)M * R * 4;
    static constexpr size_t SUMBUF = (size_t)G * R * 4 + (((size_t)G * 4 + 15) & ~(size_t)15);
    // + 80 bytes: four 16-byte descriptor slots and two mbarriers
    static constexpr size_t smem_bytes(size_t cap) { return 2 * stage_bytes(cap) + ACC + SUMBUF + 80; }
    // the larger stage tile when kBlocksPerSM blocks of it fit in an SM's 228 KB
    // (1 KB of each block is reserved by the system); FLYCOO_STAGE_TILE forces one
#ifdef FLYCOO_STAGE_TILE
    static constexpr int TZ = FLYCOO_STAGE_TILE == FLYCOO_STAGE_TILE_LARGE ? 1 : 0;
#else
    static constexpr int TZ = (kBlocksPerSM * (smem_bytes(kStageTile[1]) + 1024) <= 228 * 1024) ? 1 : 0;
#endif
    static constexpr int CAP = (int)kStageTile[TZ];
    static constexpr size_t STAGE = stage_bytes(CAP);
    static constexpr size_t SMEM = smem_bytes(CAP);
    static_assert(R % VEC == 0 && L >= 1 && L <= 32 && 32 % L == 0 && (R / CV) % CPL == 0, "rank not supported");
    static_assert(STAGE % 16 == 0 && SUMBUF % 16 == 0 && ACC % 16 == 0, "shared-memory alignment");
};

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and 1-D TMA bulk copy (global -> shared)
// ---------------------------------------------------------------------------
__device__ __forceinline__ u32 smem_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, u32 parity) {
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bulk prefetch of [src, src + bytes) into L2 (16-byte aligned, a multiple of 16 bytes)
__device__ __forceinline__ void l2_prefetch_bulk(const void *src, u32 bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// a streamed 32-bit value read once: not kept in L1, first out of L2
__device__ __forceinline__ u32 ld_stream_u32(const u32 *p, uint64_t policy) {
    u32 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(policy));
    return v;
}

__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, u32 bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// L2 cache policies.  The pass streams the element buffers (read once, written
// once) past factor matrices that every nonzero gathers from: the streams are
// marked evict-first so the factor rows, marked evict-last, stay in L2.
#ifndef FLYCOO_L2_HINTS
#define FLYCOO_L2_HINTS 1
#endif
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void tma_load_1d_hint(void *dst, const void *src, u32 bytes, uint64_t *bar,
                                                 uint64_t policy) {
#if FLYCOO_L2_HINTS
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
#else
    tma_load_1d(dst, src, bytes, bar);
#endif
}
// CW 32-bit words of a factor row, loaded by one lane in one instruction
template <int CW> struct __align__(CW * 4) Chunk { u32 w[CW]; };

__device__ __forceinline__ Chunk<4> ld_factor(const Chunk<4> *p, uint64_t policy) {
    Chunk<4> v;
#if FLYCOO_L2_HINTS
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3])
        : "l"(p), "l"(policy));
#else
    asm("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3])
        : "l"(p));
#endif
    return v;
}

__device__ __forceinline__ Chunk<8> ld_factor(const Chunk<8> *p, uint64_t policy) {
    Chunk<8> v;
#if FLYCOO_L2_HINTS
    asm("ld.global.nc.L2::cache_hint.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
        : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3]), "=r"(v.w[4]), "=r"(v.w[5]), "=r"(v.w[6]),
          "=r"(v.w[7])
        : "l"(p), "l"(policy));
#else
    asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3]), "=r"(v.w[4]), "=r"(v.w[5]), "=r"(v.w[6]),
          "=r"(v.w[7])
        : "l"(p));
#endif
    return v;
}

// 16-byte cp.async (global -> shared) for thread 0's look-ahead descriptors:
// the copy lands while the tile is computed; the thread waits for its own group
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int Pending>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(Pending) : "memory");
}

// bounded wait (at most `limit` polls); true on success
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, u32 parity, u32 limit = kSpinLimit) {
    for (u32 i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------------------
// the FP32 values of a chunk: one per word, or two per word for BF16
template <bool BF16, int CW>
__device__ __forceinline__ void widen(const Chunk<CW> &v, float *f) {
#pragma unroll
    for (int q = 0; q < CW; ++q) {
        if constexpr (BF16) {
            f[2 * q] = __uint_as_float(v.w[q] << 16);
            f[2 * q + 1] = __uint_as_float(v.w[q] & 0xffff0000u);
        } else {
            f[q] = __uint_as_float(v.w[q]);
        }
    }
}

// a remapped nonzero: written once and not read again in this pass, so it is
// kept out of L1, where the factor rows being gathered live
__device__ __forceinline__ void st_no_l1(uint4 *p, const uint4 v, uint64_t policy) {
#if FLYCOO_L2_HINTS
    asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x),
                 "r"(v.y), "r"(v.z), "r"(v.w), "l"(policy)
                 : "memory");
#else
    asm volatile("st.global.L1::no_allocate.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
#endif
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
__device__ __forceinline__ void add_vec(float *acc, const float *src) {
    float x[VEC];
    load_vec<VEC>(src, x);
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] += x[v];
}

// A tile descriptor: four words start, len | flags << 16, super-shard, shard.
constexpr u32 kTileFirst = 1u, kTileLast = 2u, kTileAlone = 4u;

template <int N, int R, bool BF16, bool CPOPT>
__global__ void __launch_bounds__(FLYCOO_WARPS * 32, kBlocksPerSM) fused_mttkrp_remap_kernel(const FusedArgs a) {
    using C = FusedCfg<N, R, BF16>;
    static_assert(!(CPOPT && BF16), "the CP-OPT gradient pass takes FP32 factors");
    constexpr int VEC = C::VEC;     // factor values per lane
    constexpr int CV = C::CV;       // values per lane load
    constexpr int CPL = C::CPL;     // loads per row per lane
    constexpr int RV = R / CV;      // load-sized chunks per factor row
    constexpr int RC = RV / CPL;    // chunks per part of a row (lane k loads chunk k of each part)
    using ChunkT = Chunk<C::CW>;
    constexpr int CAP = C::CAP;
    constexpr int G = C::G;
    constexpr int M = C::M;
    constexpr int NF = CPOPT ? N : N - 1;            // factor rows gathered per nonzero
    // nonzeros per group per step: the gathered rows of a step take at most 32
    // registers per lane (U * NF * CPL loads of CW words)
    constexpr int LOADREGS = NF * CPL * C::CW;
    constexpr int U = (N >= 5 || FLYCOO_LOAD_REGS / LOADREGS < 1)
                          ? 1
                          : ((FLYCOO_LOAD_REGS / LOADREGS) > FLYCOO_UNROLL3 ? FLYCOO_UNROLL3
                                                                            : FLYCOO_LOAD_REGS / LOADREGS);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *acc = reinterpret_cast<float *>(smem_raw + 2 * C::STAGE);          // [M][R]
    float *hacc = acc + M * R;                                               // [G][R] head partials
    u32 *pass = reinterpret_cast<u32 *>(hacc + G * R);                       // [G]
    // sdesc[0..1]: descriptor of the tile in each stage; sdesc[2 + (t & 1)]:
    // thread 0's look-ahead copy of the descriptor of tile t
    uint4 *sdesc = reinterpret_cast<uint4 *>(smem_raw + 2 * C::STAGE + C::ACC + C::SUMBUF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sdesc + 4);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int k = lane % C::L;
    const int grp = warp * C::GPW + lane / C::L;
    const bool remap = a.elem_out != nullptr;
    const uint4 *__restrict__ ein = static_cast<const uint4 *>(a.elem_in);
    uint4 *__restrict__ eout = static_cast<uint4 *>(a.elem_out);
    const ChunkT *Yp[N - 1];
#pragma unroll
    for (int t = 0; t < N - 1; ++t) Yp[t] = static_cast<const ChunkT *>(a.Y[t]) + k;
    // CP-OPT: the output mode's own factor, for the model value at each nonzero
    const ChunkT *Yo = CPOPT ? static_cast<const ChunkT *>(a.Yout) + k : nullptr;
    double loss = 0.0;      // CP-OPT: this lane's sum of the tiles' squared residuals
    float *my_hacc = hacc + grp * R;
    // this lane's values of a row: part c holds columns c*(R/CPL) + k*CV .. + CV-1
    auto lane_store = [&](float *row, const float *v) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) store_vec<CV>(row + c * (R / CPL) + k * CV, v + c * CV);
    };
    auto lane_add = [&](float *v, const float *row) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) add_vec<CV>(v + c * CV, row + c * (R / CPL) + k * CV);
    };
    // add this lane's values to a row of the accumulator in shared memory (a
    // load, add and store: measured faster than red.shared.add here)
    auto lane_red = [&](float *row, float *v) {
        lane_add(v, row);
        lane_store(row, v);
    };
    const uint64_t pol_stream = l2_policy_evict_first();
    const uint64_t pol_factor = l2_policy_evict_last();
    const uint4 *__restrict__ tiles = a.tiles[C::TZ];
    const uint16_t *__restrict__ gperm = a.perm[C::TZ];
    const u32 t_begin = a.tile_bin_ptr[C::TZ][blockIdx.x];
    const u32 ntile = a.tile_bin_ptr[C::TZ][blockIdx.x + 1] - t_begin;

    // the accumulator starts at zero; the flush at the end of every shard zeroes it again
    for (u32 i = tid; i < (u32)(M * R / 4); i += C::THREADS)
        reinterpret_cast<float4 *>(acc)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // thread 0: load a tile (its nonzeros and its compute order) into a stage
    // and prefetch its next-layout slots into L2.  The order and slot ranges
    // are rounded out to the 16-byte boundaries around the tile (both arrays
    // are padded at the end).  The descriptor written to sdesc reaches the
    // waiting threads through the release of the arrive and the acquire of
    // their wait on the same barrier.
    auto issue = [&](int st, const uint4 d) {
        const u32 start = d.x, len = d.y & 0xffffu;
        unsigned char *sb = smem_raw + (size_t)st * C::STAGE;
        const u32 plo = start & ~7u;
        const u32 phi = (start + len + 7u) & ~7u;
        sdesc[st] = d;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[st], len * C::EB + (phi - plo) * 2u);
        tma_load_1d_hint(sb, ein + (size_t)start * C::EQ, len * C::EB, &bar[st], pol_stream);
        tma_load_1d_hint(sb + C::PERM_OFF(CAP), gperm + plo, (phi - plo) * 2u, &bar[st], pol_stream);
        if (remap) {
            const u32 nlo = start & ~3u;
            const u32 nhi = (start + len + 3u) & ~3u;
            l2_prefetch_bulk(a.next + nlo, (nhi - nlo) * 4u);
        }
    };
    if (tid == 0) {
        if (ntile > 0) issue(0, tiles[t_begin]);
        if (ntile > 1) issue(1, tiles[t_begin + 1]);
        if (ntile > 2) cp_async16(&sdesc[2], tiles + t_begin + 2);
        cp_async_commit();
    }

    for (u32 q = 0; q < ntile; ++q) {
        const int st = q & 1;
        // warp-uniform, so the warp-collective code below runs with every lane or none
        const bool timed_out = __any_sync(0xffffffffu, !mbar_wait_bounded(&bar[st], (q >> 1) & 1u, a.wait_limit));
        // the descriptor is valid only after a successful wait (it is published by
        // the arrive that the wait acquires); a tile that gave up uses length 1 and
        // touches no global memory, so every index below stays inside the stage
        const uint4 d = sdesc[st];
        if (tid == 0) { // the descriptor of tile q + 3, needed when tile q + 1 ends
            if (q + 3 < ntile) cp_async16(&sdesc[2 + ((q + 3) & 1)], tiles + t_begin + q + 3);
            cp_async_commit();
        }
        const u32 tstart = d.x;
        const u32 tlen = timed_out ? 1u : min(d.y & 0xffffu, (u32)CAP);
        const u32 flags = d.y >> 16;
        const u32 row_base = d.z * a.m;
        const u32 m_eff = min(a.m, a.I_out - row_base);
        const unsigned char *sb = smem_raw + (size_t)st * C::STAGE;
        const uint4 *selem = reinterpret_cast<const uint4 *>(sb);
        const u32 *gnext = a.next + tstart; // this tile's next-layout slots (prefetched into L2)
        // sperm[p]: tile-local index of the nonzero at compute position p; every
        // read is clamped to the stage, so even the unloaded order of a tile whose
        // wait gave up cannot index outside it
        const uint16_t *sperm = reinterpret_cast<const uint16_t *>(sb + C::PERM_OFF(CAP)) + (tstart & 7u);
        auto elem_at = [&](u32 p) { return min((u32)sperm[p], (u32)CAP - 1u); };

        // 1. remap burst: thread i stores the nonzeros i, i + THREADS, ... of the
        // tile at their slots, loading two slots before each pair of stores
        if (remap && !timed_out) {
            constexpr int RPT = (CAP + C::THREADS - 1) / C::THREADS;
            constexpr int PAIR = RPT >= 2 ? 2 : 1;
#pragma unroll
            for (int r0 = 0; r0 < RPT; r0 += PAIR) {
            u32 dst[PAIR];
#pragma unroll
            for (int r = 0; r < PAIR; ++r) {
                const u32 i = tid + (r0 + r) * C::THREADS;
                dst[r] = i < tlen ? ld_stream_u32(gnext + i, pol_stream) : 0u;
            }
#pragma unroll
            for (int r = 0; r < PAIR; ++r) {
                const u32 i = tid + (r0 + r) * C::THREADS;
                if (i >= tlen) break;
                u32 w[C::EW], o[C::EW];
#pragma unroll
                for (int c = 0; c < C::EQ; ++c) {
                    const uint4 x = selem[i * C::EQ + c];
                    w[4 * c] = x.x;
                    w[4 * c + 1] = x.y;
                    w[4 * c + 2] = x.z;
                    w[4 * c + 3] = x.w;
                }
#pragma unroll
                for (int t = 0; t < C::EW; ++t) o[t] = (t < N) ? w[(t + 1) % N] : w[t];
#pragma unroll
                for (int c = 0; c < C::EQ; ++c)
                    st_no_l1(eout + (size_t)dst[r] * C::EQ + c,
                             make_uint4(o[4 * c], o[4 * c + 1], o[4 * c + 2], o[4 * c + 3]), pol_stream);
            }
            }
        }

        // 2. compute this group's slice [lo, hi) of the tile's compute order,
        // in which each row's nonzeros are contiguous.  Slices are chunk positions long
        // (odd, so the groups of a warp read different shared-memory banks).  A
        // run of one row that lies inside the slice is added by this group
        // alone; a run that crosses a slice edge is summed in step 3.
        // (a full tile, the common case, takes the compile-time values)
        // (exactly CAP / G when that splits into whole steps; else odd)
        constexpr u32 kChunkFull = ((u32)CAP % (u32)(G * U) == 0) ? (u32)CAP / G : (((u32)(CAP + G - 1) / G) | 1u);
        constexpr u32 kGeffFull = ((u32)CAP + kChunkFull - 1) / kChunkFull;
        const u32 chunk = (tlen == (u32)CAP) ? kChunkFull : (((tlen + G - 1) / G) | 1u);
        const u32 geff = (tlen == (u32)CAP) ? kGeffFull : (tlen + chunk - 1) / chunk;
        const u32 *sw = reinterpret_cast<const u32 *>(sb); // word 0 of a stored nonzero is its row index
        // row of the nonzero at compute position p
        auto row_at = [&](u32 p) { return sw[(size_t)elem_at(p) * C::EW]; };
        const u32 lo = min((u32)grp * chunk, tlen);
        const u32 hi = min(lo + chunk, tlen);
        // the slice's first run continues the previous slice's row / its last run
        // continues into the next slice
        const bool head_shared = lo > 0 && lo < hi && row_at(lo) == row_at(lo - 1);
        const bool tail_shared = hi < tlen && lo < hi && row_at(hi) == row_at(hi - 1);
        // every group of a warp runs the same number of steps: positions past
        // the slice end repeat the slice's last nonzero with weight 0 (same
        // row, so no run ends there), and an empty slice repeats the tile's
        // last nonzero the same way
        const u32 wlen = chunk;
        const u32 last = (lo < hi) ? hi - 1 : tlen - 1;
        float racc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) racc[v] = 0.f;
        // CP-OPT: squared residuals of this slice (at most a few dozen terms) in
        // FP32, added to the lane's FP64 sum once per tile
        float tloss = 0.f;
        u32 crow = min(row_at(min(lo, last)) - row_base, (u32)M - 1u);
        // the first run goes to the head slot when it continues the previous slice's row
        bool first_run = head_shared;
        // FULL: every position of the step lies inside the slice (no clamp, weight val)
        auto steps = [&](u32 j0, auto count, auto full) {
            constexpr int UU = decltype(count)::value;
            constexpr bool FULL = decltype(full)::value;
            u32 w[UU][N + 1];
            ChunkT y[UU][NF][CPL];
#pragma unroll
            for (int u = 0; u < UU; ++u) {
                const u32 e = elem_at(FULL ? lo + j0 + u : min(lo + j0 + u, last));
#pragma unroll
                for (int c = 0; c < C::EQ; ++c) {
                    const uint4 x = selem[(size_t)e * C::EQ + c];
                    const u32 xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (4 * c + e <= N) w[u][4 * c + e] = xs[e];
                }
            }
#pragma unroll
            for (int u = 0; u < UU; ++u) {
#pragma unroll
                for (int t = 0; t < N - 1; ++t)
#pragma unroll
                    for (int c = 0; c < CPL; ++c)
                        y[u][t][c] = ld_factor(Yp[t] + (size_t)w[u][t + 1] * RV + c * RC, pol_factor);
                if constexpr (CPOPT)
#pragma unroll
                    for (int c = 0; c < CPL; ++c) y[u][N - 1][c] = ld_factor(Yo + (size_t)w[u][0] * RV + c * RC, pol_factor);
            }
#pragma unroll
            for (int u = 0; u < UU; ++u) {
                const bool valid = FULL || lo + j0 + u < hi;
                const u32 row = min(w[u][0] - row_base, (u32)M - 1u);
                float prod[VEC];
#pragma unroll
                for (int c = 0; c < CPL; ++c) widen<BF16>(y[u][0][c], prod + c * CV);
#pragma unroll
                for (int t = 1; t < N - 1; ++t) {
                    float f[VEC];
#pragma unroll
                    for (int c = 0; c < CPL; ++c) widen<BF16>(y[u][t][c], f + c * CV);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) prod[v] *= f[v];
                }
                const float val = __uint_as_float(w[u][N]);
                float coef = valid ? val : 0.f;
                if constexpr (CPOPT) {
                    // model value m = <Y_n[c_n], prod>: lane partials summed over the group
                    float yo[VEC];
#pragma unroll
                    for (int c = 0; c < CPL; ++c) widen<false>(y[u][N - 1][c], yo + c * CV);
                    float mpart = 0.f;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) mpart = fmaf(yo[v], prod[v], mpart);
#pragma unroll
                    for (int off = C::L / 2; off >= 1; off >>= 1) mpart += __shfl_xor_sync(0xffffffffu, mpart, off);
                    const float e = val - mpart; // residual x - m
                    if (valid) tloss = fmaf(e, e, tloss);
                    coef = valid ? -e : 0.f;     // dL/dY_n += -e * prod
                }
                if (row != crow) {
                    if (first_run) {
                        lane_store(my_hacc, racc);
                        if (k == 0) pass[grp] = 0u;
                        first_run = false;
                    } else {
                        // a whole row of this tile: only this group holds it
                        lane_red(acc + crow * R, racc);
                    }
                    crow = row;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) racc[v] = 0.f;
                }
#pragma unroll
                for (int v = 0; v < VEC; ++v) racc[v] = fmaf(coef, prod[v], racc[v]);
            }
        };
        if (!timed_out) {
            using One = std::integral_constant<int, 1>;
            using Many = std::integral_constant<int, U>;
            using Yes = std::true_type;
            using No = std::false_type;
            u32 j0 = 0;
            // warp-uniform: every group of the warp has a full slice of whole steps
            if (FLYCOO_FULL_FAST && __all_sync(0xffffffffu, hi - lo == wlen && wlen % U == 0)) {
                if (kChunkFull % U == 0 && tlen == (u32)CAP) {
                    // a full tile: every slice is kChunkFull positions, a compile-time trip count
#pragma unroll kFullUnroll
                    for (u32 jj = 0; jj < kChunkFull; jj += U) steps(jj, Many{}, Yes{});
                } else {
                    for (; j0 < wlen; j0 += U) steps(j0, Many{}, Yes{});
                }
            } else {
                for (; j0 + U <= wlen; j0 += U) steps(j0, Many{}, No{});
                for (; j0 < wlen; ++j0) steps(j0, One{}, No{});
            }
        }
        if constexpr (CPOPT) {
            // every lane of a group holds the group's residuals: one lane counts them
            if (k == 0) loss += (double)tloss;
        }
        // the slice's last run: added here when it ends at the slice end, else kept
        // for step 3 (in registers when its row starts in this slice, in the head
        // slot, marked pass-through, when the whole slice is one piece of a longer row)
        bool chain_start = false;
        if (!timed_out && lo < hi) {
            if (tail_shared) {
                if (first_run) {
                    lane_store(my_hacc, racc);
                    if (k == 0) pass[grp] = 1u;
                } else {
                    chain_start = true;
                }
            } else if (first_run) {
                lane_store(my_hacc, racc);
                if (k == 0) pass[grp] = 0u;
            } else {
                lane_red(acc + crow * R, racc);
            }
        }
        // one barrier reports both: every lane of a warp that gave up counts (32 per
        // warp), and lane 0 of a warp holding a chain start counts once (at most
        // C::WARPS < 32), so count >= 32 means a wait gave up and count > 0 that
        // step 3 has work
        static_assert(C::WARPS < 32, "the barrier count encoding needs fewer than 32 warps");
        const bool warp_chain = __any_sync(0xffffffffu, chain_start);
        const int nsync = __syncthreads_count(timed_out || (lane == 0 && warp_chain));
        if (nsync >= 32) {
            if (tid == 0) {
                atomicOr(a.err, 1u);
                // let the copies still in flight land before the block's shared memory is
                // released (always with the full bound, whatever a.wait_limit is)
                mbar_wait_bounded(&bar[st], (q >> 1) & 1u);
                if (q + 1 < ntile) mbar_wait_bounded(&bar[st ^ 1], ((q + 1) >> 1) & 1u);
                cp_async_wait<0>();
            }
            return;
        }
        // every thread is past its reads of this stage: load the tile after next into it
        if (tid == 0 && q + 2 < ntile) {
            cp_async_wait<1>(); // every group but the one committed at this tile's start
            issue(st, sdesc[2 + ((q + 2) & 1)]);
        }

        // 3. rows longer than a chunk: the group where such a row starts adds the
        // head partials of the following slices, in slice order, through the last
        // one that is not a pass-through, then adds the sum to the accumulator
        if (nsync > 0) {
            if (chain_start) {
                for (u32 g2 = grp + 1; g2 < geff; ++g2) {
                    lane_add(racc, hacc + g2 * R);
                    if (!pass[g2]) break;
                }
                float *dst = acc + crow * R;
                lane_add(racc, dst);
                lane_store(dst, racc);
            }
            // the next tile's slices may hold this row: their adds wait here
            __syncthreads();
        }
        // end of the segment: its super-shard's rows to the output (the only
        // segment of its super-shard) or to the segment's row block, and the
        // accumulator back to zero
        if (flags & kTileLast) {
            float4 *dst = (flags & kTileAlone) ? reinterpret_cast<float4 *>(a.out + (size_t)row_base * R)
                                               : reinterpret_cast<float4 *>(a.partials + (size_t)d.w * a.m * R);
            const u32 nout = m_eff * (R / 4);
            for (u32 i = tid; i < (u32)(M * R / 4); i += C::THREADS) {
                float4 *ai = reinterpret_cast<float4 *>(acc) + i;
                if (i < nout) dst[i] = *ai;
                *ai = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
        }
    }
    if (tid == 0) cp_async_wait<0>(); // no look-ahead copy outlives the block
    if constexpr (CPOPT) {
        // half the sum of squared residuals of this block, reduced in a fixed order
        if (a.loss_part) {
            __shared__ double wsum[C::WARPS];
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, off);
            if (lane == 0) wsum[warp] = loss;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < C::WARPS; ++w) t += wsum[w];
                a.loss_part[blockIdx.x] = 0.5 * t;
            }
        }
    }
}

// K4: rows of the super-shards that do not have exactly one segment: the sum of
// their segments' row blocks (zero for an empty super-shard), in an order fixed
// by the plan, so the sum is the same in every run.
//  * A light item (at most kFixupLightSegs segments) has one block: thread t
//    sums float4 columns t, t + 256, ... of the row blocks in four interleaved
//    chains (segments i, i + 4, i + 8, ... in chain i), added as (0 + 1) + (2 + 3).
//  * Any other item has one block per 64 floats of its row block: 16 parts of 16
//    threads take every 16th segment, each part in four chains the same way,
//    and the parts are added in a fixed tree order.
// Independent chains keep four loads of a thread in flight, and a light item's
// dependent loads (item, segment range, row blocks) are paid once per block.
static __global__ void __launch_bounds__(256) super_shard_fixup_kernel(const FixupArgs a, u32 R) {
    constexpr u32 kParts = 16, kChains = 4;
    __shared__ float4 part_sum[kParts][16];
    const u32 b = blockIdx.x;
    const bool light = b < a.nlight;
    const u32 chunks = (a.m * R + 63) / 64;
    const u32 item = light ? b : a.nlight + (b - a.nlight) / chunks;
    const u32 j = a.items[item];
    const u32 row_base = j * a.m;
    const u32 m_eff = min(a.m, a.I_out - row_base);
    const u32 nfl = m_eff * R;                         // a multiple of 4 (R is)
    const u32 s0 = a.ss_seg_ptr[j], s1 = a.ss_seg_ptr[j + 1];
    const size_t block = (size_t)a.m * R;
    auto add4 = [](float4 p, float4 q) { return make_float4(p.x + q.x, p.y + q.y, p.z + q.z, p.w + q.w); };
    // chains c of segments first, first + stride c, first + 2 stride c, ... below s1
    auto chains = [&](u32 first, u32 stride, u32 f) {
        float4 ch[kChains];
#pragma unroll
        for (u32 c = 0; c < kChains; ++c) ch[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        u32 s = first;
        for (; s + (kChains - 1) * stride < s1; s += kChains * stride) {
            float4 x[kChains];
#pragma unroll
            for (u32 c = 0; c < kChains; ++c)
                x[c] = *reinterpret_cast<const float4 *>(a.partials + (size_t)(s + c * stride) * block + f);
#pragma unroll
            for (u32 c = 0; c < kChains; ++c) ch[c] = add4(ch[c], x[c]);
        }
        // at most kChains - 1 segments are left
#pragma unroll
        for (u32 c = 0; c + 1 < kChains; ++c)
            if (s + c * stride < s1)
                ch[c] = add4(ch[c], *reinterpret_cast<const float4 *>(a.partials + (size_t)(s + c * stride) * block + f));
        return add4(add4(ch[0], ch[1]), add4(ch[2], ch[3]));
    };
    if (light) {
        for (u32 f = threadIdx.x * 4; f < nfl; f += 256 * 4)
            *reinterpret_cast<float4 *>(a.out + (size_t)row_base * R + f) = chains(s0, 1, f);
        return;
    }
    const u32 c4 = threadIdx.x & 15;
    const u32 part = threadIdx.x >> 4;
    const u32 f = (b - a.nlight) % chunks * 64 + c4 * 4;
    part_sum[part][c4] = f < nfl ? chains(s0 + part, kParts, f) : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
#pragma unroll
    for (u32 h = kParts / 2; h >= 1; h >>= 1) {
        if (part < h) part_sum[part][c4] = add4(part_sum[part][c4], part_sum[part + h][c4]);
        __syncthreads();
    }
    if (part == 0 && f < nfl) *reinterpret_cast<float4 *>(a.out + (size_t)row_base * R + f) = part_sum[0][c4];
}

template <int N, int R, bool BF16, bool CPOPT = false>
flycoo_status launch_fused_t(const FusedArgs &a, cudaStream_t s) {
    using C = FusedCfg<N, R, BF16>;
    auto kern = fused_mttkrp_remap_kernel<N, R, BF16, CPOPT>;
    if (C::SMEM > 48 * 1024)
        FLY_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    kern<<<a.bins, C::THREADS, C::SMEM, s>>>(a);
    FLY_TRY_CUDA(cudaGetLastError());
    return FLYCOO_OK;
}

template <int N>
flycoo_status launch_fused_dispatch(int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s) {
    const bool bf = dt == FLYCOO_BF16;
    if (a.Yout) { // CP-OPT gradient pass (FP32 factors)
        if (bf) {
            set_error("the CP-OPT gradient pass takes FP32 factors");
            return FLYCOO_ERR_UNSUPPORTED;
        }
        switch (R) {
        case 16: return launch_fused_t<N, 16, false, true>(a, s);
        case 32: return launch_fused_t<N, 32, false, true>(a, s);
        case 64: return launch_fused_t<N, 64, false, true>(a, s);
        default: break;
        }
        set_error("rank %d not built (16, 32 or 64)", R);
        return FLYCOO_ERR_UNSUPPORTED;
    }
    switch (R) {
    case 16: return bf ? launch_fused_t<N, 16, true>(a, s) : launch_fused_t<N, 16, false>(a, s);
    case 32: return bf ? launch_fused_t<N, 32, true>(a, s) : launch_fused_t<N, 32, false>(a, s);
    case 64: return bf ? launch_fused_t<N, 64, true>(a, s) : launch_fused_t<N, 64, false>(a, s);
    case 128:
        if constexpr (N == 3) return bf ? launch_fused_t<N, 128, true>(a, s) : launch_fused_t<N, 128, false>(a, s);
        break;
    default: break;
    }
    set_error("rank %d not built for %d modes", R, N);
    return FLYCOO_ERR_UNSUPPORTED;
}

} // namespace flycoo
