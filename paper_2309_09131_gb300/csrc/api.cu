// api.cu -- the C ABI of include/flycoo.h: argument checks, the host-side
// FLYCOO bookkeeping (Section III-A pointers, Algorithm 3 schedules, tile
// descriptors, the K4 work list) and the dispatch of the kernels.
#include "fused.cuh"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <functional>
#include <memory>
#include <new>
#include <numeric>
#include <queue>
#include <stdexcept>

namespace flycoo {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

u64 Tensor::device_bytes() const {
    u64 b = elem[0].bytes + elem[1].bytes + orig.bytes + partials.bytes + err.bytes + loss_part.bytes + als.bytes() +
            host_factors.bytes + host_outs.bytes;
    for (int n = 0; n < N; ++n) {
        const ModeMeta &m = mode[n];
        b += m.d_ss_seg_ptr.bytes + m.d_k4.bytes + m.d_next.bytes + m.d_perm[0].bytes + m.d_perm[1].bytes +
             m.d_tiles[0].bytes + m.d_tiles[1].bytes + m.d_tile_bin_ptr[0].bytes + m.d_tile_bin_ptr[1].bytes;
    }
    return b;
}

flycoo_status launch_fused(int N, int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s) {
    switch (N) {
    case 3: return launch_fused_n3(R, dt, a, s);
    case 4: return launch_fused_n4(R, dt, a, s);
    case 5: return launch_fused_n5(R, dt, a, s);
    default: break;
    }
    set_error("N = %d not built (3, 4 or 5)", N);
    return FLYCOO_ERR_UNSUPPORTED;
}

// Algorithm 3: items sorted by size, descending (ties: ascending id); each goes
// to the least-loaded bin (ties: lowest bin index).  CSR output, bins in
// assignment order.
static void lpt_schedule(const std::vector<u64> &size, u32 bins, std::vector<u32> &bin_ptr,
                         std::vector<u32> &items) {
    std::vector<u32> order(size.size());
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](u32 a, u32 b) { return size[a] > size[b]; });
    using P = std::pair<u64, u32>;
    std::priority_queue<P, std::vector<P>, std::greater<P>> heap;
    for (u32 b = 0; b < bins; ++b) heap.push({0, b});
    std::vector<u32> bin_of(size.size());
    std::vector<u32> count(bins, 0);
    for (u32 it : order) {
        P top = heap.top();
        heap.pop();
        bin_of[it] = top.second;
        ++count[top.second];
        heap.push({top.first + size[it], top.second});
    }
    bin_ptr.assign(bins + 1, 0);
    for (u32 b = 0; b < bins; ++b) bin_ptr[b + 1] = bin_ptr[b] + count[b];
    items.assign(size.size(), 0);
    std::vector<u32> fill(bin_ptr.begin(), bin_ptr.end() - 1);
    for (u32 it : order) items[fill[bin_of[it]]++] = it;
}

// block-cyclic assignment: item i to bin i mod bins, ascending within a bin
static void block_cyclic_schedule(size_t nitems, u32 bins, std::vector<u32> &bin_ptr, std::vector<u32> &items) {
    bin_ptr.assign(bins + 1, 0);
    for (u32 b = 0; b < bins; ++b) bin_ptr[b + 1] = bin_ptr[b] + (u32)(nitems / bins + (b < nitems % bins ? 1 : 0));
    items.assign(nitems, 0);
    std::vector<u32> fill(bin_ptr.begin(), bin_ptr.end() - 1);
    for (size_t i = 0; i < nitems; ++i) items[fill[i % bins]++] = (u32)i;
}

template <class T>
static flycoo_status upload(DevBuf &d, const std::vector<T> &h, cudaStream_t s) {
    FLY_TRY(d.alloc(std::max<size_t>(h.size() * sizeof(T), 16)));
    if (!h.empty()) FLY_TRY_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return FLYCOO_OK;
}

flycoo_status check_pass_rank(const Tensor &t, int mode, int R, const char *who) {
    if (R == 16 || R == 32 || R == 64) return FLYCOO_OK;
    if (R == kRank128) {
        if (t.N != 3) {
            set_error("%s: rank 128 is built for 3-mode tensors only (this one has %d modes)", who, t.N);
            return FLYCOO_ERR_UNSUPPORTED;
        }
        if (t.mode[mode].m > kMaxRowsAtRank128) {
            set_error("%s: rank 128 needs super-shards of at most %u rows in mode %d (m = %llu); create the "
                      "handle with flycoo_params.m[%d] <= %u",
                      who, kMaxRowsAtRank128, mode, (unsigned long long)t.mode[mode].m, mode, kMaxRowsAtRank128);
            return FLYCOO_ERR_UNSUPPORTED;
        }
        return FLYCOO_OK;
    }
    set_error("%s: rank %d not built (16, 32, 64, or 128 on 3-mode tensors)", who, R);
    return R > 0 ? FLYCOO_ERR_UNSUPPORTED : FLYCOO_ERR_INVALID_ARG;
}

long long g_alloc_fail_after = -1;

// runs an entry point's body; a failed host allocation becomes FLYCOO_ERR_OOM
// instead of an exception crossing the C ABI
template <class F> static flycoo_status host_guarded(const char *who, F &&body) {
    try {
        return body();
    } catch (const std::bad_alloc &) {
        set_error("%s: a host allocation failed", who);
        return FLYCOO_ERR_OOM;
    } catch (const std::exception &e) {
        set_error("%s: %s", who, e.what());
        return FLYCOO_ERR_CUDA;
    }
}

// a handle whose remapping pass gave up has an undefined layout
flycoo_status check_usable(const Tensor &t, const char *who) {
    if (t.poisoned) {
        set_error("%s: a remapping pass on this handle gave up (FLYCOO_ERR_TIMEOUT), so its layout is "
                  "undefined; destroy the handle and create it again", who);
        return FLYCOO_ERR_LAYOUT;
    }
    return FLYCOO_OK;
}

// reads and clears the device error word (waits for the stream); TIMEOUT if a
// bounded device wait gave up since the last check
flycoo_status check_error_word(Tensor &t, cudaStream_t s, const char *who) {
    u32 e = 0;
    FLY_TRY_CUDA(cudaMemcpyAsync(&e, t.err.p, sizeof(u32), cudaMemcpyDeviceToHost, s));
    FLY_TRY_CUDA(cudaStreamSynchronize(s));
    const bool remapped = t.remap_since_sync;
    t.remap_since_sync = false;
    if (e) {
        FLY_TRY_CUDA(cudaMemsetAsync(t.err.p, 0, sizeof(u32), s));
        FLY_TRY_CUDA(cudaStreamSynchronize(s));
        if (remapped) t.poisoned = true;
        set_error("%s: a bounded device wait gave up (error word 0x%x)%s", who, e,
                  remapped ? "; a remapping pass was among the failed work, so the handle's layout is undefined"
                           : "");
        return FLYCOO_ERR_TIMEOUT;
    }
    return FLYCOO_OK;
}

// Default super-shard width: kDefaultSuperShardRows (32) when the modes have
// at most 2^18 rows together (factor matrices that stay in L2), else 64 rows.
// On a 12,000 x 9,000 x 29,000 tensor with 77M nonzeros at R = 32, 32 rows were
// faster than 16, 24, 40, 48, 64 or 128; on tensors with hundreds of thousands
// to millions of rows per mode (4.8M x 1.8M x 1.8M, 1.2M x 1.2M x 50K x 10K,
// 20K x 200K x 500K) 64 rows were faster than 32.
constexpr u32 kWideSuperShardRows = 64;
constexpr u64 kNarrowMaxTotalRows = u64(1) << 18;

// Default shard size: the largest power of two in [1024, 32768] that gives
// every bin at least 16 shards (whole 1024-nonzero stage tiles from 1024 up).
// Fewer, larger shards leave the last whole shard of a bin dominating its load
// (on a 77M-nonzero 3-mode tensor, 8 per bin put the heaviest bin 4-7% above
// the mean, 16 per bin 2%, and the pass ran 1.3% faster); many smaller ones add
// row-block flushes and fixup work.
u64 default_shard_size(u64 nnz, u32 bins) {
    u64 g = 32768;
    while (g > 1024 && nnz / g < 16ull * bins) g >>= 1;
    return g;
}

// Section III-A: super-shard j is cut into runs of g consecutive nonzeros
// (shards); Algorithm 3 (or block-cyclic) schedules the super-shards by shard
// count and the shards by nonzero count.  The shard schedule is then written
// out as tile descriptors for both stage-tile sizes, with the shards of a bin
// grouped into segments (runs of shards of one super-shard that follow each
// other in the bin: a block keeps accumulating across them).
void plan_mode(ModePlan &md, u64 nnz, u64 g, u32 bins, u32 schedule) {
    md.shard_ptr.clear();
    md.shard_ss.clear();
    md.ss_shard_ptr.assign(md.k + 1, 0);
    std::vector<u64> ss_shards(md.k);
    for (u64 j = 0; j < md.k; ++j) {
        const u64 size = md.ss_ptr[j + 1] - md.ss_ptr[j];
        ss_shards[j] = (size + g - 1) / g;
        md.ss_shard_ptr[j] = (u32)md.shard_ptr.size();
        for (u64 q = 0; q * g < size; ++q) {
            md.shard_ptr.push_back((u32)(md.ss_ptr[j] + q * g));
            md.shard_ss.push_back((u32)j);
        }
    }
    md.S = md.shard_ptr.size();
    md.ss_shard_ptr[md.k] = (u32)md.S;
    md.shard_ptr.push_back((u32)nnz);
    std::vector<u64> shard_size(md.S);
    for (int z = 0; z < 2; ++z) md.tile_ptr[z].clear();
    for (u64 q = 0; q < md.S; ++q) {
        shard_size[q] = md.shard_ptr[q + 1] - md.shard_ptr[q];
        for (int z = 0; z < 2; ++z)
            for (u64 p = md.shard_ptr[q]; p < md.shard_ptr[q + 1]; p += kStageTile[z])
                md.tile_ptr[z].push_back((u32)p);
    }
    for (int z = 0; z < 2; ++z) md.tile_ptr[z].push_back((u32)nnz);
    if (schedule == FLYCOO_SCHEDULE_BLOCK_CYCLIC) {
        block_cyclic_schedule(ss_shards.size(), bins, md.ss_bin_ptr, md.ss_items);
        block_cyclic_schedule(shard_size.size(), bins, md.sh_bin_ptr, md.sh_items);
    } else {
        lpt_schedule(ss_shards, bins, md.ss_bin_ptr, md.ss_items);
        lpt_schedule(shard_size, bins, md.sh_bin_ptr, md.sh_items);
    }
    // segments in schedule order (bin by bin), then numbered so that the
    // segments of each super-shard are consecutive, in schedule order
    std::vector<u32> seg_of_item(md.S), seg_first; // temporary numbering
    std::vector<u32> tmp_ss;
    for (u32 b = 0; b < bins; ++b)
        for (u64 it = md.sh_bin_ptr[b]; it < md.sh_bin_ptr[b + 1]; ++it) {
            const u32 j = md.shard_ss[md.sh_items[it]];
            if (it == md.sh_bin_ptr[b] || md.shard_ss[md.sh_items[it - 1]] != j) tmp_ss.push_back(j);
            seg_of_item[it] = (u32)tmp_ss.size() - 1;
        }
    md.ss_seg_ptr.assign(md.k + 1, 0);
    for (u32 j : tmp_ss) ++md.ss_seg_ptr[j + 1];
    for (u64 j = 0; j < md.k; ++j) md.ss_seg_ptr[j + 1] += md.ss_seg_ptr[j];
    std::vector<u32> renum(tmp_ss.size());
    {
        std::vector<u32> fill(md.ss_seg_ptr.begin(), md.ss_seg_ptr.end() - 1);
        for (size_t q = 0; q < tmp_ss.size(); ++q) renum[q] = fill[tmp_ss[q]]++;
    }
    md.seg_ss.assign(tmp_ss.size(), 0);
    for (size_t q = 0; q < tmp_ss.size(); ++q) md.seg_ss[renum[q]] = tmp_ss[q];
    // tile descriptors of the block schedule, for both stage-tile sizes
    for (int z = 0; z < 2; ++z) {
        const u32 tile = kStageTile[z];
        std::vector<u32> &td = md.tiles[z];
        td.clear();
        md.tile_bin_ptr[z].assign((size_t)bins + 1, 0);
        for (u32 b = 0; b < bins; ++b) {
            md.tile_bin_ptr[z][b] = (u32)(td.size() / 4);
            const u64 i0 = md.sh_bin_ptr[b], i1 = md.sh_bin_ptr[b + 1];
            for (u64 it = i0; it < i1; ++it) {
                const u32 sh = md.sh_items[it];
                const u32 j = md.shard_ss[sh];
                const u32 seg = renum[seg_of_item[it]];
                const bool seg_begin = it == i0 || seg_of_item[it - 1] != seg_of_item[it];
                const bool seg_end = it + 1 == i1 || seg_of_item[it + 1] != seg_of_item[it];
                const u32 lo = md.shard_ptr[sh], hi = md.shard_ptr[sh + 1];
                const u32 alone = md.ss_seg_ptr[j + 1] - md.ss_seg_ptr[j] == 1 ? 4u : 0u;
                for (u32 p = lo; p < hi; p += tile) {
                    const u32 len = std::min<u32>(tile, hi - p);
                    const u32 flags = (seg_begin && p == lo ? 1u : 0u) | (seg_end && p + len == hi ? 2u : 0u) | alone;
                    td.insert(td.end(), {p, len | (flags << 16), j, seg});
                }
            }
        }
        md.tile_bin_ptr[z][bins] = (u32)(td.size() / 4);
    }
    // K4 writes the rows of every super-shard that does not have exactly one segment
    md.k4_items.clear();
    for (u64 j = 0; j < md.k; ++j)
        if (md.ss_seg_ptr[j + 1] - md.ss_seg_ptr[j] != 1) md.k4_items.push_back((u32)j);
    md.k4_order.clear();
    for (u32 j : md.k4_items)
        if (md.ss_seg_ptr[j + 1] - md.ss_seg_ptr[j] <= kFixupLightSegs) md.k4_order.push_back(j);
    md.k4_nlight = (u32)md.k4_order.size();
    for (u32 j : md.k4_items)
        if (md.ss_seg_ptr[j + 1] - md.ss_seg_ptr[j] > kFixupLightSegs) md.k4_order.push_back(j);
}

flycoo_status partition_mode(Tensor &t, int n, const std::vector<u32> &ssp, cudaStream_t s) {
    ModeMeta &md = t.mode[n];
    const u64 I = t.dims[n];
    md.I = I;
    md.k = (I + md.m - 1) / md.m;
    md.ss_ptr.assign(ssp.begin(), ssp.end());
    plan_mode(md, t.nnz, t.g, t.bins, t.schedule);
    FLY_TRY(upload(md.d_ss_seg_ptr, md.ss_seg_ptr, s));
    FLY_TRY(upload(md.d_k4, md.k4_order, s));
    for (int z = 0; z < 2; ++z) {
        FLY_TRY(upload(md.d_tiles[z], md.tiles[z], s));
        FLY_TRY(upload(md.d_tile_bin_ptr[z], md.tile_bin_ptr[z], s));
    }
    return FLYCOO_OK;
}

flycoo_status launch_fixup(int R, const FixupArgs &a, cudaStream_t s) {
    if (a.nitems == 0) return FLYCOO_OK;
    // one block per light item, one per 64 floats of a row block per other item
    const u32 chunks = (a.m * (u32)R + 63) / 64;
    const u32 grid = a.nlight + (a.nitems - a.nlight) * chunks;
    super_shard_fixup_kernel<<<grid, 256, 0, s>>>(a, (u32)R);
    FLY_TRY_CUDA(cudaGetLastError());
    return FLYCOO_OK;
}

FusedArgs fused_args(const Tensor &t, int mode, const void *const *F, float *d_out, bool remap, float *partials) {
    const ModeMeta &md = t.mode[mode];
    FusedArgs a{};
    a.elem_in = t.elem[t.cur].p;
    a.elem_out = remap ? t.elem[1 - t.cur].p : nullptr;
    a.next = remap ? md.d_next.as<u32>() : nullptr;
    for (int q = 1; q < t.N; ++q) a.Y[q - 1] = F[(mode + q) % t.N];
    a.out = d_out;
    for (int z = 0; z < 2; ++z) {
        a.tiles[z] = md.d_tiles[z].as<uint4>();
        a.tile_bin_ptr[z] = md.d_tile_bin_ptr[z].as<u32>();
        a.perm[z] = md.d_perm[z].as<uint16_t>();
    }
    a.partials = partials;
    a.err = t.err.as<u32>();
    a.I_out = (u32)t.dims[mode];
    a.m = (u32)md.m;
    a.bins = t.bins;
    a.wait_limit = t.wait_limit;
    return a;
}

FixupArgs fixup_args(const Tensor &t, int mode, float *d_out, const float *partials) {
    const ModeMeta &md = t.mode[mode];
    FixupArgs f{};
    f.items = md.d_k4.as<u32>();
    f.nitems = (u32)md.k4_order.size();
    f.nlight = md.k4_nlight;
    f.ss_seg_ptr = md.d_ss_seg_ptr.as<u32>();
    f.partials = partials;
    f.out = d_out;
    f.I_out = (u32)t.dims[mode];
    f.m = (u32)md.m;
    return f;
}

} // namespace flycoo

using namespace flycoo;

// --------------------------------------------------------------------------
// the C ABI
// --------------------------------------------------------------------------
extern "C" const char *flycoo_last_error(void) { return g_last_error.c_str(); }

static flycoo_status create_impl(int N, const uint64_t *h_dims, uint64_t nnz, const uint32_t *d_idx,
                                 const float *d_vals, const flycoo_params *params, flycoo_stream_t stream,
                                 flycoo_handle *out) {
    if (!out) {
        set_error("flycoo_create: out is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (N < 1 || N > FLYCOO_MAX_MODES || !h_dims) {
        set_error("flycoo_create: N must be in [1, %d] with dims given", FLYCOO_MAX_MODES);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (N < 3 || N > 5) {
        set_error("flycoo_create: N = %d not built (3, 4 or 5)", N);
        return FLYCOO_ERR_UNSUPPORTED;
    }
    for (int w = 0; w < N; ++w)
        if (h_dims[w] == 0 || h_dims[w] > 0xffffffffull) {
            set_error("flycoo_create: dims[%d] = %llu outside [1, 2^32-1]", w, (unsigned long long)h_dims[w]);
            return FLYCOO_ERR_INVALID_ARG;
        }
    if (nnz >= 0xffffffffull) {
        set_error("flycoo_create: nnz must be < 2^32 - 1");
        return FLYCOO_ERR_UNSUPPORTED;
    }
    if (nnz && (!d_idx || !d_vals)) {
        set_error("flycoo_create: d_idx / d_vals is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto t = std::make_unique<flycoo_tensor>();
    FLY_TRY_CUDA(cudaGetDevice(&t->device));
    FLY_TRY_CUDA(cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, t->device));
    t->N = N;
    t->nnz = nnz;
    for (int w = 0; w < N; ++w) t->dims[w] = h_dims[w];
    t->bins = (params && params->bins) ? params->bins : (u32)(kBlocksPerSM * t->sm_count);
    if (t->bins > kMaxBins) {
        set_error("flycoo_create: bins = %u exceeds %u", t->bins, kMaxBins);
        return FLYCOO_ERR_INVALID_ARG;
    }
    t->wait_limit = kSpinLimit;
    t->schedule = params ? params->schedule : FLYCOO_SCHEDULE_LPT;
    if (t->schedule != FLYCOO_SCHEDULE_LPT && t->schedule != FLYCOO_SCHEDULE_BLOCK_CYCLIC) {
        set_error("flycoo_create: unknown schedule %u", t->schedule);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (params && params->reserved != 0) {
        set_error("flycoo_create: flycoo_params.reserved must be 0");
        return FLYCOO_ERR_INVALID_ARG;
    }
    t->order = params ? params->order : FLYCOO_ORDER_KEY;
    if (t->order != FLYCOO_ORDER_KEY && t->order != FLYCOO_ORDER_MORTON) {
        set_error("flycoo_create: unknown order %u", t->order);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (params && params->g) {
        t->g = params->g;
    } else {
        t->g = default_shard_size(nnz, t->bins);
    }
    if (t->g > 0xffffffffull) {
        set_error("flycoo_create: g too large");
        return FLYCOO_ERR_INVALID_ARG;
    }
    u64 total_rows = 0;
    for (int w = 0; w < N; ++w) total_rows += h_dims[w];
    const u64 m_default = std::min<u64>(total_rows <= kNarrowMaxTotalRows ? kDefaultSuperShardRows : kWideSuperShardRows,
                                        kMaxSuperShardRows);
    for (int w = 0; w < N; ++w) {
        // a super-shard's output rows live in shared memory: at most kMaxSuperShardRows
        u64 m = (params && params->m[w]) ? params->m[w] : std::min<u64>(h_dims[w], m_default);
        if (m > kMaxSuperShardRows) {
            set_error("flycoo_create: m[%d] = %llu exceeds %u rows", w, (unsigned long long)m, kMaxSuperShardRows);
            return FLYCOO_ERR_INVALID_ARG;
        }
        t->mode[w].m = std::max<u64>(m, 1);
        t->max_rows = std::max<u64>(t->max_rows, t->mode[w].m);
    }
    t->elem_words = elem_words_for(N);

    std::vector<std::vector<u32>> ss_ptr;
    FLY_TRY(build_flycoo(*t, d_idx, d_vals, ss_ptr, s));
    for (int n = 0; n < N; ++n) t->max_seg = std::max<u64>(t->max_seg, t->mode[n].nseg());
    // one row block per segment, large enough for m x R at every rank the pass is
    // built for (R <= 64 with m <= 128, R = 128 with m <= 64)
    const u64 block = std::max<u64>(t->max_rows * kMaxRank, std::min<u64>(t->max_rows, kMaxRowsAtRank128) * kRank128);
    FLY_TRY(t->partials.alloc(std::max<u64>(t->max_seg, 1) * block * sizeof(float)));
    FLY_TRY(t->loss_part.alloc((size_t)t->bins * sizeof(double)));
    FLY_TRY(t->err.alloc(sizeof(u32)));
    FLY_TRY_CUDA(cudaMemsetAsync(t->err.p, 0, sizeof(u32), s));
    FLY_TRY_CUDA(cudaStreamSynchronize(s));
    *out = t.release();
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_create(int N, const uint64_t *h_dims, uint64_t nnz, const uint32_t *d_idx,
                                       const float *d_vals, const flycoo_params *params,
                                       flycoo_stream_t stream, flycoo_handle *out) {
    clear_error();
    return host_guarded("flycoo_create",
                        [&] { return create_impl(N, h_dims, nnz, d_idx, d_vals, params, stream, out); });
}

extern "C" void flycoo_destroy(flycoo_handle h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    delete h;
}

// two events of the pool for one timed launch; also reserves the pending
// entry, so nothing is allocated once the launch is enqueued
static flycoo_status next_event_pair(Tensor &t, cudaEvent_t *a, cudaEvent_t *b) {
    FLY_TRY(host_guarded("flycoo timing", [&] {
        t.ev_pool.reserve(t.ev_used + 2);
        t.ev_pending.reserve(t.ev_pending.size() + 1);
        return FLYCOO_OK;
    }));
    while (t.ev_pool.size() < t.ev_used + 2) {
        cudaEvent_t e;
        FLY_TRY_CUDA(cudaEventCreate(&e));
        t.ev_pool.push_back(e);
    }
    *a = t.ev_pool[t.ev_used++];
    *b = t.ev_pool[t.ev_used++];
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_spmttkrp(flycoo_handle h, int mode, const void *const *h_factors,
                                         flycoo_dtype fdt, int R, float *d_out, int next_mode,
                                         flycoo_stream_t stream) {
    clear_error();
    if (!h) {
        set_error("flycoo_spmttkrp: handle is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    Tensor &t = *h;
    if (mode < 0 || mode >= t.N) {
        set_error("flycoo_spmttkrp: mode %d outside [0, %d)", mode, t.N);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (fdt != FLYCOO_F32 && fdt != FLYCOO_BF16) {
        set_error("flycoo_spmttkrp: unknown factor dtype %d", (int)fdt);
        return FLYCOO_ERR_INVALID_ARG;
    }
    FLY_TRY(check_pass_rank(t, mode, R, "flycoo_spmttkrp"));
    if (next_mode != -1 && next_mode != (mode + 1) % t.N) {
        set_error("flycoo_spmttkrp: next_mode must be -1 or (mode+1) mod N = %d", (mode + 1) % t.N);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15u)) {
        set_error("flycoo_spmttkrp: d_out is NULL or not 16-byte aligned");
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (!h_factors) {
        set_error("flycoo_spmttkrp: h_factors is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    for (int w = 0; w < t.N; ++w) {
        if (w == mode) continue;
        if (!h_factors[w] || (reinterpret_cast<uintptr_t>(h_factors[w]) & 15u)) {
            set_error("flycoo_spmttkrp: factor %d is NULL or not 16-byte aligned", w);
            return FLYCOO_ERR_INVALID_ARG;
        }
    }
    if (t.layout != mode) {
        set_error("flycoo_spmttkrp: tensor is in layout L_%d, mode %d needs L_%d", t.layout, mode, mode);
        return FLYCOO_ERR_LAYOUT;
    }
    DeviceGuard dg(t.device);
    FLY_TRY(dg.status(__func__));
    FLY_TRY(check_usable(t, "flycoo_spmttkrp"));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (t.nnz == 0) {
        FLY_TRY_CUDA(cudaMemsetAsync(d_out, 0, (size_t)t.dims[mode] * R * sizeof(float), s));
        if (next_mode >= 0) t.layout = next_mode;
        return FLYCOO_OK;
    }
    const FusedArgs a = fused_args(t, mode, h_factors, d_out, next_mode >= 0, t.partials.as<float>());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (t.timing) {
        FLY_TRY(next_event_pair(t, &e0, &e1));
        FLY_TRY_CUDA(cudaEventRecord(e0, s));
    }
    FLY_TRY(launch_fused(t.N, R, fdt, a, s));
    if (t.timing) {
        FLY_TRY_CUDA(cudaEventRecord(e1, s));
        t.ev_pending.push_back({e0, e1});
    }
    const FixupArgs f = fixup_args(t, mode, d_out, a.partials);
    FLY_TRY(launch_fixup(R, f, s));
    if (next_mode >= 0) {
        t.cur = 1 - t.cur;
        t.remap_since_sync = true;
        t.layout = next_mode;
    }
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_all_modes_host(flycoo_handle h, const void *const *h_factors, flycoo_dtype fdt, int R,
                                               float *const *h_out, flycoo_stream_t stream) {
    clear_error();
    if (!h || !h_factors || !h_out) {
        set_error("flycoo_all_modes_host: NULL handle, factor list or output list");
        return FLYCOO_ERR_INVALID_ARG;
    }
    Tensor &t = *h;
    if (fdt != FLYCOO_F32 && fdt != FLYCOO_BF16) {
        set_error("flycoo_all_modes_host: unknown factor dtype %d", (int)fdt);
        return FLYCOO_ERR_INVALID_ARG;
    }
    for (int n = 0; n < t.N; ++n) FLY_TRY(check_pass_rank(t, n, R, "flycoo_all_modes_host"));
    for (int w = 0; w < t.N; ++w)
        if (!h_factors[w] || !h_out[w]) {
            set_error("flycoo_all_modes_host: factor or output %d is NULL", w);
            return FLYCOO_ERR_INVALID_ARG;
        }
    DeviceGuard dg(t.device);
    FLY_TRY(dg.status("flycoo_all_modes_host"));
    FLY_TRY(check_usable(t, "flycoo_all_modes_host"));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t fb = fdt == FLYCOO_BF16 ? 2 : 4;
    // per-mode offsets, each rounded up to 256 bytes
    size_t foff[FLYCOO_MAX_MODES + 1] = {}, ooff[FLYCOO_MAX_MODES + 1] = {};
    for (int w = 0; w < t.N; ++w) {
        foff[w + 1] = foff[w] + ((t.dims[w] * R * fb + 255) & ~(size_t)255);
        ooff[w + 1] = ooff[w] + ((t.dims[w] * R * 4 + 255) & ~(size_t)255);
    }
    if (t.host_factors.bytes < foff[t.N]) FLY_TRY(t.host_factors.alloc(foff[t.N]));
    if (t.host_outs.bytes < ooff[t.N]) FLY_TRY(t.host_outs.alloc(ooff[t.N]));
    const void *F[FLYCOO_MAX_MODES] = {};
    for (int w = 0; w < t.N; ++w) {
        void *d = static_cast<char *>(t.host_factors.p) + foff[w];
        FLY_TRY_CUDA(cudaMemcpyAsync(d, h_factors[w], t.dims[w] * R * fb, cudaMemcpyHostToDevice, s));
        F[w] = d;
    }
    while (t.layout != 0) {
        FLY_TRY(launch_remap_step(t, t.layout, t.elem[t.cur].p, t.elem[1 - t.cur].p, s));
        t.cur = 1 - t.cur;
        t.remap_since_sync = true;
        t.layout = (t.layout + 1) % t.N;
    }
    for (int n = 0; n < t.N; ++n) {
        float *d_out = reinterpret_cast<float *>(static_cast<char *>(t.host_outs.p) + ooff[n]);
        FLY_TRY(run_pass(t, n, F, fdt, R, d_out, nullptr, nullptr, s));
        FLY_TRY_CUDA(cudaMemcpyAsync(h_out[n], d_out, t.dims[n] * R * 4, cudaMemcpyDeviceToHost, s));
    }
    return check_error_word(t, s, "flycoo_all_modes_host");
}

extern "C" flycoo_status flycoo_sync(flycoo_handle h, flycoo_stream_t stream) {
    clear_error();
    if (!h) {
        set_error("flycoo_sync: handle is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->device);
    FLY_TRY(dg.status(__func__));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return check_error_word(*h, s, "flycoo_sync");
}

// One fused pass of mode `mode` in its layout: spMTTKRP (Yout == nullptr) or the
// CP-OPT gradient pass; fused remap to the next layout; then K4.
flycoo_status flycoo::run_pass(Tensor &t, int mode, const void *const *F, flycoo_dtype fdt, int R, float *d_out,
                               const void *Yout, double *loss_part, cudaStream_t s) {
    if (t.nnz == 0) {
        FLY_TRY_CUDA(cudaMemsetAsync(d_out, 0, (size_t)t.dims[mode] * R * sizeof(float), s));
        t.layout = (mode + 1) % t.N;
        return FLYCOO_OK;
    }
    FusedArgs a = fused_args(t, mode, F, d_out, true, t.partials.as<float>());
    a.Yout = Yout;
    a.loss_part = loss_part;
    FLY_TRY(launch_fused(t.N, R, fdt, a, s));
    const FixupArgs f = fixup_args(t, mode, d_out, a.partials);
    FLY_TRY(launch_fixup(R, f, s));
    t.cur = 1 - t.cur;
    t.remap_since_sync = true;
    t.layout = (mode + 1) % t.N;
    return FLYCOO_OK;
}

static flycoo_status check_factor_ptrs(const Tensor &t, const void *const *F, int skip, int R, const char *who) {
    if (R != 16 && R != 32 && R != 64) {
        set_error("%s: rank %d not built (16, 32 or 64)", who, R);
        return R > 0 ? FLYCOO_ERR_UNSUPPORTED : FLYCOO_ERR_INVALID_ARG;
    }
    if (!F) {
        set_error("%s: factor array is NULL", who);
        return FLYCOO_ERR_INVALID_ARG;
    }
    for (int w = 0; w < t.N; ++w) {
        if (w == skip) continue;
        if (!F[w] || (reinterpret_cast<uintptr_t>(F[w]) & 15u)) {
            set_error("%s: factor %d is NULL or not 16-byte aligned", who, w);
            return FLYCOO_ERR_INVALID_ARG;
        }
    }
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_mttkrp_adjoint(flycoo_handle h, int mode, const void *const *h_factors,
                                               flycoo_dtype fdt, int R, const void *d_gout,
                                               float *const *h_gfactors, float *d_gvals, flycoo_stream_t stream) {
    clear_error();
    if (!h || mode < 0 || mode >= h->N) {
        set_error("flycoo_mttkrp_adjoint: bad handle or mode");
        return FLYCOO_ERR_INVALID_ARG;
    }
    Tensor &t = *h;
    if (fdt != FLYCOO_F32 && fdt != FLYCOO_BF16) {
        set_error("flycoo_mttkrp_adjoint: unknown factor dtype %d", (int)fdt);
        return FLYCOO_ERR_INVALID_ARG;
    }
    FLY_TRY(check_factor_ptrs(t, h_factors, mode, R, "flycoo_mttkrp_adjoint"));
    if (!d_gout || (reinterpret_cast<uintptr_t>(d_gout) & 15u) || !h_gfactors) {
        set_error("flycoo_mttkrp_adjoint: d_gout / h_gfactors NULL or d_gout not 16-byte aligned");
        return FLYCOO_ERR_INVALID_ARG;
    }
    for (int w = 0; w < t.N; ++w)
        if (w != mode && h_gfactors[w] && (reinterpret_cast<uintptr_t>(h_gfactors[w]) & 15u)) {
            set_error("flycoo_mttkrp_adjoint: gradient %d not 16-byte aligned", w);
            return FLYCOO_ERR_INVALID_ARG;
        }
    DeviceGuard dg(t.device);
    FLY_TRY(dg.status("flycoo_mttkrp_adjoint"));
    FLY_TRY(check_usable(t, "flycoo_mttkrp_adjoint"));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the factor list of every pass: Y_w, with the output mode's slot holding G
    const void *F[FLYCOO_MAX_MODES] = {};
    for (int w = 0; w < t.N; ++w) F[w] = (w == mode) ? d_gout : h_factors[w];
    // the value gradient runs when the walk below passes through L_0 (every
    // layout is visited: from L_{mode+1} around to L_mode)
    bool vals_done = d_gvals == nullptr;
    auto value_grad_if_l0 = [&]() -> flycoo_status {
        if (!vals_done && t.layout == 0) {
            FLY_TRY(launch_value_grad(t, mode, h_factors, d_gout, fdt, R, d_gvals, s));
            vals_done = true;
        }
        return FLYCOO_OK;
    };
    auto remap_one = [&]() -> flycoo_status {
        FLY_TRY(launch_remap_step(t, t.layout, t.elem[t.cur].p, t.elem[1 - t.cur].p, s));
        t.cur = 1 - t.cur;
        t.remap_since_sync = true;
        t.layout = (t.layout + 1) % t.N;
        return FLYCOO_OK;
    };
    FLY_TRY(value_grad_if_l0());
    const int first = (mode + 1) % t.N;
    while (t.layout != first) {
        FLY_TRY(remap_one());
        FLY_TRY(value_grad_if_l0());
    }
    for (int q = 1; q < t.N; ++q) {
        const int w = (mode + q) % t.N;
        if (h_gfactors[w]) {
            FLY_TRY(run_pass(t, w, F, fdt, R, h_gfactors[w], nullptr, nullptr, s));
        } else {
            FLY_TRY(remap_one());
        }
        FLY_TRY(value_grad_if_l0());
    }
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_cpopt_grad(flycoo_handle h, const float *const *h_factors, int R,
                                           float *const *h_grads, double *h_loss, flycoo_stream_t stream) {
    clear_error();
    if (!h) {
        set_error("flycoo_cpopt_grad: handle is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    Tensor &t = *h;
    FLY_TRY(check_factor_ptrs(t, reinterpret_cast<const void *const *>(h_factors), -1, R, "flycoo_cpopt_grad"));
    if (!h_grads) {
        set_error("flycoo_cpopt_grad: h_grads is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    for (int w = 0; w < t.N; ++w)
        if (!h_grads[w] || (reinterpret_cast<uintptr_t>(h_grads[w]) & 15u)) {
            set_error("flycoo_cpopt_grad: gradient %d is NULL or not 16-byte aligned", w);
            return FLYCOO_ERR_INVALID_ARG;
        }
    DeviceGuard dg(t.device);
    FLY_TRY(dg.status(__func__));
    FLY_TRY(check_usable(t, "flycoo_cpopt_grad"));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const void *const *F = reinterpret_cast<const void *const *>(h_factors);
    double *lp = t.loss_part.as<double>();
    std::vector<double> part; // per-block loss partials, allocated before any work is enqueued
    if (h_loss) FLY_TRY(host_guarded("flycoo_cpopt_grad", [&] {
        part.assign(t.bins, 0.0);
        return FLYCOO_OK;
    }));
    if (t.nnz) FLY_TRY_CUDA(cudaMemsetAsync(lp, 0, (size_t)t.bins * sizeof(double), s));
    const int start = t.layout;
    for (int q = 0; q < t.N; ++q) {
        const int n = (start + q) % t.N;
        FLY_TRY(run_pass(t, n, F, FLYCOO_F32, R, h_grads[n], F[n], q == 0 ? lp : nullptr, s));
    }
    if (h_loss) {
        if (t.nnz)
            FLY_TRY_CUDA(cudaMemcpyAsync(part.data(), lp, (size_t)t.bins * sizeof(double), cudaMemcpyDeviceToHost, s));
        FLY_TRY(check_error_word(t, s, "flycoo_cpopt_grad"));
        double L = 0.0;
        for (double x : part) L += x; // fixed order
        *h_loss = L;
    }
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_cp_als_step(flycoo_handle h, void *const *h_factors, flycoo_dtype fdt, int R,
                                            double *d_lambda, double *h_fit, flycoo_stream_t stream) {
    clear_error();
    if (!h) {
        set_error("flycoo_cp_als_step: handle is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    Tensor &t = *h;
    if (fdt != FLYCOO_F32 && fdt != FLYCOO_BF16) {
        set_error("flycoo_cp_als_step: unknown factor dtype %d", (int)fdt);
        return FLYCOO_ERR_INVALID_ARG;
    }
    FLY_TRY(check_factor_ptrs(t, reinterpret_cast<const void *const *>(h_factors), -1, R, "flycoo_cp_als_step"));
    if (!d_lambda) {
        set_error("flycoo_cp_als_step: d_lambda is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    DeviceGuard dg(t.device);
    FLY_TRY(dg.status(__func__));
    FLY_TRY(check_usable(t, "flycoo_cp_als_step"));
    return als_step(t, h_factors, fdt, R, 1, d_lambda, h_fit, reinterpret_cast<cudaStream_t>(stream),
                    "flycoo_cp_als_step");
}

extern "C" flycoo_status flycoo_cp_als(flycoo_handle h, void *const *h_factors, flycoo_dtype fdt, int R, int iters,
                                       double *d_lambda, double *h_fits, flycoo_stream_t stream) {
    clear_error();
    if (!h) {
        set_error("flycoo_cp_als: handle is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    Tensor &t = *h;
    if (fdt != FLYCOO_F32 && fdt != FLYCOO_BF16) {
        set_error("flycoo_cp_als: unknown factor dtype %d", (int)fdt);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (iters < 1 || iters > 1000000) {
        set_error("flycoo_cp_als: iters = %d outside [1, 10^6]", iters);
        return FLYCOO_ERR_INVALID_ARG;
    }
    FLY_TRY(check_factor_ptrs(t, reinterpret_cast<const void *const *>(h_factors), -1, R, "flycoo_cp_als"));
    if (!d_lambda) {
        set_error("flycoo_cp_als: d_lambda is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    DeviceGuard dg(t.device);
    FLY_TRY(dg.status("flycoo_cp_als"));
    FLY_TRY(check_usable(t, "flycoo_cp_als"));
    return als_step(t, h_factors, fdt, R, iters, d_lambda, h_fits, reinterpret_cast<cudaStream_t>(stream),
                    "flycoo_cp_als");
}

extern "C" flycoo_status flycoo_remap(flycoo_handle h, int next_mode, flycoo_stream_t stream) {
    clear_error();
    if (!h || next_mode < 0 || next_mode >= h->N) {
        set_error("flycoo_remap: bad handle or next_mode");
        return FLYCOO_ERR_INVALID_ARG;
    }
    Tensor &t = *h;
    DeviceGuard dg(t.device);
    FLY_TRY(dg.status(__func__));
    FLY_TRY(check_usable(t, "flycoo_remap"));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    while (t.layout != next_mode) {
        FLY_TRY(launch_remap_step(t, t.layout, t.elem[t.cur].p, t.elem[1 - t.cur].p, s));
        t.cur = 1 - t.cur;
        t.remap_since_sync = true;
        t.layout = (t.layout + 1) % t.N;
    }
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_get_info(flycoo_handle h, flycoo_info *out) {
    clear_error();
    if (!h || !out) {
        set_error("flycoo_get_info: NULL argument");
        return FLYCOO_ERR_INVALID_ARG;
    }
    const Tensor &t = *h;
    std::memset(out, 0, sizeof *out);
    out->N = t.N;
    out->layout_mode = t.layout;
    out->nnz = t.nnz;
    out->g = t.g;
    out->bins = t.bins;
    out->elem_bytes = (uint32_t)(t.elem_words * 4);
    out->schedule = t.schedule;
    out->order = t.order;
    for (int n = 0; n < t.N; ++n) {
        out->dims[n] = t.dims[n];
        out->m[n] = t.mode[n].m;
        out->super_shards[n] = t.mode[n].k;
        out->shards[n] = t.mode[n].S;
        out->segments[n] = t.mode[n].nseg();
        out->fixup_super_shards[n] = t.mode[n].k4_items.size();
    }
    out->device_bytes = t.device_bytes();
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_export_layout(flycoo_handle h, uint32_t *d_idx_out, float *d_vals_out,
                                              flycoo_stream_t stream) {
    clear_error();
    if (!h || (h->nnz && (!d_idx_out || !d_vals_out))) {
        set_error("flycoo_export_layout: NULL argument");
        return FLYCOO_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->device);
    FLY_TRY(dg.status(__func__));
    FLY_TRY(check_usable(*h, "flycoo_export_layout"));
    return launch_export_layout(*h, h->elem[h->cur].p, d_idx_out, d_vals_out,
                                reinterpret_cast<cudaStream_t>(stream));
}

extern "C" flycoo_status flycoo_export_partition(flycoo_handle h, int mode, uint64_t *h_ss_ptr,
                                                 uint64_t *h_shard_ptr, uint32_t *h_shard_ss) {
    clear_error();
    if (!h || mode < 0 || mode >= h->N) {
        set_error("flycoo_export_partition: bad handle or mode");
        return FLYCOO_ERR_INVALID_ARG;
    }
    const ModeMeta &md = h->mode[mode];
    if (h_ss_ptr) std::copy(md.ss_ptr.begin(), md.ss_ptr.end(), h_ss_ptr);
    if (h_shard_ptr)
        for (size_t i = 0; i < md.shard_ptr.size(); ++i) h_shard_ptr[i] = md.shard_ptr[i];
    if (h_shard_ss) std::copy(md.shard_ss.begin(), md.shard_ss.end(), h_shard_ss);
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_export_schedule(flycoo_handle h, int mode, int which, uint64_t *h_bin_ptr,
                                                uint64_t *h_items) {
    clear_error();
    if (!h || mode < 0 || mode >= h->N || (which != 0 && which != 1)) {
        set_error("flycoo_export_schedule: bad handle, mode or which");
        return FLYCOO_ERR_INVALID_ARG;
    }
    const ModeMeta &md = h->mode[mode];
    const std::vector<u32> &bp = which == 0 ? md.ss_bin_ptr : md.sh_bin_ptr;
    const std::vector<u32> &it = which == 0 ? md.ss_items : md.sh_items;
    if (h_bin_ptr)
        for (size_t i = 0; i < bp.size(); ++i) h_bin_ptr[i] = bp[i];
    if (h_items)
        for (size_t i = 0; i < it.size(); ++i) h_items[i] = it[i];
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_export_next(flycoo_handle h, int mode, uint32_t *d_next,
                                            flycoo_stream_t stream) {
    clear_error();
    if (!h || mode < 0 || mode >= h->N || (h->nnz && !d_next)) {
        set_error("flycoo_export_next: bad argument");
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (h->nnz == 0) return FLYCOO_OK;
    DeviceGuard dg(h->device);
    FLY_TRY(dg.status(__func__));
    FLY_TRY_CUDA(cudaMemcpyAsync(d_next, h->mode[mode].d_next.p, h->nnz * 4, cudaMemcpyDeviceToDevice,
                                 reinterpret_cast<cudaStream_t>(stream)));
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_export_tile_order(flycoo_handle h, int mode, int stage, uint16_t *d_order,
                                                  flycoo_stream_t stream) {
    clear_error();
    if (!h || mode < 0 || mode >= h->N || (stage != 512 && stage != 1024) || (h->nnz && !d_order)) {
        set_error("flycoo_export_tile_order: bad handle, mode, stage (512 or 1024) or NULL output");
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (h->nnz == 0) return FLYCOO_OK;
    DeviceGuard dg(h->device);
    FLY_TRY(dg.status("flycoo_export_tile_order"));
    FLY_TRY_CUDA(cudaMemcpyAsync(d_order, h->mode[mode].d_perm[stage == 1024 ? 1 : 0].p, h->nnz * 2,
                                 cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)));
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_timing_enable(flycoo_handle h, int enable) {
    clear_error();
    if (!h) {
        set_error("flycoo_timing_enable: handle is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    h->timing = enable != 0;
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_timing_read(flycoo_handle h, double *h_ms, uint64_t *h_launches) {
    clear_error();
    if (!h) {
        set_error("flycoo_timing_read: handle is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->device);
    FLY_TRY(dg.status(__func__));
    double total = 0.0;
    for (auto &pr : h->ev_pending) {
        FLY_TRY_CUDA(cudaEventSynchronize(pr.second));
        float ms = 0.f;
        FLY_TRY_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        total += ms;
    }
    if (h_ms) *h_ms = total;
    if (h_launches) *h_launches = h->ev_pending.size();
    h->ev_pending.clear();
    h->ev_used = 0;
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_debug_set_wait_limit(flycoo_handle h, int64_t polls) {
    clear_error();
    if (!h) {
        set_error("flycoo_debug_set_wait_limit: handle is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    h->wait_limit = polls < 0 ? kSpinLimit : (u32)std::min<int64_t>(polls, kSpinLimit);
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_debug_fail_alloc_after(int64_t n) {
    clear_error();
    g_alloc_fail_after = n < 0 ? -1 : n;
    return FLYCOO_OK;
}

// --------------------------------------------------------------------------
// host-only planner
// --------------------------------------------------------------------------
struct flycoo_plan_s : flycoo::ModePlan {
    u64 g = 0;
    u32 bins = 0;
};

static flycoo_status plan_create_impl(uint64_t nnz, uint64_t k, const uint64_t *h_ss_ptr, uint64_t g,
                                      uint32_t bins, uint32_t schedule, flycoo_plan *out) {
    if (!out) {
        set_error("flycoo_plan_create: out is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (nnz >= 0xffffffffull) {
        set_error("flycoo_plan_create: nnz must be < 2^32 - 1");
        return FLYCOO_ERR_UNSUPPORTED;
    }
    if (!h_ss_ptr || k == 0 || k >= 0xffffffffull) {
        set_error("flycoo_plan_create: need 1 <= k < 2^32 - 1 and k + 1 super-shard pointers");
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (bins == 0 || bins > kMaxBins) {
        set_error("flycoo_plan_create: bins = %u outside [1, %u]", bins, kMaxBins);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (schedule != FLYCOO_SCHEDULE_LPT && schedule != FLYCOO_SCHEDULE_BLOCK_CYCLIC) {
        set_error("flycoo_plan_create: unknown schedule %u", schedule);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (g == 0) g = default_shard_size(nnz, bins);
    if (g > 0xffffffffull) {
        set_error("flycoo_plan_create: g too large");
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (h_ss_ptr[0] != 0 || h_ss_ptr[k] != nnz) {
        set_error("flycoo_plan_create: super-shard pointers must run from 0 to nnz");
        return FLYCOO_ERR_INVALID_ARG;
    }
    for (u64 j = 0; j < k; ++j)
        if (h_ss_ptr[j] > h_ss_ptr[j + 1]) {
            set_error("flycoo_plan_create: super-shard pointer %llu decreases", (unsigned long long)j);
            return FLYCOO_ERR_INVALID_ARG;
        }
    auto p = std::make_unique<flycoo_plan_s>();
    p->k = k;
    p->ss_ptr.assign(h_ss_ptr, h_ss_ptr + k + 1);
    p->g = g;
    p->bins = bins;
    plan_mode(*p, nnz, g, bins, schedule);
    *out = p.release();
    return FLYCOO_OK;
}

extern "C" flycoo_status flycoo_plan_create(uint64_t nnz, uint64_t k, const uint64_t *h_ss_ptr, uint64_t g,
                                            uint32_t bins, uint32_t schedule, flycoo_plan *out) {
    clear_error();
    return host_guarded("flycoo_plan_create",
                        [&] { return plan_create_impl(nnz, k, h_ss_ptr, g, bins, schedule, out); });
}

extern "C" flycoo_status flycoo_plan_get(flycoo_plan p, int which, uint64_t *h_out, uint64_t *count) {
    clear_error();
    if (!p || !count) {
        set_error("flycoo_plan_get: plan or count is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    const u64 g1[1] = {p->g};
    const u64 nl1[1] = {p->k4_nlight};
    const u64 *wide = nullptr;
    const std::vector<u32> *v = nullptr;
    u64 n = 0;
    switch (which) {
    case FLYCOO_PLAN_G: wide = g1; n = 1; break;
    case FLYCOO_PLAN_K4_NLIGHT: wide = nl1; n = 1; break;
    case FLYCOO_PLAN_SHARD_PTR: v = &p->shard_ptr; break;
    case FLYCOO_PLAN_SHARD_SS: v = &p->shard_ss; break;
    case FLYCOO_PLAN_SS_SHARD_PTR: v = &p->ss_shard_ptr; break;
    case FLYCOO_PLAN_SS_BIN_PTR: v = &p->ss_bin_ptr; break;
    case FLYCOO_PLAN_SS_ITEMS: v = &p->ss_items; break;
    case FLYCOO_PLAN_SHARD_BIN_PTR: v = &p->sh_bin_ptr; break;
    case FLYCOO_PLAN_SHARD_ITEMS: v = &p->sh_items; break;
    case FLYCOO_PLAN_K4_ITEMS: v = &p->k4_items; break;
    case FLYCOO_PLAN_TILE_BIN_PTR_512: v = &p->tile_bin_ptr[0]; break;
    case FLYCOO_PLAN_TILES_512: v = &p->tiles[0]; break;
    case FLYCOO_PLAN_TILE_BIN_PTR_1024: v = &p->tile_bin_ptr[1]; break;
    case FLYCOO_PLAN_TILES_1024: v = &p->tiles[1]; break;
    case FLYCOO_PLAN_SEG_SS: v = &p->seg_ss; break;
    case FLYCOO_PLAN_SS_SEG_PTR: v = &p->ss_seg_ptr; break;
    case FLYCOO_PLAN_K4_ORDER: v = &p->k4_order; break;
    default:
        set_error("flycoo_plan_get: unknown array %d", which);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (v) n = v->size();
    if (h_out) {
        if (*count < n) {
            set_error("flycoo_plan_get: array %d has %llu entries, the buffer %llu", which, (unsigned long long)n,
                      (unsigned long long)*count);
            *count = n;
            return FLYCOO_ERR_INVALID_ARG;
        }
        for (u64 i = 0; i < n; ++i) h_out[i] = v ? (*v)[i] : wide[i];
    }
    *count = n;
    return FLYCOO_OK;
}

extern "C" void flycoo_plan_destroy(flycoo_plan p) { delete p; }
