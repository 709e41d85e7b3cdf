// internal.cuh -- shared declarations of the FLYCOO CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "flycoo.h"

namespace flycoo {

using u32 = uint32_t;
using u64 = uint64_t;

// --------------------------------------------------------------------------
// errors
// --------------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();

#define FLY_TRY_CUDA(call)                                                                    \
    do {                                                                                      \
        cudaError_t e__ = (call);                                                             \
        if (e__ != cudaSuccess) {                                                             \
            ::flycoo::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e__),      \
                                __FILE__, __LINE__);                                          \
            return e__ == cudaErrorMemoryAllocation ? FLYCOO_ERR_OOM : FLYCOO_ERR_CUDA;       \
        }                                                                                     \
    } while (0)

#define FLY_TRY(call)                                                                         \
    do {                                                                                      \
        flycoo_status s__ = (call);                                                           \
        if (s__ != FLYCOO_OK) return s__;                                                     \
    } while (0)

// Owning device allocation (freed on destruction).
// test hook: the number of device allocations that still succeed before one
// fails with FLYCOO_ERR_OOM; negative = never (flycoo_debug_fail_alloc_after)
extern long long g_alloc_fail_after;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    flycoo_status alloc(size_t n) {
        release();
        if (n == 0) n = 16;
        if (g_alloc_fail_after == 0) {
            set_error("cudaMalloc(%zu) refused by the allocation-failure test hook", n);
            return FLYCOO_ERR_OOM;
        }
        if (g_alloc_fail_after > 0) --g_alloc_fail_after;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? FLYCOO_ERR_OOM : FLYCOO_ERR_CUDA;
        }
        bytes = n;
        return FLYCOO_OK;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
    void swap(DevBuf &o) {
        std::swap(p, o.p);
        std::swap(bytes, o.bytes);
    }
};

// Makes the handle's device current for the life of the guard and restores
// the caller's device afterwards.  status() reports a failed switch, so no
// work is enqueued on the wrong device.
struct DeviceGuard {
    int prev = -1;
    int dev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int d) : dev(d) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    }
    flycoo_status status(const char *who) const {
        if (err != cudaSuccess) {
            set_error("%s: could not make device %d current: %s", who, dev, cudaGetErrorString(err));
            return FLYCOO_ERR_CUDA;
        }
        return FLYCOO_OK;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// The ranks a fused spMTTKRP pass of `mode` is built for: 16, 32, 64, and 128
// on 3-mode tensors whose output mode has super-shards of at most 64 rows.
// Defined in api.cu.
struct Tensor;
flycoo_status check_pass_rank(const Tensor &t, int mode, int R, const char *who);

// --------------------------------------------------------------------------
// FLYCOO description of one mode (Section III-A)
// --------------------------------------------------------------------------
// the host part: what plan_mode derives from the super-shard pointers
struct ModePlan {
    u64 I = 0, m = 0, k = 0, S = 0;
    std::vector<u64> ss_ptr;              // k + 1: first position of each super-shard in L_n
    std::vector<u32> shard_ptr;           // S + 1: first position of each shard in L_n
    std::vector<u32> shard_ss;            // S: super-shard of each shard
    std::vector<u32> ss_shard_ptr;        // k + 1: shards of super-shard j are [ss_shard_ptr[j], ss_shard_ptr[j+1])
    std::vector<u32> ss_bin_ptr, ss_items;  // Algorithm 3 over super-shards
    std::vector<u32> sh_bin_ptr, sh_items;  // Algorithm 3 over shards (kernel schedule)
    // segments: maximal runs of shards of one super-shard that follow each
    // other in one bin of the shard schedule.  A thread block accumulates a
    // segment's rows in shared memory without flushing between its shards;
    // each segment of a super-shard with several segments writes one row
    // block, numbered so that the blocks of super-shard j are
    // [ss_seg_ptr[j], ss_seg_ptr[j+1]) in schedule order
    std::vector<u32> seg_ss;                // segments: super-shard of each
    std::vector<u32> ss_seg_ptr;            // k + 1
    std::vector<u32> k4_items;              // super-shards whose rows K4 writes (not exactly one segment)
    // K4's launch order of k4_items: the k4_nlight items of at most
    // kFixupLightSegs segments first, then the others
    std::vector<u32> k4_order;
    u32 k4_nlight = 0;
    std::vector<u32> tile_ptr[2];           // T_z + 1: stage tiles of each size (K1 only)
    // tile descriptors in block-schedule order (bin b: tiles [tile_bin_ptr[b],
    // tile_bin_ptr[b+1])), four words each: start, len | flags << 16,
    // super-shard, segment; flags: 1 first tile of its segment, 2 last tile,
    // 4 the super-shard has no other segment
    // (one set per stage-tile size, kStageTile)
    std::vector<u32> tiles[2], tile_bin_ptr[2];
    u64 nseg() const { return seg_ss.size(); }
};

struct ModeMeta : ModePlan {
    DevBuf d_ss_seg_ptr, d_k4, d_next;
    // compute order of each stage tile (u16 per position, one array per stage
    // size): entry p of a tile is the tile-local index of the nonzero at rank p
    // when the tile is stably sorted by output index
    DevBuf d_perm[2];
    DevBuf d_tiles[2], d_tile_bin_ptr[2];
};

// CP-ALS workspace (als.cu), allocated by the first flycoo_cp_als_step
struct AlsWork {
    DevBuf M;       // max_n I_n x kMaxRank FP32: spMTTKRP of the mode being updated
    DevBuf Y;       // max_n I_n x kMaxRank double-float pairs: M V^{-1} before normalisation
    DevBuf G;       // N x R x R FP64 Gram matrices of the stored factors
    DevBuf gpart;   // per-block Gram partials
    DevBuf W;       // R x R FP64 inverse of the normal-equation matrix
    DevBuf colsq;   // per-block column sums of squares
    DevBuf inner;   // per-block partials of <X, Xhat>
    DevBuf scal;    // small FP64 results (||X||^2, fit) and the status word
    DevBuf fits;    // the fit after each iteration of one call
    u64 rows = 0;
    int nblk = 0;
    bool normx2_valid = false;
    double normx2 = 0.0;
    u64 bytes() const {
        return M.bytes + Y.bytes + G.bytes + gpart.bytes + W.bytes + colsq.bytes + inner.bytes + scal.bytes +
               fits.bytes;
    }
};

struct Tensor {
    int N = 0;
    int device = 0;
    int sm_count = 0;
    u64 nnz = 0;
    u64 dims[FLYCOO_MAX_MODES] = {};
    u64 g = 0;
    u32 bins = 0;
    u32 schedule = 0;   // FLYCOO_SCHEDULE_*
    u32 order = 0;      // FLYCOO_ORDER_*: key order or Z-Morton inside super-shards
    int layout = 0;     // current layout mode
    int elem_words = 4; // 32-bit words per stored nonzero
    int cur = 0;        // which element buffer holds the current layout
    u64 max_seg = 0;   // max over modes of the segment count (row blocks of scratch)
    DevBuf elem[2];
    DevBuf orig;        // nnz u32: input (COO) position of the nonzero at each position of L_0
    u64 max_rows = 0;   // max over modes of min(m_n, I_n): rows of a super-shard
    DevBuf partials;    // max_seg x max_rows x kMaxRank floats: one row block per segment
    DevBuf err;         // device error word: bit 0 = a bounded device wait gave up
    DevBuf loss_part;   // bins doubles: per-block CP-OPT loss partials
    u32 wait_limit = 0;            // mbarrier polls before a fused pass gives up (set by create)
    bool remap_since_sync = false; // a remapping pass was enqueued since the last error-word check
    bool poisoned = false;         // a remapping pass gave up: the layout is undefined
    AlsWork als;
    // device staging of flycoo_all_modes_host (allocated by its first call):
    // the factors (sum_w I_w x R x factor bytes) and the outputs (sum_n I_n x R FP32)
    DevBuf host_factors, host_outs;
    ModeMeta mode[FLYCOO_MAX_MODES];
    // kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    size_t ev_used = 0;
    u64 device_bytes() const;
};

constexpr int kMaxRank = 64;   // largest rank of CP-ALS, CP-OPT and the adjoint
// the spMTTKRP pass is also built for rank 128 on 3-mode tensors; its
// accumulator then holds super-shards of at most 64 rows (m x R FP32 in
// shared memory either way)
constexpr int kRank128 = 128;
constexpr u32 kMaxRowsAtRank128 = 64;
// largest super-shard width m_n: the fused kernel keeps a super-shard's output
// rows (m_n x R FP32) in shared memory
#ifndef FLYCOO_MAX_SS_ROWS
#define FLYCOO_MAX_SS_ROWS 64
#endif
constexpr u32 kMaxSuperShardRows = FLYCOO_MAX_SS_ROWS;
static_assert(kMaxSuperShardRows >= 32 && kMaxSuperShardRows % 32 == 0 && kMaxSuperShardRows <= 1024,
              "super-shard rows: a multiple of 32");
// default super-shard width of tensors with few rows in all modes (factor
// matrices that stay in L2): min(I_n, 32).  Narrower super-shards put fewer
// output rows in a stage tile (longer row runs, fewer accumulator flushes) and
// fewer factor rows behind each key window (more L1 hits).  The rule for
// larger tensors sits beside the shard-size rule of the planner.
constexpr u32 kDefaultSuperShardRows = 32;
// stage tiles: the fused kernel streams a shard one stage tile at a time (runs
// of 1024 positions from the shard start when three blocks of that size fit on
// an SM, else 512) and computes each tile in row order through its
// precomputed permutation; the schedule and the permutations exist for both sizes
#ifndef FLYCOO_STAGE_TILE_SMALL
#define FLYCOO_STAGE_TILE_SMALL 512
#endif
#ifndef FLYCOO_STAGE_TILE_LARGE
#define FLYCOO_STAGE_TILE_LARGE 1024
#endif
constexpr u32 kStageTile[2] = {FLYCOO_STAGE_TILE_SMALL, FLYCOO_STAGE_TILE_LARGE};
static_assert(FLYCOO_STAGE_TILE_LARGE <= 0xffffu && FLYCOO_STAGE_TILE_SMALL % 8 == 0, "stage tile sizes");
// iteration limit of every device-side wait (mbarrier polls); ~0.1-1 s
constexpr u32 kSpinLimit = 1u << 24;

// resident blocks per SM the fused kernel is built for (registers and shared
// memory are sized for it); the default number of schedule bins is this
// times the SM count, so one launch is one wave
#ifndef FLYCOO_BLOCKS_PER_SM
#define FLYCOO_BLOCKS_PER_SM 3
#endif
constexpr int kBlocksPerSM = FLYCOO_BLOCKS_PER_SM;
// most schedule bins (thread blocks of a fused pass) a handle or plan takes
constexpr u32 kMaxBins = 1u << 20;
// nonzeros of a 3-mode tensor whose factor-row gathers one thread group issues
// together (each step of the fused kernel's inner loop)
#ifndef FLYCOO_UNROLL3
#define FLYCOO_UNROLL3 3
#endif

inline int elem_words_for(int N) { return (N + 1 <= 4) ? 4 : 8; }

// --------------------------------------------------------------------------
// device building blocks (partition.cu)
// --------------------------------------------------------------------------
// exclusive scan of n uint32 values (in place allowed); scratch >= scan_scratch_words(n)
u64 scan_scratch_words(u64 n);
flycoo_status exclusive_scan_u32(const u32 *in, u32 *out, u64 n, u32 *scratch, cudaStream_t s);

// K1: layouts, remap permutations, super-shard pointers and the L_0 element buffer
flycoo_status build_flycoo(Tensor &t, const u32 *d_idx, const float *d_vals,
                           std::vector<std::vector<u32>> &ss_ptr_host, cudaStream_t s);

// the default shard size g for nnz nonzeros over `bins` schedule bins (api.cu)
u64 default_shard_size(u64 nnz, u32 bins);
// host only: shards, schedules, the K4 list and the tile descriptors of one
// mode from p.ss_ptr and p.k (api.cu); no device work
void plan_mode(ModePlan &p, u64 nnz, u64 g, u32 bins, u32 schedule);
// plan_mode for mode n of a tensor, then the device copies of its schedule (api.cu)
flycoo_status partition_mode(Tensor &t, int n, const std::vector<u32> &ssp, cudaStream_t s);

// standalone remap step L_n -> L_{n+1} (and layout export)
flycoo_status launch_remap_step(const Tensor &t, int n, const void *in, void *out, cudaStream_t s);
flycoo_status launch_export_layout(const Tensor &t, const void *elem, u32 *idx_out, float *vals_out,
                                   cudaStream_t s);

// --------------------------------------------------------------------------
// fused spMTTKRP + remap (K2) and the fixup of multi-shard super-shards (K4)
// --------------------------------------------------------------------------
struct FusedArgs {
    const void *elem_in;
    void *elem_out;            // nullptr: no remap
    const u32 *next;           // nullptr: no remap
    const void *Y[FLYCOO_MAX_MODES - 1]; // factors of slots 1..N-1 of the current layout
    float *out;
    const uint4 *tiles[2];     // tile descriptors, block-schedule order, per stage-tile size
    const u32 *tile_bin_ptr[2]; // bins + 1, per stage-tile size
    const uint16_t *perm[2];   // compute order of each stage tile, per stage-tile size
    float *partials;           // row block of segment s at s * m * R
    u32 *err;                  // device error word
    const void *Yout;          // CP-OPT pass: the output mode's factor (nullptr: plain spMTTKRP)
    double *loss_part;         // CP-OPT pass: per-block half sum of squared residuals (nullable)
    u32 I_out;
    u32 m;                     // super-shard width of the output mode
    u32 bins;                  // thread blocks (schedule bins)
    u32 wait_limit;            // polls of a tile's barrier before the pass gives up
};

// K4 gives a super-shard of at most this many segments one thread block
constexpr u32 kFixupLightSegs = 16;

struct FixupArgs {
    const u32 *items;          // super-shards K4 writes: nlight light ones, then the others
    u32 nitems;
    u32 nlight;
    const u32 *ss_seg_ptr;     // row blocks of super-shard j: [ss_seg_ptr[j], ss_seg_ptr[j+1])
    const float *partials;
    float *out;
    u32 I_out;
    u32 m;
};

flycoo_status launch_fused(int N, int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s);
// the arguments of a fused pass of `mode` in its layout (api.cu): factors F
// (N pointers, entry `mode` unused), output d_out, remap to the next layout or
// not, row blocks of multi-segment super-shards in `partials`
FusedArgs fused_args(const Tensor &t, int mode, const void *const *F, float *d_out, bool remap, float *partials);
FixupArgs fixup_args(const Tensor &t, int mode, float *d_out, const float *partials);
// one fused pass of `mode` in its layout (K2 + K4), leaving the tensor in L_{mode+1}:
// spMTTKRP into d_out, or with Yout set the CP-OPT gradient pass (api.cu)
flycoo_status run_pass(Tensor &t, int mode, const void *const *F, flycoo_dtype fdt, int R, float *d_out,
                       const void *Yout, double *loss_part, cudaStream_t s);
// handle checks (api.cu): not poisoned by a failed remapping pass / the device
// error word (waits for the stream; TIMEOUT when a bounded wait gave up)
flycoo_status check_usable(const Tensor &t, const char *who);
flycoo_status check_error_word(Tensor &t, cudaStream_t s, const char *who);
// K7/K8: `iters` CP-ALS iterations, modes 0..N-1 each, from layout L_0; the
// fit after each iteration into h_fits (nullable); waits for the stream (als.cu)
flycoo_status als_step(Tensor &t, void *const *F, flycoo_dtype fdt, int R, int iters, double *d_lambda,
                       double *h_fits, cudaStream_t s, const char *who);
flycoo_status launch_fixup(int R, const FixupArgs &a, cudaStream_t s);
// gradient of spMTTKRP_mode with respect to the nonzero values for the upstream
// gradient G (I_mode x R, type fdt): d_gvals[e] for every input position e; the
// tensor must be in L_0 (grad.cu)
flycoo_status launch_value_grad(const Tensor &t, int mode, const void *const *Y, const void *G, flycoo_dtype fdt,
                                int R, float *d_gvals, cudaStream_t s);

// launchers implemented per mode count (fused_n3.cu, fused_n4.cu, fused_n5.cu)
flycoo_status launch_fused_n3(int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s);
flycoo_status launch_fused_n4(int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s);
flycoo_status launch_fused_n5(int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s);

} // namespace flycoo

// the opaque handle type of the C ABI
struct flycoo_tensor : flycoo::Tensor {};
