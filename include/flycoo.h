/*
 * flycoo.h -- C ABI of the GB300 (sm_103a) FLYCOO spMTTKRP library.
 *
 * The library computes sparse MTTKRP (spMTTKRP) for every mode of an N-mode
 * sparse tensor held in the FLYCOO format, and remaps the tensor to the next
 * mode's shard order inside the same pass (Wijeratne, Kannan, Prasanna,
 * "Dynasor", arXiv 2309.09131: Section II-C, Section III, Algorithm 2).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are DEVICE pointers on the handle's device; pointers
 *    named h_* are HOST pointers.  The caller owns every buffer it passes;
 *    the handle owns the FLYCOO buffers it allocates in flycoo_create and
 *    frees them in flycoo_destroy.
 *  - Dense matrices are row-major.  Factor matrix Y_w is I_w x R; an output
 *    M_n is I_n x R in FP32.  Coordinates are 0-based (Section II-A).
 *  - Work is ordered on the given stream (a cudaStream_t; NULL is the legacy
 *    default stream).  Only flycoo_create, flycoo_sync, flycoo_cpopt_grad
 *    (for its loss), flycoo_cp_als_step, the export_* calls that fill host
 *    buffers and flycoo_timing_read wait for the stream.
 *  - Every entry point returns a flycoo_status and never aborts or traps;
 *    flycoo_last_error() then describes the failure (per calling thread).
 *  - A handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef FLYCOO_H
#define FLYCOO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *flycoo_stream_t; /* a cudaStream_t */

typedef enum {
    FLYCOO_OK = 0,
    FLYCOO_ERR_INVALID_ARG = 1,  /* a size, mode, pointer or parameter is invalid   */
    FLYCOO_ERR_INDEX_RANGE = 2,  /* a coordinate is >= its mode's size               */
    FLYCOO_ERR_OOM = 3,          /* a device or host allocation failed               */
    FLYCOO_ERR_LAYOUT = 4,       /* the tensor is not in the layout the call needs   */
    FLYCOO_ERR_NOT_SPD = 5,      /* an ALS normal-equation matrix is not SPD         */
    FLYCOO_ERR_TIMEOUT = 6,      /* a bounded device wait gave up                    */
    FLYCOO_ERR_CUDA = 7,         /* a CUDA runtime call failed                       */
    FLYCOO_ERR_UNSUPPORTED = 8   /* valid, but not built (mode count, rank, dtype)   */
} flycoo_status;

typedef enum {
    FLYCOO_F32 = 0,  /* factor matrices stored as IEEE binary32                      */
    FLYCOO_BF16 = 1  /* factor matrices stored as bfloat16; products and sums in FP32 */
} flycoo_dtype;

#define FLYCOO_MAX_MODES 8

/* Partitioning parameters (Section III-A and III-C).  Zero selects the default.
 *  m[n]  super-shard width of mode n: super-shard j holds the nonzeros whose
 *        mode-n index lies in [j*m[n], (j+1)*m[n]).  At most 64: the fused
 *        kernel keeps a super-shard's m[n] output rows in shared memory (the
 *        cache budget of Eq. 3).  Default min(I_n, 32) when the dims sum to
 *        at most 2^18 rows (factor matrices that stay in L2: fewer rows per
 *        stage tile give longer row runs and more factor-row cache hits),
 *        else min(I_n, 64).
 *  g     shard size in nonzeros: each super-shard is cut into runs of g
 *        consecutive nonzeros (the last one shorter).  Default: the largest
 *        power of two in [1024, 32768] that leaves at least sixteen shards
 *        per bin (1024 when none does).
 *  bins  number of schedule bins of Algorithm 3, which is also the number of
 *        thread blocks of the fused kernel; at most 2^20.  Default: 3 x the
 *        SM count.
 *  schedule  FLYCOO_SCHEDULE_LPT (0, default): Algorithm 3 -- items sorted by
 *        size, each to the least-loaded bin; FLYCOO_SCHEDULE_BLOCK_CYCLIC (1):
 *        item i to bin i mod bins, in ascending order (the baseline the paper
 *        compares Algorithm 3 with, Section V-D).  Applies to both schedules.
 *  order  FLYCOO_ORDER_KEY (0, default): inside each super-shard of mode n
 *        the nonzeros follow the other modes' super-shard ids in the order
 *        n-1, n-2, ..., n+1 (the key order of flycoo_create);
 *        FLYCOO_ORDER_MORTON (1): they follow the Z-Morton code of the other
 *        modes' super-shard ids (the Z-Morton ordering of super-shards of the
 *        preprocessing in Section V-J): bit levels from the most significant
 *        down, modes n+1, n+2, ..., n-1 at each level, each id with the bit
 *        width of its mode's largest id; the widths of a mode's other modes
 *        must add up to at most 64 bits.  Ties keep the input order. */
#define FLYCOO_SCHEDULE_LPT 0
#define FLYCOO_SCHEDULE_BLOCK_CYCLIC 1
#define FLYCOO_ORDER_KEY 0
#define FLYCOO_ORDER_MORTON 1
typedef struct {
    uint64_t m[FLYCOO_MAX_MODES];
    uint64_t g;
    uint32_t bins;
    uint32_t schedule;
    uint32_t order;
    uint32_t reserved;   /* must be 0 */
} flycoo_params;

/* Read-only description of a handle. */
typedef struct {
    int32_t N;                                  /* number of modes                    */
    int32_t layout_mode;                        /* mode whose layout L_n is current   */
    uint64_t nnz;                               /* nonzeros (duplicates count apart)  */
    uint64_t dims[FLYCOO_MAX_MODES];            /* I_n                                */
    uint64_t m[FLYCOO_MAX_MODES];               /* super-shard width used             */
    uint64_t g;                                 /* shard size used                    */
    uint32_t bins;                              /* schedule bins used                 */
    uint32_t elem_bytes;                        /* bytes of one stored nonzero        */
    uint32_t schedule;                          /* FLYCOO_SCHEDULE_*                  */
    uint32_t order;                             /* FLYCOO_ORDER_*                     */
    uint32_t reserved;
    uint64_t super_shards[FLYCOO_MAX_MODES];    /* k_n = ceil(I_n / m_n)              */
    uint64_t shards[FLYCOO_MAX_MODES];          /* S_n = sum_j ceil(|SS_n,j| / g)     */
    uint64_t segments[FLYCOO_MAX_MODES];        /* runs of one super-shard's shards in one bin */
    uint64_t fixup_super_shards[FLYCOO_MAX_MODES]; /* super-shards without exactly one segment */
    uint64_t device_bytes;                      /* device memory the handle holds     */
} flycoo_info;

typedef struct flycoo_tensor *flycoo_handle;

/* ------------------------------------------------------------------------ */
/* flycoo_create -- convert a COO tensor to FLYCOO (Section III-A; the       */
/* preprocessing of Section V-J).  For every mode n it computes the layout   */
/* L_n: nonzeros ordered by their super-shard ids (ss_n, ss_{n-1}, ...,      */
/* ss_{n+1}, input position) with ss_w = c_w div m[w], cut into super-shards */
/* and shards; each nonzero's slot in L_{(n+1) mod N}; the Algorithm 3       */
/* schedules; and, for every stage tile the fused pass streams (runs of 512  */
/* and of 1024 positions from each shard start), the order that sorts the    */
/* tile stably by c_n (flycoo_export_tile_order).  The tensor is then stored */
/* in layout L_0.                                                            */
/*  N       number of modes, 3 <= N <= 5.                                    */
/*  h_dims  N mode sizes, each in [1, 2^32 - 1].                             */
/*  nnz     nonzeros, < 2^32 - 1.  0 is allowed.                             */
/*  d_idx   N x nnz uint32, mode-major: coordinate of mode w of nonzero e is */
/*          d_idx[w*nnz + e].  Copied; the caller may free it on return.      */
/*  d_vals  nnz float32 values.  Copied.                                     */
/*  params  NULL or partition parameters (zeros = defaults).                 */
/*  out     receives the handle.                                             */
/* With params->order = FLYCOO_ORDER_MORTON the order inside each           */
/* super-shard is the Z-Morton variant described at flycoo_params.           */
/* Errors: INVALID_ARG (also m[n] > 64, bins > 2^20, unknown schedule or     */
/* order, Morton codes wider than 64 bits),                                  */
/* INDEX_RANGE (any coordinate >= its I_w), UNSUPPORTED (N outside 3..5,     */
/* nnz >= 2^32 - 1), OOM, CUDA.  Waits for `stream`.                         */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_create(int N, const uint64_t *h_dims, uint64_t nnz, const uint32_t *d_idx,
                            const float *d_vals, const flycoo_params *params,
                            flycoo_stream_t stream, flycoo_handle *out);

/* Free every buffer the handle owns.  NULL is ignored. */
void flycoo_destroy(flycoo_handle h);

/* ------------------------------------------------------------------------ */
/* flycoo_spmttkrp -- spMTTKRP of one mode with the fused dynamic remap      */
/* (Algorithm 2 for one value of n; elementwise equation of Section IV):     */
/*   d_out[i, r] = sum over nonzeros x with c_mode(x) = i of                 */
/*                 val(x) * prod_{w != mode} Y_w[c_w(x), r]                   */
/* Rows that no nonzero touches are written as 0.  Accumulation is FP32 in a */
/* fixed order: the result is bitwise reproducible for a given handle.       */
/*  mode       output mode; the tensor must be in layout L_mode.             */
/*  h_factors  HOST array of N DEVICE pointers, Y_w is I_w x R row-major in  */
/*             `fdt`, 16-byte aligned.  Entry `mode` is not read (may be     */
/*             NULL).                                                        */
/*  R          rank: 16, 32 or 64; or 128 on a 3-mode tensor (else          */
/*             UNSUPPORTED).                                                 */
/*  d_out      I_mode x R FP32, 16-byte aligned, written in full.  It must   */
/*             not overlap a factor.                                         */
/*  next_mode  -1: no remap.  (mode + 1) mod N: store every nonzero at its   */
/*             slot of L_next during the pass (Algorithm 2, the Store of the  */
/*             remap step); the tensor is then in layout L_next.             */
/* Errors: INVALID_ARG, LAYOUT (tensor not in L_mode, or a remapping pass   */
/* on this handle gave up, see flycoo_sync), UNSUPPORTED, CUDA.              */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_spmttkrp(flycoo_handle h, int mode, const void *const *h_factors,
                              flycoo_dtype fdt, int R, float *d_out, int next_mode,
                              flycoo_stream_t stream);

/* ------------------------------------------------------------------------ */
/* flycoo_all_modes_host -- Algorithm 2 end to end from host memory: copy   */
/* the N factors in, spMTTKRP of every mode n = 0..N-1 in turn with the     */
/* fused remap to the next layout (the tensor is first remapped to L_0 if  */
/* it is elsewhere, and ends in L_0), each output copied back as soon as    */
/* its pass ends; then wait for the stream and check the device error word. */
/*  h_factors  HOST array of N HOST pointers, Y_w is I_w x R row-major in   */
/*             `fdt` (pinned memory makes the copies asynchronous)          */
/*  R          16, 32 or 64, or 128 as flycoo_spmttkrp allows it            */
/*  h_out      HOST array of N HOST pointers, M_n is I_n x R FP32,          */
/*             overwritten                                                  */
/* The first call allocates device staging for the factors and outputs     */
/* (kept until flycoo_destroy, reallocated when a later call needs more).  */
/* Waits for `stream`.  Errors: INVALID_ARG, LAYOUT, UNSUPPORTED, OOM,       */
/* TIMEOUT, CUDA.                                                           */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_all_modes_host(flycoo_handle h, const void *const *h_factors, flycoo_dtype fdt, int R,
                                    float *const *h_out, flycoo_stream_t stream);

/* ------------------------------------------------------------------------ */
/* flycoo_spmttkrp_static_scratch -- the paper has no counterpart; this is a  */
/* library convenience.  Same computation, arguments, errors and results as   */
/* flycoo_spmttkrp, but the call allocates nothing: the row blocks of the    */
/* super-shards split over several segments go to a fixed device array inside */
/* the library (8 MiB per GPU, held by every GPU that loads the library until */
/* the process exits) instead of the scratch buffer flycoo_create allocated.  */
/* It is meant for callers that must not allocate device memory at the point  */
/* of the call, for example code running while another allocator owns the    */
/* GPU's free memory, or code that must not enter cudaMalloc on a time-bound  */
/* path.  The handle itself still comes from flycoo_create, which allocates.  */
/*  - Limit: Q_mode x m_mode x R x 4 bytes must fit in 8 MiB (Q_mode =        */
/*    segments and m_mode = super-shard width of the mode, see               */
/*    flycoo_get_info); larger requests return INVALID_ARG and               */
/*    flycoo_last_error() gives both sizes.  A larger g lowers Q_mode.        */
/*  - flycoo_timing_enable does not time this pass (recording its events     */
/*    could create them).                                                    */
/*  - The first call on a device looks up the array's device address with     */
/*    that device current; make that first call before any stream capture.    */
/*  - All calls on a device share the one array and it keeps the last call's  */
/*    contents; nothing in it needs to start at zero (every partial row is     */
/*    written before it is read in the same call).  Calls whose work overlaps  */
/*    on the GPU (different streams, or different handles at once) race on it. */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_spmttkrp_static_scratch(flycoo_handle h, int mode, const void *const *h_factors,
                                             flycoo_dtype fdt, int R, float *d_out, int next_mode,
                                             flycoo_stream_t stream);

/* ------------------------------------------------------------------------ */
/* flycoo_mttkrp_adjoint -- adjoint of flycoo_spmttkrp.  The elementwise     */
/* update of Section IV (Eq. 4) is linear in each input factor and in each   */
/* nonzero value.  For an upstream gradient G = d loss / d M_mode            */
/* (I_mode x R):                                                             */
/*   dY_w = spMTTKRP_w(X, Y with Y_mode replaced by G)      for each w != mode */
/*   dval(x) = sum_r G[c_mode(x), r] prod_{w != mode} Y_w[c_w(x), r]         */
/* Each dY_w is one fused pass of mode w in layout L_w, so it reuses that    */
/* mode's shards without atomics (and remaps as it goes).  The tensor is     */
/* first remapped to L_{mode+1} if it is elsewhere and ends in L_mode; the   */
/* value gradient is formed when the walk passes through L_0 (one gather of  */
/* the N rows of every nonzero, FP32 products, a fixed-order sum).           */
/*  h_factors   HOST array of N DEVICE factor pointers of type fdt, I_w x R, */
/*              16-byte aligned (entry mode unused, may be NULL)             */
/*  fdt         FLYCOO_F32 or FLYCOO_BF16: the type of the factors and of G  */
/*  R           16, 32 or 64                                                 */
/*  d_gout      I_mode x R upstream gradient of type fdt                     */
/*  h_gfactors  HOST array of N DEVICE pointers, I_w x R FP32 outputs,       */
/*              overwritten; NULL entries (and entry mode) are skipped       */
/*  d_gvals     DEVICE nnz floats, or NULL: d_gvals[e] is dval of the        */
/*              nonzero given at input position e of flycoo_create (the     */
/*              caller's COO order), overwritten                            */
/* Errors: INVALID_ARG, LAYOUT (a remapping pass gave up earlier),           */
/* UNSUPPORTED (rank), CUDA.                                                 */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_mttkrp_adjoint(flycoo_handle h, int mode, const void *const *h_factors,
                                    flycoo_dtype fdt, int R, const void *d_gout,
                                    float *const *h_gfactors, float *d_gvals, flycoo_stream_t stream);

/* ------------------------------------------------------------------------ */
/* flycoo_cpopt_grad -- weighted CP on the observed entries (CP-OPT loss):   */
/*   L = 1/2 sum_x (x - m_x)^2,   m_x = sum_r prod_w Y_w[c_w(x), r] (Eq. 1)  */
/*   dL/dY_n = -spMTTKRP_n with each value x replaced by its residual x - m_x */
/* One fused pass per mode (N passes, each remapping to the next layout, so  */
/* the tensor ends where it started); the residual is formed inside the      */
/* pass from the gathered rows.  FP32 arithmetic, the loss summed in FP64 in */
/* a fixed order.                                                            */
/*  h_factors  HOST array of N DEVICE FP32 factor pointers (I_w x R)         */
/*  h_grads    HOST array of N DEVICE FP32 outputs (I_w x R), overwritten    */
/*  h_loss     HOST double; NULL skips the loss (and the wait for it)        */
/* Waits for `stream` when h_loss is given.  Errors: INVALID_ARG,            */
/* UNSUPPORTED (rank), CUDA.                                                 */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_cpopt_grad(flycoo_handle h, const float *const *h_factors, int R,
                                float *const *h_grads, double *h_loss, flycoo_stream_t stream);

/* ------------------------------------------------------------------------ */
/* flycoo_cp_als_step -- one CP-ALS iteration (Algorithm 1, Section II-B).   */
/* Modes are updated in order 0..N-1, each with the newest factors:          */
/*   M_n = spMTTKRP_n(X, Y)                 (one fused pass, remapping on)   */
/*   V   = hadamard_{w != n} Y_w^T Y_w      (R x R, FP64)                    */
/*   Y_n = M_n V^{-1}                       (V = L D L^T in FP64)            */
/*   lambda_r = ||Y_n[:, r]||_2,  Y_n[:, r] /= lambda_r  (0 norms kept as 1) */
/* Algorithm 1 names the spMTTKRP and the normalisation; the least-squares   */
/* solve between them is the standard CP-ALS update the paper builds on.     */
/* The tensor is first remapped to L_0 if it is elsewhere; N passes later it */
/* is back in L_0.  After the last mode                                      */
/*   fit = 1 - ||X - Xhat||_F / ||X||_F,  Xhat = [[lambda; Y_0..Y_{N-1}]],  */
/* from ||Xhat||^2 = lambda^T (hadamard_w Y_w^T Y_w) lambda and             */
/* <X, Xhat> = sum_r lambda_r sum_i M_{N-1}[i,r] Y_{N-1}[i,r].               */
/*  h_factors  HOST array of N DEVICE factor pointers (I_w x R, row-major,   */
/*             type fdt, 16-byte aligned); updated in place                   */
/*  fdt        FLYCOO_F32 or FLYCOO_BF16: the storage type of the factors;  */
/*             an updated factor is rounded to FP32, then to BF16 (nearest  */
/*             even) when stored in BF16, before later modes read it        */
/*  R          16, 32 or 64                                                  */
/*  d_lambda   DEVICE array of R doubles: the last mode's column norms       */
/*  h_fit      HOST double, or NULL                                          */
/* Waits for `stream`.  Allocates a workspace on the first call (about       */
/* 2 x max_w I_w x 64 x 4 bytes), kept until flycoo_destroy.  Errors:        */
/* INVALID_ARG (NULL or misaligned pointers, a tensor whose values are all  */
/* zero), UNSUPPORTED (rank), NOT_SPD (a matrix V with a pivot <= 0: the     */
/* modes before it were updated, the others are unchanged), OOM, CUDA.       */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_cp_als_step(flycoo_handle h, void *const *h_factors, flycoo_dtype fdt, int R,
                                 double *d_lambda, double *h_fit, flycoo_stream_t stream);

/* ------------------------------------------------------------------------ */
/* flycoo_cp_als -- `iters` CP-ALS iterations in one call (Algorithm 1's     */
/* loop), each exactly as flycoo_cp_als_step.  The Gram matrices are        */
/* computed from the factors as given once, at the start; later iterations  */
/* reuse the Gram matrix computed after each factor update, which the       */
/* single-step call cannot (the caller may change the factors between        */
/* calls).  The results equal `iters` calls of flycoo_cp_als_step.           */
/*  iters   1 .. 10^6                                                       */
/*  h_fits  HOST array of `iters` doubles (the fit after each iteration), or */
/*          NULL                                                            */
/* Other arguments, allocation and errors as flycoo_cp_als_step; waits for  */
/* `stream` once, at the end.  After NOT_SPD in some iteration, the later    */
/* ones leave the factors unchanged.                                        */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_cp_als(flycoo_handle h, void *const *h_factors, flycoo_dtype fdt, int R, int iters,
                            double *d_lambda, double *h_fits, flycoo_stream_t stream);

/* ------------------------------------------------------------------------ */
/* flycoo_remap -- dynamic tensor remapping alone (Section III-B): move the  */
/* tensor from its current layout to L_next_mode.  Each step stores every    */
/* nonzero at its slot of the following mode's layout; the call takes       */
/* (next_mode - layout_mode) mod N steps (0 steps if already there).        */
/* Errors: INVALID_ARG, CUDA.                                                */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_remap(flycoo_handle h, int next_mode, flycoo_stream_t stream);

/* Wait for `stream`, then report device-side failures since the last check: */
/* FLYCOO_ERR_TIMEOUT if a bounded device wait (on a tile-load barrier) gave  */
/* up; the flag is cleared.  The kernels never trap: this is how they report.  */
/* A block that gives up lets its own copies in flight land (bounded) and     */
/* returns, so the GPU context stays usable.  If a remapping pass was among   */
/* the work checked, the handle's layout is undefined from then on: every     */
/* later call that uses the layout returns FLYCOO_ERR_LAYOUT (recreate the    */
/* handle).  flycoo_cp_als_step and flycoo_cpopt_grad (with h_loss) make the  */
/* same check before they return.                                            */
flycoo_status flycoo_sync(flycoo_handle h, flycoo_stream_t stream);

/* Fill *out with the handle's sizes and parameters. */
flycoo_status flycoo_get_info(flycoo_handle h, flycoo_info *out);

/* ------------------------------------------------------------------------ */
/* Exports of the FLYCOO structures, for checks against a reference.         */
/* ------------------------------------------------------------------------ */

/* The current layout as COO: d_idx_out (N x nnz uint32, mode-major, input  */
/* coordinate order) and d_vals_out (nnz float32), position p of the layout */
/* in column p.  Stream-ordered. */
flycoo_status flycoo_export_layout(flycoo_handle h, uint32_t *d_idx_out, float *d_vals_out,
                                   flycoo_stream_t stream);

/* Section III-A pointers of mode n into host buffers (any may be NULL):     */
/*  h_ss_ptr[k_n + 1]  start of super-shard j in L_n, then nnz;              */
/*  h_shard_ptr[S_n+1] start of each shard in L_n, then nnz;                 */
/*  h_shard_ss[S_n]    super-shard of each shard.                            */
flycoo_status flycoo_export_partition(flycoo_handle h, int mode, uint64_t *h_ss_ptr,
                                      uint64_t *h_shard_ptr, uint32_t *h_shard_ss);

/* Algorithm 3 schedules of mode n as CSR lists into host buffers:           */
/*  which = 0: super-shards binned by shard count (the SS_List of the paper),*/
/*             h_items has k_n entries;                                      */
/*  which = 1: shards binned by nonzero count (the thread-block schedule of */
/*             the fused kernel), h_items has S_n entries.                   */
/* Bin b holds h_items[h_bin_ptr[b] .. h_bin_ptr[b+1]) in assignment order;  */
/* h_bin_ptr has bins + 1 entries.                                           */
flycoo_status flycoo_export_schedule(flycoo_handle h, int mode, int which, uint64_t *h_bin_ptr,
                                     uint64_t *h_items);

/* d_next[p] (nnz uint32): slot in L_{(mode+1) mod N} of the nonzero at      */
/* position p of L_mode -- the remap permutation of mode `mode`.             */
flycoo_status flycoo_export_next(flycoo_handle h, int mode, uint32_t *d_next,
                                 flycoo_stream_t stream);

/* d_order (nnz uint16, DEVICE): compute order of the stage tiles of mode    */
/* `mode` for stage size `stage` (512 or 1024).  The stage tiles are the     */
/* runs of `stage` positions from each shard start of L_mode (the last run   */
/* of a shard shorter); for the tile starting at position s with length len, */
/* d_order[s + p], p < len, is the tile-local index of the nonzero that      */
/* comes p-th when the tile is sorted stably by its mode-`mode` coordinate.  */
/* The fused pass accumulates each tile in this order, so every output row's */
/* nonzeros in a tile are contiguous; the stored layout is not moved.        */
/* Stream-ordered.  Errors: INVALID_ARG (mode, stage, NULL with nnz > 0).    */
flycoo_status flycoo_export_tile_order(flycoo_handle h, int mode, int stage, uint16_t *d_order,
                                       flycoo_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Host-only planner: the partition and schedule step of flycoo_create for   */
/* one mode, on its own.  It touches no device (it runs where no GPU is).    */
/* ------------------------------------------------------------------------ */
typedef struct flycoo_plan_s *flycoo_plan;

/* From the super-shard pointers of one mode (Section III-A), cut every      */
/* super-shard into shards of g nonzeros, schedule the super-shards by shard */
/* count and the shards by nonzero count (Algorithm 3, or block-cyclic), and */
/* write the shard schedule out as the fused kernel's tile descriptors.      */
/* Consecutive shards of one super-shard in one bin form a segment: the      */
/* thread block accumulates the super-shard's rows across the whole segment  */
/* and writes them once (to the output when the super-shard has a single     */
/* segment, else to the segment's row block, which K4 sums).                 */
/* flycoo_create runs exactly this for every mode of a handle.               */
/*  nnz       nonzeros, < 2^32 - 1.                                          */
/*  k         super-shards k_n = ceil(I_n / m_n), in [1, 2^32 - 2].          */
/*  h_ss_ptr  k + 1 host values: start of super-shard j in L_n, then nnz;    */
/*            0 = h_ss_ptr[0] <= h_ss_ptr[1] <= ... <= h_ss_ptr[k] = nnz.     */
/*            Copied.                                                        */
/*  g         shard size; 0 = flycoo_create's default for nnz and bins.     */
/*  bins      schedule bins, in [1, 2^20].                                   */
/*  schedule  FLYCOO_SCHEDULE_LPT or FLYCOO_SCHEDULE_BLOCK_CYCLIC.           */
/*  out       receives the plan; the caller frees it with flycoo_plan_destroy*/
/* Errors: INVALID_ARG (NULL pointers, k, bins, schedule or g out of range,  */
/* pointers that do not split [0, nnz]), UNSUPPORTED (nnz >= 2^32 - 1), OOM  */
/* (host allocation).                                                        */
flycoo_status flycoo_plan_create(uint64_t nnz, uint64_t k, const uint64_t *h_ss_ptr, uint64_t g,
                                 uint32_t bins, uint32_t schedule, flycoo_plan *out);

/* Arrays of a plan.  S = shards, Q = segments, T_z = stage tiles of size    */
/* 512 (z = 0) or 1024 (z = 1).  Schedules are CSR lists: bin b holds        */
/* items[bin_ptr[b] .. bin_ptr[b+1]) in assignment order.  Segments are      */
/* numbered by super-shard, then in schedule order (bin, then position in    */
/* the bin).  A tile descriptor is four values (start, len | flags << 16,    */
/* super-shard, segment), flags 1 = first tile of its segment, 2 = last,     */
/* 4 = the only segment of its super-shard; descriptors run bin by bin in    */
/* the order of the shard schedule.                                          */
typedef enum {
    FLYCOO_PLAN_G = 0,              /* 1: the shard size used                 */
    FLYCOO_PLAN_SHARD_PTR = 1,      /* S + 1: start of each shard, then nnz   */
    FLYCOO_PLAN_SHARD_SS = 2,       /* S: super-shard of each shard           */
    FLYCOO_PLAN_SS_SHARD_PTR = 3,   /* k + 1: first shard of each super-shard */
    FLYCOO_PLAN_SS_BIN_PTR = 4,     /* bins + 1: super-shard schedule         */
    FLYCOO_PLAN_SS_ITEMS = 5,       /* k                                      */
    FLYCOO_PLAN_SHARD_BIN_PTR = 6,  /* bins + 1: shard (thread-block) schedule*/
    FLYCOO_PLAN_SHARD_ITEMS = 7,    /* S                                      */
    FLYCOO_PLAN_K4_ITEMS = 8,       /* super-shards without exactly one segment */
    FLYCOO_PLAN_TILE_BIN_PTR_512 = 9,   /* bins + 1, in descriptors           */
    FLYCOO_PLAN_TILES_512 = 10,         /* 4 x T_0                            */
    FLYCOO_PLAN_TILE_BIN_PTR_1024 = 11, /* bins + 1                           */
    FLYCOO_PLAN_TILES_1024 = 12,        /* 4 x T_1                            */
    FLYCOO_PLAN_SEG_SS = 13,            /* Q: super-shard of each segment     */
    FLYCOO_PLAN_SS_SEG_PTR = 14,        /* k + 1: segments of each super-shard */
    /* the fixup kernel's launch order of the K4 items: those of at most 16   */
    /* segments (one thread block each) in ascending order, then the others   */
    /* (one block per 64 floats of their row block) in ascending order        */
    FLYCOO_PLAN_K4_ORDER = 15,          /* |K4 items|                         */
    FLYCOO_PLAN_K4_NLIGHT = 16          /* 1: how many of them come first     */
} flycoo_plan_array;

/* Copy array `which` into h_out, widened to uint64.  *count is in: the     */
/* capacity of h_out; out: the array's length.  h_out NULL only reports the  */
/* length.  Errors: INVALID_ARG (NULL plan or count, unknown array, capacity */
/* too small -- *count then holds the length needed).                       */
flycoo_status flycoo_plan_get(flycoo_plan p, int which, uint64_t *h_out, uint64_t *count);

/* Free a plan (NULL is ignored). */
void flycoo_plan_destroy(flycoo_plan p);

/* ------------------------------------------------------------------------ */
/* Kernel timing of the fused spMTTKRP + remap kernel.  While enabled, each  */
/* flycoo_spmttkrp records CUDA events around that kernel on its stream.     */
/* flycoo_timing_read waits for them, returns the summed milliseconds and   */
/* the launch count since the last read, and clears them.                    */
/* ------------------------------------------------------------------------ */
flycoo_status flycoo_timing_enable(flycoo_handle h, int enable);
flycoo_status flycoo_timing_read(flycoo_handle h, double *h_ms, uint64_t *h_launches);

/* Message of the last failed call on this thread ("" if none). */
const char *flycoo_last_error(void);

/* ------------------------------------------------------------------------ */
/* Test hooks for the failure paths (no counterpart in the paper).           */
/* ------------------------------------------------------------------------ */

/* Polls of a tile-load barrier before a fused pass of this handle gives up: */
/* `polls` >= 0 sets the limit (0 gives up at the first tile without        */
/* polling), negative restores the default (2^24 polls).  The drain of the   */
/* copies in flight after giving up keeps the default bound.  Errors:        */
/* INVALID_ARG.                                                              */
flycoo_status flycoo_debug_set_wait_limit(flycoo_handle h, int64_t polls);

/* Process-wide: the next `n` device allocations of the library succeed and  */
/* the one after fails with FLYCOO_ERR_OOM (then every later one, until the  */
/* hook is reset); negative switches the hook off.  Not thread-safe.        */
flycoo_status flycoo_debug_fail_alloc_after(int64_t n);

#ifdef __cplusplus
}
#endif

#endif /* FLYCOO_H */
