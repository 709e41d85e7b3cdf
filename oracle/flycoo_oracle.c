/*
 * flycoo_oracle.c -- plain, slow FP64 CPU oracle for FLYCOO spMTTKRP.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code,
 * header, table or helper with the CUDA library; it is written directly from
 * the paper (Wijeratne, Kannan, Prasanna, "Dynasor", arXiv 2309.09131):
 *
 *   - the elementwise spMTTKRP update (Section II-C and the elementwise
 *     equation of Section IV): M_n[c_n, r] += val * prod_{w != n} Y_w[c_w, r];
 *   - the FLYCOO partition (Section III-A): super-shards are intervals of m_n
 *     output indices, shards are runs of g elements inside a super-shard;
 *   - the super-shard scheduling (Algorithm 3): sort by size, descending, and
 *     give each item to the least-loaded bin.
 *
 * Every floating-point sum is a sequential FP64 loop over the COO input in its
 * given order.  Nothing is blocked, fused or reordered.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* spMTTKRP, Section II-C (steps 1-8) and the elementwise equation of        */
/* Section IV: for every nonzero x = (c_0..c_{N-1}, val):                    */
/*   l = 1;  for w != n: l = l * Y_w[c_w, :];   M_n[c_n, :] += val * l.       */
/* Rows of M_n that no nonzero touches stay 0 (Algorithm 2 zeroes Y^_n).     */
/* idx is mode-major: coordinate of mode w of element e is idx[w*nnz + e].   */
/* ------------------------------------------------------------------------ */
int oracle_mttkrp(int N, const uint64_t *dims, uint64_t nnz, const uint32_t *idx,
                  const double *vals, const double *const *Y, int R, int n, double *M)
{
    if (N < 1 || n < 0 || n >= N || R < 1) return -1;
    memset(M, 0, (size_t)dims[n] * (size_t)R * sizeof(double));
    double *ell = (double *)malloc((size_t)R * sizeof(double));
    if (!ell) return -2;
    for (uint64_t e = 0; e < nnz; ++e) {
        for (int r = 0; r < R; ++r) ell[r] = 1.0;
        for (int w = 0; w < N; ++w) {
            if (w == n) continue;
            const double *row = Y[w] + (size_t)idx[(size_t)w * nnz + e] * (size_t)R;
            for (int r = 0; r < R; ++r) ell[r] *= row[r];
        }
        double *out = M + (size_t)idx[(size_t)n * nnz + e] * (size_t)R;
        for (int r = 0; r < R; ++r) out[r] += vals[e] * ell[r];
    }
    free(ell);
    return 0;
}

/* The same sum split over `threads` POSIX threads for the timed CPU         */
/* baseline: thread t runs the loop above over the contiguous nonzeros       */
/* [t*nnz/threads, (t+1)*nnz/threads) into a private FP64 matrix, and the    */
/* private matrices are added into M in thread order, so the result does not */
/* depend on thread timing.  threads = 1 is the sequential loop.             */
struct mt_job {
    int N, R, n;
    const uint64_t *dims;
    uint64_t nnz, lo, hi;
    const uint32_t *idx;
    const double *vals;
    const double *const *Y;
    double *M;
    int rc;
};

static void *mt_run(void *arg)
{
    struct mt_job *j = (struct mt_job *)arg;
    double *ell = (double *)malloc((size_t)j->R * sizeof(double));
    if (!ell) { j->rc = -2; return NULL; }
    memset(j->M, 0, (size_t)j->dims[j->n] * (size_t)j->R * sizeof(double));
    for (uint64_t e = j->lo; e < j->hi; ++e) {
        for (int r = 0; r < j->R; ++r) ell[r] = 1.0;
        for (int w = 0; w < j->N; ++w) {
            if (w == j->n) continue;
            const double *row = j->Y[w] + (size_t)j->idx[(size_t)w * j->nnz + e] * (size_t)j->R;
            for (int r = 0; r < j->R; ++r) ell[r] *= row[r];
        }
        double *out = j->M + (size_t)j->idx[(size_t)j->n * j->nnz + e] * (size_t)j->R;
        for (int r = 0; r < j->R; ++r) out[r] += j->vals[e] * ell[r];
    }
    free(ell);
    j->rc = 0;
    return NULL;
}

int oracle_mttkrp_threads(int N, const uint64_t *dims, uint64_t nnz, const uint32_t *idx,
                          const double *vals, const double *const *Y, int R, int n, int threads,
                          double *M)
{
    if (N < 1 || n < 0 || n >= N || R < 1 || threads < 1 || threads > 256) return -1;
    if (threads == 1) return oracle_mttkrp(N, dims, nnz, idx, vals, Y, R, n, M);
    const size_t cells = (size_t)dims[n] * (size_t)R;
    struct mt_job *jobs = (struct mt_job *)calloc((size_t)threads, sizeof(struct mt_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    double *priv = (double *)malloc((size_t)threads * cells * sizeof(double));
    if (!jobs || !tid || !priv) { free(jobs); free(tid); free(priv); return -2; }
    int started = 0, rc = 0;
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (struct mt_job){N, R, n, dims, nnz, nnz * (uint64_t)t / (uint64_t)threads,
                                  nnz * (uint64_t)(t + 1) / (uint64_t)threads, idx, vals, Y,
                                  priv + (size_t)t * cells, -3};
        if (pthread_create(&tid[t], NULL, mt_run, &jobs[t]) != 0) { rc = -4; break; }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    for (int t = 0; t < started && rc == 0; ++t)
        if (jobs[t].rc) rc = jobs[t].rc;
    if (rc == 0) {
        memcpy(M, priv, cells * sizeof(double));
        for (int t = 1; t < threads; ++t) {
            const double *p = priv + (size_t)t * cells;
            for (size_t c = 0; c < cells; ++c) M[c] += p[c];
        }
    }
    free(jobs); free(tid); free(priv);
    return rc;
}

/* Same sum, restricted to a list of output rows (for full-size sampling).   */
/* rows[] holds nrows row ids of mode n; M_rows is nrows x R.                */
int oracle_mttkrp_rows(int N, const uint64_t *dims, uint64_t nnz, const uint32_t *idx,
                       const double *vals, const double *const *Y, int R, int n,
                       uint64_t nrows, const uint32_t *rows, double *M_rows)
{
    if (N < 1 || n < 0 || n >= N || R < 1) return -1;
    int64_t *slot = (int64_t *)malloc((size_t)dims[n] * sizeof(int64_t));
    double *ell = (double *)malloc((size_t)R * sizeof(double));
    if (!slot || !ell) { free(slot); free(ell); return -2; }
    for (uint64_t i = 0; i < dims[n]; ++i) slot[i] = -1;
    for (uint64_t q = 0; q < nrows; ++q) {
        if (rows[q] >= dims[n]) { free(slot); free(ell); return -3; }
        slot[rows[q]] = (int64_t)q;
    }
    memset(M_rows, 0, (size_t)nrows * (size_t)R * sizeof(double));
    for (uint64_t e = 0; e < nnz; ++e) {
        int64_t s = slot[idx[(size_t)n * nnz + e]];
        if (s < 0) continue;
        for (int r = 0; r < R; ++r) ell[r] = 1.0;
        for (int w = 0; w < N; ++w) {
            if (w == n) continue;
            const double *row = Y[w] + (size_t)idx[(size_t)w * nnz + e] * (size_t)R;
            for (int r = 0; r < R; ++r) ell[r] *= row[r];
        }
        double *out = M_rows + (size_t)s * (size_t)R;
        for (int r = 0; r < R; ++r) out[r] += vals[e] * ell[r];
    }
    free(slot);
    free(ell);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sampled CP value: out[e] = sum_r prod_w F_w[c_w, r] over ALL modes w.     */
/* With F = the CP factors this is the model value at nonzero e (Eq. 1, the  */
/* CPD sum of outer products, evaluated at one cell).  With F_n replaced by   */
/* an upstream gradient G it is the adjoint of spMTTKRP with respect to the  */
/* nonzero values: d<G, M_n>/d val_e.                                         */
/* ------------------------------------------------------------------------ */
int oracle_sampled(int N, uint64_t nnz, const uint32_t *idx, const double *const *F, int R,
                   double *out)
{
    double *ell = (double *)malloc((size_t)R * sizeof(double));
    if (!ell) return -2;
    for (uint64_t e = 0; e < nnz; ++e) {
        for (int r = 0; r < R; ++r) ell[r] = 1.0;
        for (int w = 0; w < N; ++w) {
            const double *row = F[w] + (size_t)idx[(size_t)w * nnz + e] * (size_t)R;
            for (int r = 0; r < R; ++r) ell[r] *= row[r];
        }
        double s = 0.0;
        for (int r = 0; r < R; ++r) s += ell[r];
        out[e] = s;
    }
    free(ell);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Layout L_n (Section III-B: "the tensor is ordered according to the shard  */
/* IDs of mode n"; Section III-A: every element carries its super-shard and  */
/* shard in each mode).  Reading: with ss_w(x) = c_w(x) div m_w the          */
/* super-shard id of x in mode w, elements are ordered by the key            */
/*   (ss_n, ss_{n-1}, ss_{n-2}, ..., ss_{n+1}, e)      (mode indices mod N)   */
/* so the super-shards of mode n are runs of consecutive positions, shards   */
/* are runs of g positions inside them, and the order inside a super-shard   */
/* follows the super-shards of the other modes.  With all m_w = 1 the key is */
/* the coordinates themselves.  qsort with this comparator is the           */
/* definition.                                                               */
/* ------------------------------------------------------------------------ */
static const uint32_t *g_idx;
static const uint64_t *g_m;
static uint64_t g_nnz;
static int g_N, g_n;

static int cmp_layout(const void *a, const void *b)
{
    uint32_t ea = *(const uint32_t *)a, eb = *(const uint32_t *)b;
    for (int t = 0; t < g_N; ++t) {
        int w = ((g_n - t) % g_N + g_N) % g_N;
        uint64_t ca = g_idx[(size_t)w * g_nnz + ea] / g_m[w];
        uint64_t cb = g_idx[(size_t)w * g_nnz + eb] / g_m[w];
        if (ca != cb) return ca < cb ? -1 : 1;
    }
    return ea < eb ? -1 : (ea > eb ? 1 : 0);
}

/* order[p] = original COO index of the element at position p of L_n;       */
/* m[w] >= 1 is the super-shard width of mode w.                            */
int oracle_layout_order(int N, uint64_t nnz, const uint32_t *idx, const uint64_t *m, int n,
                        uint32_t *order)
{
    if (N < 1 || n < 0 || n >= N || nnz > 0xffffffffull) return -1;
    for (int w = 0; w < N; ++w)
        if (m[w] == 0) return -1;
    for (uint64_t e = 0; e < nnz; ++e) order[e] = (uint32_t)e;
    g_idx = idx;
    g_m = m;
    g_nnz = nnz;
    g_N = N;
    g_n = n;
    qsort(order, (size_t)nnz, sizeof(uint32_t), cmp_layout);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* FLYCOO partition of mode n (Section III-A).                               */
/*  - super-shard j collects the elements whose c_n lies in the interval     */
/*    [j*m, (j+1)*m); there are k = ceil(I/m) of them (the last may be       */
/*    shorter);                                                              */
/*  - ss_ptr[j] = number of elements with c_n < j*m, so super-shard j is     */
/*    positions [ss_ptr[j], ss_ptr[j+1]) of L_n;                             */
/*  - each super-shard is cut into ceil(|SS_j| / g) shards of g consecutive  */
/*    positions, the last one possibly short; shard_ptr lists the shard      */
/*    starts of all super-shards in order and ends with nnz.                 */
/* rows[e] is the mode-n coordinate of element e (any order).                */
/* shard_cap is the capacity of shard_ptr; *S_out receives the shard count.  */
/* ------------------------------------------------------------------------ */
int oracle_partition(uint64_t I, uint64_t nnz, const uint32_t *rows, uint64_t m, uint64_t g,
                     uint64_t *ss_ptr, uint64_t *shard_ptr, uint64_t shard_cap, uint64_t *S_out)
{
    if (m == 0 || g == 0 || I == 0) return -1;
    uint64_t k = (I + m - 1) / m;
    memset(ss_ptr, 0, (size_t)(k + 1) * sizeof(uint64_t));
    for (uint64_t e = 0; e < nnz; ++e) {
        if (rows[e] >= I) return -3;
        ss_ptr[rows[e] / m + 1] += 1;
    }
    for (uint64_t j = 0; j < k; ++j) ss_ptr[j + 1] += ss_ptr[j];
    uint64_t S = 0;
    for (uint64_t j = 0; j < k; ++j) {
        uint64_t size = ss_ptr[j + 1] - ss_ptr[j];
        for (uint64_t q = 0; q * g < size; ++q) {
            if (S >= shard_cap) return -4;
            shard_ptr[S++] = ss_ptr[j] + q * g;
        }
    }
    if (S >= shard_cap) return -4;
    shard_ptr[S] = nnz;
    *S_out = S;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 (super-shard scheduling, longest processing time first).      */
/* Items are sorted by size, descending; equal sizes keep ascending item id. */
/* Each item in that order goes to the bin with the smallest load, the       */
/* lowest bin index on ties; the bin's load grows by the item's size.        */
/* order[] receives the processing order, bin_of[] each item's bin.          */
/* ------------------------------------------------------------------------ */
static const uint64_t *g_size;

static int cmp_lpt(const void *a, const void *b)
{
    uint64_t ia = *(const uint64_t *)a, ib = *(const uint64_t *)b;
    if (g_size[ia] != g_size[ib]) return g_size[ia] > g_size[ib] ? -1 : 1;
    return ia < ib ? -1 : (ia > ib ? 1 : 0);
}

int oracle_lpt(uint64_t nitems, const uint64_t *size, uint64_t nbins, uint64_t *order,
               uint64_t *bin_of, uint64_t *load)
{
    if (nbins == 0) return -1;
    for (uint64_t i = 0; i < nitems; ++i) order[i] = i;
    g_size = size;
    qsort(order, (size_t)nitems, sizeof(uint64_t), cmp_lpt);
    memset(load, 0, (size_t)nbins * sizeof(uint64_t));
    for (uint64_t t = 0; t < nitems; ++t) {
        uint64_t it = order[t];
        uint64_t best = 0;
        for (uint64_t b = 1; b < nbins; ++b)
            if (load[b] < load[best]) best = b;
        bin_of[it] = best;
        load[best] += size[it];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* IEEE binary32 -> bfloat16 by round-to-nearest, ties-to-even; the result  */
/* is returned widened back to binary32 (its low 16 bits are zero).  NaNs   */
/* stay NaN.  This is the rounding of the BF16 factor storage.               */
/* ------------------------------------------------------------------------ */
void oracle_round_bf16(uint64_t n, const float *in, float *out)
{
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, &in[i], 4);
        if ((u & 0x7fffffffu) > 0x7f800000u) {
            u = (u | 0x00400000u) & 0xffff0000u;
        } else {
            uint32_t lsb = (u >> 16) & 1u;
            u = (u + 0x7fffu + lsb) & 0xffff0000u;
        }
        memcpy(&out[i], &u, 4);
    }
}
