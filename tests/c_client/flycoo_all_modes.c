/*
 * A plain C99 client of the FLYCOO library: no Python, no PyTorch.
 *
 * Reads a sparse tensor and its factor matrices from a binary file, converts
 * the tensor to FLYCOO (flycoo_create), runs the spMTTKRP of every mode with
 * the remap to the next mode fused into each pass (Algorithm 2), checks that
 * the tensor is back in layout L_0, and writes the N outputs to a file.  It
 * also runs the host-only planner on mode 0's exported super-shard pointers
 * and checks that it reproduces the handle's shards and shard schedule.
 *
 *   flycoo_all_modes <in.bin> <out.bin>
 *
 * in.bin (little-endian): uint32 N, uint32 R, uint64 nnz, uint64 dims[N],
 *   uint32 idx[N * nnz] (mode-major), float vals[nnz], then for w = 0..N-1
 *   float Y_w[dims[w] * R] (row-major).
 * out.bin: for n = 0..N-1, float M_n[dims[n] * R] (row-major).
 *
 * Exit status: 0 on success, 10 + the flycoo_status of a failed library call,
 * 2 for a file or CUDA runtime error, 3 when a check fails.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "flycoo.h"

#define CHECK_FLY(call)                                                                   \
    do {                                                                                  \
        flycoo_status st_ = (call);                                                       \
        if (st_ != FLYCOO_OK) {                                                           \
            fprintf(stderr, "%s: status %d: %s\n", #call, (int)st_, flycoo_last_error()); \
            exit(10 + (int)st_);                                                          \
        }                                                                                 \
    } while (0)

#define CHECK_CUDA(call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));                   \
            exit(2);                                                                      \
        }                                                                                 \
    } while (0)

static void read_exact(FILE *f, void *p, size_t bytes) {
    if (bytes && fread(p, 1, bytes, f) != bytes) {
        fprintf(stderr, "short read\n");
        exit(2);
    }
}

static void *xmalloc(size_t bytes) {
    void *p = malloc(bytes ? bytes : 1);
    if (!p) {
        fprintf(stderr, "out of host memory\n");
        exit(2);
    }
    return p;
}

static void *to_device(const void *h, size_t bytes) {
    void *d = NULL;
    CHECK_CUDA(cudaMalloc(&d, bytes ? bytes : 16));
    if (bytes) CHECK_CUDA(cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice));
    return d;
}

int main(int argc, char **argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s <in.bin> <out.bin>\n", argv[0]);
        return 2;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) {
        perror(argv[1]);
        return 2;
    }
    uint32_t N = 0, R = 0;
    uint64_t nnz = 0;
    read_exact(in, &N, 4);
    read_exact(in, &R, 4);
    read_exact(in, &nnz, 8);
    if (N < 1 || N > FLYCOO_MAX_MODES) {
        fprintf(stderr, "bad N\n");
        return 2;
    }
    uint64_t dims[FLYCOO_MAX_MODES];
    read_exact(in, dims, 8 * (size_t)N);
    uint32_t *idx = xmalloc(4 * (size_t)N * nnz);
    float *vals = xmalloc(4 * (size_t)nnz);
    read_exact(in, idx, 4 * (size_t)N * nnz);
    read_exact(in, vals, 4 * (size_t)nnz);
    void *d_factors[FLYCOO_MAX_MODES];
    float *d_out[FLYCOO_MAX_MODES];
    for (uint32_t w = 0; w < N; ++w) {
        size_t bytes = 4 * (size_t)dims[w] * R;
        float *h = xmalloc(bytes);
        read_exact(in, h, bytes);
        d_factors[w] = to_device(h, bytes);
        free(h);
        CHECK_CUDA(cudaMalloc((void **)&d_out[w], bytes));
    }
    fclose(in);

    /* FLYCOO conversion: the COO input is copied, so it can be freed after */
    void *d_idx = to_device(idx, 4 * (size_t)N * nnz);
    void *d_vals = to_device(vals, 4 * (size_t)nnz);
    flycoo_handle h = NULL;
    CHECK_FLY(flycoo_create((int)N, dims, nnz, (const uint32_t *)d_idx, (const float *)d_vals, NULL, NULL, &h));
    CHECK_CUDA(cudaFree(d_idx));
    CHECK_CUDA(cudaFree(d_vals));
    free(idx);
    free(vals);

    /* one all-mode sweep: mode n in layout L_n, remapped to L_{n+1} in the pass */
    for (uint32_t n = 0; n < N; ++n)
        CHECK_FLY(flycoo_spmttkrp(h, (int)n, (const void *const *)d_factors, FLYCOO_F32, (int)R, d_out[n],
                                  (int)((n + 1) % N), NULL));
    CHECK_FLY(flycoo_sync(h, NULL));
    flycoo_info info;
    CHECK_FLY(flycoo_get_info(h, &info));
    if (info.layout_mode != 0) {
        fprintf(stderr, "the sweep ended in layout %d, not 0\n", (int)info.layout_mode);
        return 3;
    }

    /* the host-only planner reproduces the handle's mode-0 shards and schedule */
    {
        const uint64_t k = info.super_shards[0], S = info.shards[0];
        uint64_t *ss_ptr = xmalloc(8 * (k + 1)), *shard_ptr = xmalloc(8 * (S + 1));
        uint64_t *bin_ptr = xmalloc(8 * ((uint64_t)info.bins + 1)), *items = xmalloc(8 * (S ? S : 1));
        uint32_t *shard_ss = xmalloc(4 * (S ? S : 1));
        CHECK_FLY(flycoo_export_partition(h, 0, ss_ptr, shard_ptr, shard_ss));
        CHECK_FLY(flycoo_export_schedule(h, 0, 1, bin_ptr, items));
        flycoo_plan p = NULL;
        CHECK_FLY(flycoo_plan_create(nnz, k, ss_ptr, info.g, info.bins, info.schedule, &p));
        uint64_t cnt = 0;
        CHECK_FLY(flycoo_plan_get(p, FLYCOO_PLAN_SHARD_PTR, NULL, &cnt));
        const uint64_t cap = (S + 1 > (uint64_t)info.bins + 1) ? S + 1 : (uint64_t)info.bins + 1;
        uint64_t *buf = xmalloc(8 * cap);
        int ok = cnt == S + 1;
        if (ok) {
            CHECK_FLY(flycoo_plan_get(p, FLYCOO_PLAN_SHARD_PTR, buf, &cnt));
            ok = memcmp(buf, shard_ptr, 8 * cnt) == 0;
        }
        if (ok) {
            cnt = cap;
            CHECK_FLY(flycoo_plan_get(p, FLYCOO_PLAN_SHARD_ITEMS, buf, &cnt));
            ok = cnt == S && memcmp(buf, items, 8 * S) == 0;
        }
        if (ok) {
            cnt = cap;
            CHECK_FLY(flycoo_plan_get(p, FLYCOO_PLAN_SHARD_BIN_PTR, buf, &cnt));
            ok = cnt == (uint64_t)info.bins + 1 && memcmp(buf, bin_ptr, 8 * cnt) == 0;
        }
        flycoo_plan_destroy(p);
        free(buf);
        free(ss_ptr);
        free(shard_ptr);
        free(bin_ptr);
        free(items);
        free(shard_ss);
        if (!ok) {
            fprintf(stderr, "the planner does not reproduce the handle's mode-0 schedule\n");
            return 3;
        }
    }

    FILE *out = fopen(argv[2], "wb");
    if (!out) {
        perror(argv[2]);
        return 2;
    }
    for (uint32_t n = 0; n < N; ++n) {
        size_t bytes = 4 * (size_t)dims[n] * R;
        float *hbuf = xmalloc(bytes);
        CHECK_CUDA(cudaMemcpy(hbuf, d_out[n], bytes, cudaMemcpyDeviceToHost));
        if (fwrite(hbuf, 1, bytes, out) != bytes) {
            fprintf(stderr, "short write\n");
            return 2;
        }
        free(hbuf);
        CHECK_CUDA(cudaFree(d_out[n]));
        CHECK_CUDA(cudaFree(d_factors[n]));
    }
    fclose(out);
    flycoo_destroy(h);
    printf("ok N=%u R=%u nnz=%llu shards0=%llu\n", N, R, (unsigned long long)nnz,
           (unsigned long long)info.shards[0]);
    return 0;
}
