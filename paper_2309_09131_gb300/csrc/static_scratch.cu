// static_scratch.cu -- flycoo_spmttkrp_static_scratch: the fused spMTTKRP +
// remap pass with its scratch (the row blocks of super-shards whose shards
// fall into several segments of the schedule) in a fixed, file-scope device
// array instead of the buffer that flycoo_create allocates for the handle.
// The pass is not timed by flycoo_timing_enable: recording events could
// create them, and this entry point creates nothing.
//
// Host code must not pass g_static_scratch itself to a kernel: on the host that
// name is only a stand-in object, not a device address.  The device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call that runs on the device.
#include "internal.cuh"

#include <mutex>

namespace flycoo {
namespace {

// 8 MiB per device, held by every GPU that loads the library until exit.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;
constexpr size_t kStaticScratchFloats = kStaticScratchBytes / sizeof(float);

static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float *g_scratch_dev_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on device `dev`, which the caller has
// made current.  The address is cached only after the current device has been
// read back as `dev`, so a lookup can never be filed under the wrong device.
flycoo_status static_scratch_address(int dev, float **out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("flycoo_spmttkrp_static_scratch: device %d outside [0, %d)", dev, kMaxDevices);
        return FLYCOO_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev_ptr[dev]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess || cur != dev) {
            set_error("flycoo_spmttkrp_static_scratch: device %d is not current (current %d: %s)", dev, cur,
                      cudaGetErrorString(e));
            return FLYCOO_ERR_CUDA;
        }
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("flycoo_spmttkrp_static_scratch: cudaGetSymbolAddress failed on device %d: %s", dev,
                      cudaGetErrorString(e));
            return FLYCOO_ERR_CUDA;
        }
        g_scratch_dev_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_dev_ptr[dev];
    return FLYCOO_OK;
}

} // namespace
} // namespace flycoo

using namespace flycoo;

extern "C" flycoo_status flycoo_spmttkrp_static_scratch(flycoo_handle h, int mode, const void *const *h_factors,
                                                        flycoo_dtype fdt, int R, float *d_out, int next_mode,
                                                        flycoo_stream_t stream) {
    clear_error();
    if (!h) {
        set_error("flycoo_spmttkrp_static_scratch: handle is NULL");
        return FLYCOO_ERR_INVALID_ARG;
    }
    Tensor &t = *h;
    if (mode < 0 || mode >= t.N) {
        set_error("flycoo_spmttkrp_static_scratch: mode %d outside [0, %d)", mode, t.N);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (fdt != FLYCOO_F32 && fdt != FLYCOO_BF16) {
        set_error("flycoo_spmttkrp_static_scratch: unknown factor dtype %d", (int)fdt);
        return FLYCOO_ERR_INVALID_ARG;
    }
    FLY_TRY(check_pass_rank(t, mode, R, "flycoo_spmttkrp_static_scratch"));
    if (next_mode != -1 && next_mode != (mode + 1) % t.N) {
        set_error("flycoo_spmttkrp_static_scratch: next_mode must be -1 or (mode+1) mod N = %d",
                  (mode + 1) % t.N);
        return FLYCOO_ERR_INVALID_ARG;
    }
    if (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15u) || !h_factors) {
        set_error("flycoo_spmttkrp_static_scratch: d_out/h_factors NULL or d_out not 16-byte aligned");
        return FLYCOO_ERR_INVALID_ARG;
    }
    for (int w = 0; w < t.N; ++w) {
        if (w == mode) continue;
        if (!h_factors[w] || (reinterpret_cast<uintptr_t>(h_factors[w]) & 15u)) {
            set_error("flycoo_spmttkrp_static_scratch: factor %d is NULL or not 16-byte aligned", w);
            return FLYCOO_ERR_INVALID_ARG;
        }
    }
    if (t.layout != mode) {
        set_error("flycoo_spmttkrp_static_scratch: tensor is in layout L_%d, mode %d needs L_%d", t.layout, mode,
                  mode);
        return FLYCOO_ERR_LAYOUT;
    }
    const ModeMeta &md = t.mode[mode];
    // one row block (m rows x R floats) per segment of the mode's schedule
    const size_t need = (size_t)md.nseg() * (size_t)md.m * (size_t)R;
    if (need > kStaticScratchFloats) {
        set_error("flycoo_spmttkrp_static_scratch: mode %d has %llu row blocks of %llu-row super-shards; rank %d "
                  "needs %zu bytes of scratch, the static scratch holds %zu bytes (use flycoo_spmttkrp or a "
                  "larger shard size g)",
                  mode, (unsigned long long)md.nseg(), (unsigned long long)md.m, R, need * sizeof(float),
                  kStaticScratchBytes);
        return FLYCOO_ERR_INVALID_ARG;
    }
    DeviceGuard dg(t.device);
    FLY_TRY(dg.status("flycoo_spmttkrp_static_scratch"));
    FLY_TRY(check_usable(t, "flycoo_spmttkrp_static_scratch"));
    float *scratch = nullptr;
    FLY_TRY(static_scratch_address(t.device, &scratch));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (t.nnz == 0) {
        FLY_TRY_CUDA(cudaMemsetAsync(d_out, 0, (size_t)t.dims[mode] * R * sizeof(float), s));
        if (next_mode >= 0) t.layout = next_mode;
        return FLYCOO_OK;
    }
    const FusedArgs a = fused_args(t, mode, h_factors, d_out, next_mode >= 0, scratch);
    FLY_TRY(launch_fused(t.N, R, fdt, a, s));
    FLY_TRY(launch_fixup(R, fixup_args(t, mode, d_out, scratch), s));
    if (next_mode >= 0) {
        t.cur = 1 - t.cur;
        t.remap_since_sync = true;
        t.layout = next_mode;
    }
    return FLYCOO_OK;
}
