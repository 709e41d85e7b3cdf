// static_scratch.cu -- flycoo_spmttkrp_static_scratch: the fused spMTTKRP +
// remap pass with its scratch (the per-shard row blocks of super-shards that
// span several shards) in a fixed, file-scope device array instead of the
// buffer that flycoo_create allocates for the handle.
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

// Device address of g_static_scratch on device `dev` (which must be current).
flycoo_status static_scratch_address(int dev, float **out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("flycoo_spmttkrp_static_scratch: device %d outside [0, %d)", dev, kMaxDevices);
        return FLYCOO_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
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

struct ScratchDeviceGuard {
    int prev = -1;
    explicit ScratchDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~ScratchDeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

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
    if (R != 16 && R != 32 && R != 64) {
        set_error("flycoo_spmttkrp_static_scratch: rank %d not built (16, 32 or 64)", R);
        return R > 0 ? FLYCOO_ERR_UNSUPPORTED : FLYCOO_ERR_INVALID_ARG;
    }
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
    // one row block (m rows x R floats) per shard
    const size_t need = (size_t)md.S * (size_t)md.m * (size_t)R;
    if (need > kStaticScratchFloats) {
        set_error("flycoo_spmttkrp_static_scratch: mode %d has %llu shards of %llu-row super-shards; rank %d "
                  "needs %zu bytes of scratch, the static scratch holds %zu bytes (use flycoo_spmttkrp or a "
                  "larger shard size g)",
                  mode, (unsigned long long)md.S, (unsigned long long)md.m, R, need * sizeof(float),
                  kStaticScratchBytes);
        return FLYCOO_ERR_INVALID_ARG;
    }
    ScratchDeviceGuard dg(t.device);
    FLY_TRY(check_usable(t, "flycoo_spmttkrp_static_scratch"));
    float *scratch = nullptr;
    FLY_TRY(static_scratch_address(t.device, &scratch));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (t.nnz == 0) {
        FLY_TRY_CUDA(cudaMemsetAsync(d_out, 0, (size_t)t.dims[mode] * R * sizeof(float), s));
        if (next_mode >= 0) t.layout = next_mode;
        return FLYCOO_OK;
    }
    FusedArgs a{};
    a.elem_in = t.elem[t.cur].p;
    a.elem_out = next_mode >= 0 ? t.elem[1 - t.cur].p : nullptr;
    a.next = next_mode >= 0 ? md.d_next.as<u32>() : nullptr;
    for (int q = 1; q < t.N; ++q) a.Y[q - 1] = h_factors[(mode + q) % t.N];
    a.out = d_out;
    for (int z = 0; z < 2; ++z) {
        a.tiles[z] = md.d_tiles[z].as<uint4>();
        a.tile_bin_ptr[z] = md.d_tile_bin_ptr[z].as<u32>();
    }
    a.partials = scratch;
    a.err = t.err.as<u32>();
    a.I_out = (u32)t.dims[mode];
    a.m = (u32)md.m;
    a.bins = t.bins;
    a.wait_limit = t.wait_limit;
    FLY_TRY(launch_fused(t.N, R, fdt, a, s));
    FixupArgs f{};
    f.items = md.d_k4.as<u32>();
    f.nitems = (u32)md.k4_items.size();
    f.ss_shard_ptr = md.d_ss_shard_ptr.as<u32>();
    f.partials = a.partials;
    f.out = d_out;
    f.I_out = a.I_out;
    f.m = a.m;
    FLY_TRY(launch_fixup(R, f, s));
    if (next_mode >= 0) {
        t.cur = 1 - t.cur;
        t.remap_since_sync = true;
        t.layout = next_mode;
    }
    return FLYCOO_OK;
}
