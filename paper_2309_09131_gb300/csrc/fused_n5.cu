// fused_n5.cu -- instantiations of the fused spMTTKRP + remap kernel for 5-mode tensors.
#include "fused.cuh"

namespace flycoo {
flycoo_status launch_fused_n5(int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s) {
    return launch_fused_dispatch<5>(R, dt, a, s);
}
} // namespace flycoo
