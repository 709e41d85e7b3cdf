// fused_n4.cu -- instantiations of the fused spMTTKRP + remap kernel for 4-mode tensors.
#include "fused.cuh"

namespace flycoo {
flycoo_status launch_fused_n4(int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s) {
    return launch_fused_dispatch<4>(R, dt, a, s);
}
} // namespace flycoo
