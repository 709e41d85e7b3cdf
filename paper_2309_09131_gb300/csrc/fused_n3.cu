// fused_n3.cu -- instantiations of the fused spMTTKRP + remap kernel for 3-mode tensors.
#include "fused.cuh"

namespace flycoo {
flycoo_status launch_fused_n3(int R, flycoo_dtype dt, const FusedArgs &a, cudaStream_t s) {
    return launch_fused_dispatch<3>(R, dt, a, s);
}
} // namespace flycoo
