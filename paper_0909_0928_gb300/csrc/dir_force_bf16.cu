// dir_force_bf16.cu -- force kernel instantiations for one storage combination.
#include "dir_force_kernel.cuh"

namespace dirk {

cudaError_t launch_force_bf16(int variant, const ForceArgs& a, cudaStream_t s) {
    return launch_force_types<float, float, bf16>(variant, a, s);
}

}  // namespace dirk
