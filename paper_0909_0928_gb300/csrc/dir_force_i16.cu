// dir_force_i16.cu -- force kernel instantiations for one storage combination.
#include "dir_force_kernel.cuh"

namespace dirk {

cudaError_t launch_force_i16(int variant, const ForceArgs& a, cudaStream_t s) {
    if (a.field_type == kStoreBF16) return launch_force_types<float, int16_t, bf16>(variant, a, s);
    if (a.field_type == kStoreF32) return launch_force_types<float, int16_t, float>(variant, a, s);
    return cudaErrorInvalidValue;
}

}  // namespace dirk
