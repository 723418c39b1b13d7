// dir_force_f64.cu -- force kernel instantiations for one storage combination.
#include "dir_force_kernel.cuh"

namespace dirk {

cudaError_t launch_force_f64(int variant, const ForceArgs& a, cudaStream_t s) {
    return launch_force_types<double, double, double>(variant, a, s);
}

}  // namespace dirk
