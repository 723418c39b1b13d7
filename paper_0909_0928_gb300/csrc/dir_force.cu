// dir_force.cu -- dispatch of the force kernel over storage types, and its
// launch shape (see dir_force_kernel.cuh for the kernel).
#include "dir_force_kernel.cuh"

namespace dirk {

// Brick depth: the deepest of 8, 4, 2, 1 that still gives at least
// min_blocks blocks.  The TMA-fed force kernels fetch a whole brick per copy,
// so deeper bricks (fewer, longer blocks) pay off down to about one block per
// SM (measured with dir_autotune on the 256x256x100 pyramid).
int force_brick_depth(const Grid3& g, int min_blocks) {
    const long long bxy = (long long)((g.nx + FTX - 1) / FTX) * ((g.ny + FTY - 1) / FTY);
    for (int d = 8; d > 1; d /= 2)
        if (bxy * ((g.nz + d - 1) / d) >= min_blocks) return d;
    return 1;
}

cudaError_t launch_force(int variant, bool fp64, const ForceArgs& a, cudaStream_t s, bool plain) {
    if (fp64) {
        if (a.img_type != kStoreF64 || a.field_type != kStoreF64) return cudaErrorInvalidValue;
        return launch_force_f64(variant, a, s);
    }
    if (a.img_type == kStoreI16) {
        // TMA-fed bricks (Eqs. 1-6) unless the plain kernel is asked for
        const cudaError_t e = plain ? cudaErrorNotSupported : launch_force_tma(variant, a, s);
        if (e != cudaErrorNotSupported) return e;
        return launch_force_i16(variant, a, s);
    }
    if (a.img_type != kStoreF32) return cudaErrorInvalidValue;
    if (a.field_type == kStoreBF16) return launch_force_bf16(variant, a, s);
    if (a.field_type == kStoreF32) {
        const cudaError_t e = plain ? cudaErrorNotSupported : launch_force_tma(variant, a, s);
        if (e != cudaErrorNotSupported) return e;
        return launch_force_f32(variant, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dirk
