// dir_force_zs.cu -- the one-volume kernels and launchers of the split
// iteration schedule's z + force pass (block functions in dir_split.cuh).
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_split.cuh"

namespace dirk {

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, 4)
    force_zs_kernel(const __grid_constant__ CUtensorMap tmap,
                    const __grid_constant__ CUtensorMap smap,
                    const __grid_constant__ CUtensorMap mmap, const ForceArgs a, const Taps taps) {
    zs_block<V, FTZ, TI>(&tmap, &smap, &mmap, a, taps, BlockPos::of_grid());
}

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, FTZ >= 2 ? 3 : 4)
    force_gzs_kernel(const __grid_constant__ CUtensorMap tmap,
                     const __grid_constant__ CUtensorMap smap,
                     const __grid_constant__ CUtensorMap mmap, const ForceArgs a, const Taps taps) {
    gzs_block<V, FTZ, TI>(&tmap, &smap, &mmap, a, taps, BlockPos::of_grid());
}

template <typename TI>
static bool make_zs_maps(CUtensorMap* tmap, CUtensorMap* smap, CUtensorMap* mmap,
                         const ForceArgs& a, int ftz) {
    constexpr int FSW = FZGeom<1, 0, TI>::FSW;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const Grid3& g = a.g;
    const cuuint64_t tdims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
    const cuuint64_t idims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 1};
    const cuuint64_t tstr[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                (cuuint64_t)g.cs * 4};
    const cuuint64_t istr[3] = {(cuuint64_t)g.px * sizeof(TI), (cuuint64_t)g.plane * sizeof(TI),
                                (cuuint64_t)g.cs * sizeof(TI)};
    const cuuint32_t tbox[4] = {(cuuint32_t)FTX, (cuuint32_t)FTY, (cuuint32_t)(ftz + 2 * FZR), 3u};
    const cuuint32_t ibox[4] = {(cuuint32_t)FSW, (cuuint32_t)FZSH, (cuuint32_t)(ftz + 2), 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    auto enc4 = [&](CUtensorMap* m, CUtensorMapDataType t, const void* p, const cuuint64_t* d,
                    const cuuint64_t* st, const cuuint32_t* b) {
        return enc(m, t, 4, const_cast<void*>(p), d, st, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    return enc4(tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.u, tdims, tstr, tbox) &&
           enc4(smap, tma_type<TI>(), a.S, idims, istr, ibox) &&
           enc4(mmap, tma_type<TI>(), a.M, idims, istr, ibox);
}

template <int V, int FTZ, typename TI>
static cudaError_t launch_zs(const ForceArgs& a, const Taps& taps, cudaStream_t s) {
    using F = FZGeom<FTZ, V, TI>;
    CUtensorMap tmap, smap, mmap;
    if (!make_zs_maps<TI>(&tmap, &smap, &mmap, a, FTZ)) return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    const cudaError_t e = setup_kernel(setup, force_zs_kernel<V, FTZ, TI>, F::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.g.nx + FTX - 1) / FTX, (a.g.ny + FTY - 1) / FTY, (a.g.nz + FTZ - 1) / FTZ);
    return launch_ex(force_zs_kernel<V, FTZ, TI>, grid, dim3(FTX, FTY, 1), F::SMEM, s, a.pdl, tmap,
                     smap, mmap, a, taps);
}

template <typename TI>
static cudaError_t launch_zs_types(int variant, const ForceArgs& a, const Taps& taps,
                                   cudaStream_t s) {
    switch (a.depth) {
        case 8: return variant ? launch_zs<1, 8, TI>(a, taps, s) : launch_zs<0, 8, TI>(a, taps, s);
        case 6: return variant ? launch_zs<1, 6, TI>(a, taps, s) : launch_zs<0, 6, TI>(a, taps, s);
        case 4: return variant ? launch_zs<1, 4, TI>(a, taps, s) : launch_zs<0, 4, TI>(a, taps, s);
        case 2: return variant ? launch_zs<1, 2, TI>(a, taps, s) : launch_zs<0, 2, TI>(a, taps, s);
        case 1: return variant ? launch_zs<1, 1, TI>(a, taps, s) : launch_zs<0, 1, TI>(a, taps, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int V, int FTZ, typename TI>
static cudaError_t launch_gzs(const ForceArgs& a, const Taps& taps, cudaStream_t s) {
    using F = FGGeom<FTZ, V, TI>;
    using Z = GZGeom<FTZ, V, TI>;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorInvalidValue;
    const Grid3& g = a.g;
    const cuuint64_t tdims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
    const cuuint64_t idims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 1};
    const cuuint64_t tstr[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                (cuuint64_t)g.cs * 4};
    const cuuint64_t istr[3] = {(cuuint64_t)g.px * sizeof(TI), (cuuint64_t)g.plane * sizeof(TI),
                                (cuuint64_t)g.cs * sizeof(TI)};
    const cuuint32_t tbox[4] = {(cuuint32_t)F::UW, (cuuint32_t)F::UH, (cuuint32_t)Z::NPZ, 3u};
    const cuuint32_t ibox[4] = {(cuuint32_t)F::FSW, (cuuint32_t)FSH, (cuuint32_t)F::UD, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    auto enc4 = [&](CUtensorMap* m, CUtensorMapDataType t, const void* p, const cuuint64_t* d,
                    const cuuint64_t* st, const cuuint32_t* b) {
        return enc(m, t, 4, const_cast<void*>(p), d, st, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap tmap, smap, mmap;
    if (!enc4(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.u, tdims, tstr, tbox) ||
        !enc4(&smap, tma_type<TI>(), a.S, idims, istr, ibox) ||
        !enc4(&mmap, tma_type<TI>(), a.M, idims, istr, ibox))
        return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    const cudaError_t e = setup_kernel(setup, force_gzs_kernel<V, FTZ, TI>, Z::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.nx + FTX - 1) / FTX, (g.ny + FTY - 1) / FTY, (g.nz + FTZ - 1) / FTZ);
    return launch_ex(force_gzs_kernel<V, FTZ, TI>, grid, dim3(FTX, FTY, 1), Z::SMEM, s, a.pdl, tmap,
                     smap, mmap, a, taps);
}

template <int V, typename TI>
static cudaError_t launch_gzs_depth(const ForceArgs& a, const Taps& taps, cudaStream_t s) {
    switch (a.depth) {
        case 8:
        case 6:
        case 4: return launch_gzs<V, 4, TI>(a, taps, s);  // at most 4 deep, as force_tma_gm_kernel
        case 2: return launch_gzs<V, 2, TI>(a, taps, s);
        case 1: return launch_gzs<V, 1, TI>(a, taps, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename TI>
static cudaError_t launch_gzs_types(int variant, const ForceArgs& a, const Taps& taps,
                                    cudaStream_t s) {
    switch (variant) {
        case 2: return launch_gzs_depth<2, TI>(a, taps, s);
        case 3: return launch_gzs_depth<3, TI>(a, taps, s);
        case 4: return launch_gzs_depth<4, TI>(a, taps, s);
        case 5: return launch_gzs_depth<5, TI>(a, taps, s);
        default: return cudaErrorInvalidValue;
    }
}

// Brick depth: Eq. 1 takes 6 planes where that still gives four waves of
// blocks -- the brick of t with its 2R halo planes and the S box then fit four
// blocks per SM in shared memory instead of three (measured on 256x256x100:
// 65.4 us against 70.3 us at depth 8); otherwise, and for Eq. 2 with its M box,
// the force pass's usual depth.
int force_zs_depth(int variant, const Grid3& g, int num_sms) {
    const long long bxy = (long long)((g.nx + FTX - 1) / FTX) * ((g.ny + FTY - 1) / FTY);
    if (variant == 0 && bxy * ((g.nz + 5) / 6) >= 4LL * 4 * num_sms) return 6;
    return force_brick_depth(g, num_sms);
}

bool force_zs_supported(int variant, const ForceArgs& a, const Taps& taps) {
    return variant >= 0 && variant <= 5 && a.field_type == kStoreF32 &&
           (a.img_type == kStoreF32 || a.img_type == kStoreI16) && taps.R == FZR;
}

cudaError_t launch_force_zs(int variant, const ForceArgs& a, const Taps& taps, cudaStream_t s) {
    if (!force_zs_supported(variant, a, taps)) return cudaErrorInvalidValue;
    if (variant >= 2) {
        if (a.img_type == kStoreF32) return launch_gzs_types<float>(variant, a, taps, s);
        return launch_gzs_types<int16_t>(variant, a, taps, s);
    }
    if (a.img_type == kStoreF32) return launch_zs_types<float>(variant, a, taps, s);
    return launch_zs_types<int16_t>(variant, a, taps, s);
}

}  // namespace dirk
