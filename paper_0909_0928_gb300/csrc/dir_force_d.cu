// dir_force_d.cu -- kernels and launchers of the Eqs. (3)-(6) split iteration
// with the difference image formed once per voxel (block functions in
// dir_split_d.cuh): the z + D pass and the stencil force pass.
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_split_d.cuh"

namespace dirk {

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, 4)
    force_zd_kernel(const __grid_constant__ CUtensorMap tmap, const ForceArgs a, const Taps taps) {
    zd_block<V, FTZ, TI>(&tmap, a, taps, BlockPos::of_grid());
}

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, 4)
    force_st_kernel(const __grid_constant__ CUtensorMap dmap,
                    const __grid_constant__ CUtensorMap smap,
                    const __grid_constant__ CUtensorMap umap,
                    const __grid_constant__ CUtensorMap emap, const ForceArgs a) {
    st_block<V, FTZ, TI>(&dmap, &smap, &umap, &emap, a, BlockPos::of_grid());
}

namespace {

// 4-D tiled map over a pitched volume of ncomp components (esz-byte elements)
bool map4(CUtensorMap* m, CUtensorMapDataType t, const void* p, const Grid3& g, int ncomp, int esz,
          int bx, int by, int bz) {
    EncodeTiledFn enc = encode_fn();
    if (!enc || p == nullptr) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz,
                                (cuuint64_t)ncomp};
    const cuuint64_t str[3] = {(cuuint64_t)g.px * esz, (cuuint64_t)g.plane * esz,
                               (cuuint64_t)g.cs * esz};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, (cuuint32_t)ncomp};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    return enc(m, t, 4, const_cast<void*>(p), dims, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

dim3 brick_grid(const Grid3& g, int ftz) {
    return dim3((g.nx + FTX - 1) / FTX, (g.ny + FTY - 1) / FTY, (g.nz + ftz - 1) / ftz);
}

template <int V, int FTZ, typename TI>
cudaError_t launch_zd(const ForceArgs& a, const Taps& taps, cudaStream_t s) {
    using Z = ZDGeom<FTZ>;
    CUtensorMap tmap;
    if (!map4(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.u, a.g, 3, 4, FTX, FTY, Z::NPZ))
        return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    const cudaError_t e = setup_kernel(setup, force_zd_kernel<V, FTZ, TI>, Z::SMEM);
    if (e != cudaSuccess) return e;
    return launch_ex(force_zd_kernel<V, FTZ, TI>, brick_grid(a.g, FTZ), dim3(FTX, FTY, 1), Z::SMEM,
                     s, a.pdl, tmap, a, taps);
}

template <int V, int FTZ, typename TI>
cudaError_t launch_st(const ForceArgs& a, cudaStream_t s) {
    using F = STGeom<FTZ, V, TI>;
    CUtensorMap dmap, smap, umap, emap;
    if (!map4(&dmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.dbuf, a.g, 1, 4, F::DW, F::DH, F::DD) ||
        !map4(&smap, tma_type<TI>(), a.S, a.g, 1, (int)sizeof(TI), F::FSW, FSH, F::DD) ||
        !map4(&umap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.u, a.g, 3, 4, FTX, FTY, FTZ))
        return cudaErrorInvalidValue;
    if (F::IC) {
        if (!map4(&emap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.dbuf2, a.g, 1, 4, FTX, FTY, FTZ))
            return cudaErrorInvalidValue;
    } else {
        emap = umap;  // not read
    }
    static KernelSetup setup;  // per instantiation
    const cudaError_t e = setup_kernel(setup, force_st_kernel<V, FTZ, TI>, F::SMEM);
    if (e != cudaSuccess) return e;
    return launch_ex(force_st_kernel<V, FTZ, TI>, brick_grid(a.g, FTZ), dim3(FTX, FTY, 1), F::SMEM,
                     s, a.pdl, dmap, smap, umap, emap, a);
}

template <int V, typename TI>
cudaError_t launch_d_pair(const ForceArgs& zd, const ForceArgs& st, const Taps& taps,
                          cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (zd.depth) {
        case 8: e = launch_zd<V, 8, TI>(zd, taps, s); break;
        case 6:
        case 4: e = launch_zd<V, 4, TI>(zd, taps, s); break;
        case 2: e = launch_zd<V, 2, TI>(zd, taps, s); break;
        case 1: e = launch_zd<V, 1, TI>(zd, taps, s); break;
        default: break;
    }
    if (e != cudaSuccess) return e;
    switch (st.depth) {
        case 8: return launch_st<V, 8, TI>(st, s);
        case 6:
        case 4: return launch_st<V, 4, TI>(st, s);
        case 2: return launch_st<V, 2, TI>(st, s);
        case 1: return launch_st<V, 1, TI>(st, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename TI>
cudaError_t launch_d_types(int variant, const ForceArgs& zd, const ForceArgs& st,
                           const Taps& taps, cudaStream_t s) {
    switch (variant) {
        case 2: return launch_d_pair<2, TI>(zd, st, taps, s);
        case 3: return launch_d_pair<3, TI>(zd, st, taps, s);
        case 4: return launch_d_pair<4, TI>(zd, st, taps, s);
        case 5: return launch_d_pair<5, TI>(zd, st, taps, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool force_d_supported(int variant, const ForceArgs& a, const Taps& taps) {
    return variant >= 2 && variant <= 5 && force_zs_supported(variant, a, taps);
}

int force_d_planes(int variant) { return variant == 5 ? 5 : 4; }

// Brick depth of both kernels: 8 where such bricks still number four per SM,
// else the deepest of 4 and 2 that gives one per SM, else 1 -- 8, 4 and 2 on
// the 256x256x100 pyramid, the autotuner's choice there for Eq. 3 and Eq. 6
// (Eq. 3: 10.46 ms per registration against 10.63 with 4 on every level)
int force_d_depth(const Grid3& g, int num_sms) {
    const long long bxy = (long long)((g.nx + FTX - 1) / FTX) * ((g.ny + FTY - 1) / FTY);
    if (bxy * ((g.nz + 7) / 8) >= 4LL * num_sms) return 8;
    for (int d = 4; d >= 2; d /= 2)
        if (bxy * ((g.nz + d - 1) / d) >= num_sms) return d;
    return 1;
}

cudaError_t launch_force_d(int variant, const ForceArgs& zd, const ForceArgs& st, const Taps& taps,
                           cudaStream_t s) {
    if (!force_d_supported(variant, zd, taps) || zd.dbuf == nullptr ||
        (variant == 5 && zd.dbuf2 == nullptr))
        return cudaErrorInvalidValue;
    if (zd.img_type == kStoreF32) return launch_d_types<float>(variant, zd, st, taps, s);
    return launch_d_types<int16_t>(variant, zd, st, taps, s);
}

}  // namespace dirk
