// dir_grouped.cu -- grouped launches of the split iteration schedule: one
// x/y kernel and one z + force kernel per iteration over the same pyramid
// level of several registrations (the batched form).  A block finds its job
// from the prefix sums of the jobs' block counts and runs the same block
// function as the one-volume kernels (dir_split.cuh) on that job's tensor
// maps and arguments, so every job's field is bit for bit the one of its own
// registration.  The coarse levels are bound by the fixed latencies of a
// launch (copy, compute, reduce, then the next kernel waits for the slowest
// block); a grouped launch pays them once for all the jobs of a step.
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_launch.h"
#include "dir_split.cuh"
#include "dir_split_d.cuh"

namespace dirk {

static_assert(sizeof(XYGroup) < 30000 && sizeof(ZSGroup) < 30000 && sizeof(ZDGroup) < 30000 &&
                  sizeof(STGroup) < 30000,
              "grouped launch parameters must fit the kernel parameter space");

__device__ __forceinline__ int group_job(const int* first, int n, int b) {
    int j = 0;
    while (j + 1 < n && b >= first[j + 1]) ++j;
    return j;
}

__device__ __forceinline__ BlockPos group_pos(int lb, int gx, int gy, int gz) {
    return {lb % gx, (lb / gx) % gy, lb / (gx * gy), gx, gy, gz};
}

template <int TY>
__global__ void __launch_bounds__(8 * TY)
    smooth_xy_grouped_kernel(const __grid_constant__ XYGroup G) {
    const int b = blockIdx.x;
    const int j = group_job(G.first, G.n, b);
    sxy_block<FZR, TY>(&G.map[j], G.a[j], G.zchunk,
                       group_pos(b - G.first[j], G.gx[j], G.gy[j], G.gz[j]));
}

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, (V >= 2 && FTZ >= 2) ? 3 : 4)
    force_zs_grouped_kernel(const __grid_constant__ ZSGroup G) {
    const int b = blockIdx.x;
    const int j = group_job(G.first, G.n, b);
    const BlockPos bp = group_pos(b - G.first[j], G.gx[j], G.gy[j], G.gz[j]);
    if constexpr (V <= 1)
        zs_block<V, FTZ, TI>(&G.tmap[j], &G.smap[j], &G.mmap[j], G.a[j], G.taps, bp);
    else
        gzs_block<V, FTZ, TI>(&G.tmap[j], &G.smap[j], &G.mmap[j], G.a[j], G.taps, bp);
}

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, 4) force_zd_grouped_kernel(const __grid_constant__ ZDGroup G) {
    const int b = blockIdx.x;
    const int j = group_job(G.first, G.n, b);
    zd_block<V, FTZ, TI>(&G.tmap[j], G.a[j], G.taps,
                         group_pos(b - G.first[j], G.gx[j], G.gy[j], G.gz[j]));
}

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, 4) force_st_grouped_kernel(const __grid_constant__ STGroup G) {
    const int b = blockIdx.x;
    const int j = group_job(G.first, G.n, b);
    st_block<V, FTZ, TI>(&G.dmap[j], &G.smap[j], &G.umap[j], &G.emap[j], G.a[j],
                         group_pos(b - G.first[j], G.gx[j], G.gy[j], G.gz[j]));
}

// x/y kernel shared memory of a tile height
static int sxy_smem(int ty) { return ty == 32 ? SXYSmem<FZR, 32>::SMEM : SXYSmem<FZR, S2Y>::SMEM; }

void group_shapes(int variant, const Grid3* grids, int n, int num_sms, int* ty, int* zchunk,
                  int* depth) {
    // tile rows: 32 where the group has enough tall tiles to fill the GPU
    long long tall = 0;
    for (int j = 0; j < n; ++j)
        tall += (long long)((grids[j].nx + S2X - 1) / S2X) * ((grids[j].ny + 31) / 32) * 3 *
                grids[j].nz;
    *ty = tall >= 8LL * num_sms ? 32 : S2Y;
    // z chunk: the longest of 4, 2, 1 planes that still gives a wave of blocks
    static KernelSetup s32, s16;
    int per_sm = 1;
    if (*ty == 32)
        setup_kernel(s32, smooth_xy_grouped_kernel<32>, sxy_smem(32), 8 * 32, &per_sm);
    else
        setup_kernel(s16, smooth_xy_grouped_kernel<S2Y>, sxy_smem(S2Y), 8 * S2Y, &per_sm);
    const long long slots = (long long)(per_sm < 1 ? 1 : per_sm) * num_sms;
    *zchunk = 1;
    for (int c = 4; c > 1; c /= 2) {
        long long blocks = 0;
        for (int j = 0; j < n; ++j)
            blocks += (long long)((grids[j].nx + S2X - 1) / S2X) *
                      ((grids[j].ny + *ty - 1) / *ty) * 3 * ((grids[j].nz + c - 1) / c);
        if (blocks >= slots) {
            *zchunk = c;
            break;
        }
    }
    // brick depth: the one-volume rules (force_zs_depth, force_brick_depth) on
    // the group's total block count
    auto bricks = [&](int d) {
        long long b = 0;
        for (int j = 0; j < n; ++j)
            b += (long long)((grids[j].nx + FTX - 1) / FTX) * ((grids[j].ny + FTY - 1) / FTY) *
                 ((grids[j].nz + d - 1) / d);
        return b;
    };
    if (variant == 0 && bricks(6) >= 4LL * 4 * num_sms) {
        *depth = 6;
        return;
    }
    *depth = 1;
    for (int d = variant >= 2 ? 4 : 8; d > 1; d /= 2)
        if (bricks(d) >= num_sms) {
            *depth = d;
            break;
        }
}

static bool encode4(CUtensorMap* m, CUtensorMapDataType t, const void* p, const Grid3& g, int ncomp,
                    int esz, const cuuint32_t box[4]) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz,
                                (cuuint64_t)ncomp};
    const cuuint64_t str[3] = {(cuuint64_t)g.px * esz, (cuuint64_t)g.plane * esz,
                               (cuuint64_t)g.cs * esz};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    return enc(m, t, 4, const_cast<void*>(p), dims, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool xy_group_add(XYGroup& G, const SmoothArgs& a) {
    if (G.n >= kGroupMax || (G.ty != 32 && G.ty != S2Y) || G.zchunk < 1 || a.ncomp != 3 ||
        a.in_type != kStoreF32 || a.out_type != kStoreF32 || a.taps.R != FZR)
        return false;
    const int j = G.n;
    if (j == 0) G.first[0] = 0;
    const int H = G.ty + 2 * FZR, WB = S2Geom<FZR>::WB;  // the plane box of sxy_block
    const cuuint32_t box[4] = {(cuuint32_t)WB, (cuuint32_t)H, 1u, 1u};
    if (!encode4(&G.map[j], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.in, a.g, 3, 4, box)) return false;
    G.a[j] = a;
    G.gx[j] = (a.g.nx + S2X - 1) / S2X;
    G.gy[j] = (a.g.ny + G.ty - 1) / G.ty;
    G.gz[j] = ((a.g.nz + G.zchunk - 1) / G.zchunk) * 3;
    G.first[j + 1] = G.first[j] + G.gx[j] * G.gy[j] * G.gz[j];
    G.n = j + 1;
    return true;
}

bool zs_group_add(ZSGroup& G, const ForceArgs& a) {
    const bool gm = G.variant >= 2;
    const int d = G.depth;
    if (G.n >= kGroupMax || G.variant < 0 || G.variant > 5 || a.field_type != kStoreF32 ||
        (a.img_type != kStoreF32 && a.img_type != kStoreI16) || G.taps.R != FZR ||
        !(d == 1 || d == 2 || d == 4 || (!gm && (d == 6 || d == 8))))
        return false;
    const int j = G.n;
    if (j == 0) G.first[0] = 0;
    const bool i16 = a.img_type == kStoreI16;
    const int esz = i16 ? 2 : 4;
    const int fsw = FTX + 2 * (16 / esz);  // image box: 16 bytes of x halo each side
    const CUtensorMapDataType it = i16 ? tma_type<int16_t>() : tma_type<float>();
    // t box: the brick with R halo planes (Eqs. 1-2), or the Eqs. 3-6 u box
    // (x0 - 4 .. x0 + 35, y0 - 1 .. y0 + 8) with R + 1 halo planes
    const cuuint32_t tbox[4] = {(cuuint32_t)(gm ? FTX + 8 : FTX), (cuuint32_t)(gm ? FTY + 2 : FTY),
                                (cuuint32_t)(gm ? d + 2 + 2 * FZR : d + 2 * FZR), 3u};
    const cuuint32_t ibox[4] = {(cuuint32_t)fsw, (cuuint32_t)(FTY + 2), (cuuint32_t)(d + 2), 1u};
    if (!encode4(&G.tmap[j], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.u, a.g, 3, 4, tbox) ||
        !encode4(&G.smap[j], it, a.S, a.g, 1, esz, ibox) ||
        !encode4(&G.mmap[j], it, a.M, a.g, 1, esz, ibox))
        return false;
    G.a[j] = a;
    G.gx[j] = (a.g.nx + FTX - 1) / FTX;
    G.gy[j] = (a.g.ny + FTY - 1) / FTY;
    G.gz[j] = (a.g.nz + d - 1) / d;
    G.first[j + 1] = G.first[j] + G.gx[j] * G.gy[j] * G.gz[j];
    G.n = j + 1;
    return true;
}

cudaError_t launch_smooth_xy_grouped(const XYGroup& G, cudaStream_t s, bool pdl) {
    if (G.n < 1 || G.first[G.n] < 1) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)G.first[G.n]);
    if (G.ty == 32) {
        static KernelSetup st;
        const cudaError_t e = setup_kernel(st, smooth_xy_grouped_kernel<32>, sxy_smem(32));
        if (e != cudaSuccess) return e;
        return launch_ex(smooth_xy_grouped_kernel<32>, grid, dim3(8 * 32), sxy_smem(32), s, pdl, G);
    } else if (G.ty == S2Y) {
        static KernelSetup st;
        const cudaError_t e = setup_kernel(st, smooth_xy_grouped_kernel<S2Y>, sxy_smem(S2Y));
        if (e != cudaSuccess) return e;
        return launch_ex(smooth_xy_grouped_kernel<S2Y>, grid, dim3(8 * S2Y), sxy_smem(S2Y), s, pdl,
                         G);
    }
    return cudaErrorInvalidValue;
}

template <int V, int FTZ, typename TI>
static cudaError_t launch_zsg(const ZSGroup& G, cudaStream_t s, bool pdl) {
    constexpr int SMEM = V <= 1 ? FZGeom<FTZ, V, TI>::SMEM : GZGeom<FTZ, V, TI>::SMEM;
    static KernelSetup st;  // per instantiation
    const cudaError_t e = setup_kernel(st, force_zs_grouped_kernel<V, FTZ, TI>, SMEM);
    if (e != cudaSuccess) return e;
    return launch_ex(force_zs_grouped_kernel<V, FTZ, TI>, dim3((unsigned)G.first[G.n]),
                     dim3(FTX, FTY, 1), SMEM, s, pdl, G);
}

template <int V, typename TI>
static cudaError_t launch_zsg_depth(const ZSGroup& G, cudaStream_t s, bool pdl) {
    if constexpr (V <= 1) {
        switch (G.depth) {
            case 8: return launch_zsg<V, 8, TI>(G, s, pdl);
            case 6: return launch_zsg<V, 6, TI>(G, s, pdl);
            case 4: return launch_zsg<V, 4, TI>(G, s, pdl);
            case 2: return launch_zsg<V, 2, TI>(G, s, pdl);
            case 1: return launch_zsg<V, 1, TI>(G, s, pdl);
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (G.depth) {
            case 4: return launch_zsg<V, 4, TI>(G, s, pdl);
            case 2: return launch_zsg<V, 2, TI>(G, s, pdl);
            case 1: return launch_zsg<V, 1, TI>(G, s, pdl);
            default: return cudaErrorInvalidValue;
        }
    }
}

template <typename TI>
static cudaError_t launch_zsg_types(int variant, const ZSGroup& G, cudaStream_t s, bool pdl) {
    switch (variant) {
        case 0: return launch_zsg_depth<0, TI>(G, s, pdl);
        case 1: return launch_zsg_depth<1, TI>(G, s, pdl);
        case 2: return launch_zsg_depth<2, TI>(G, s, pdl);
        case 3: return launch_zsg_depth<3, TI>(G, s, pdl);
        case 4: return launch_zsg_depth<4, TI>(G, s, pdl);
        case 5: return launch_zsg_depth<5, TI>(G, s, pdl);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_force_zs_grouped(int variant, int img_type, const ZSGroup& G, cudaStream_t s,
                                    bool pdl) {
    if (G.n < 1 || G.first[G.n] < 1 || variant != G.variant) return cudaErrorInvalidValue;
    if (img_type == kStoreF32) return launch_zsg_types<float>(variant, G, s, pdl);
    if (img_type == kStoreI16) return launch_zsg_types<int16_t>(variant, G, s, pdl);
    return cudaErrorInvalidValue;
}

bool d_group_add(ZDGroup& Z, STGroup& T, const ForceArgs& zd, const ForceArgs& st) {
    const int d = Z.depth;
    if (Z.n >= kGroupMax || Z.n != T.n || T.depth != d || Z.variant < 2 || Z.variant > 5 ||
        T.variant != Z.variant || zd.field_type != kStoreF32 ||
        (zd.img_type != kStoreF32 && zd.img_type != kStoreI16) || Z.taps.R != FZR ||
        !(d == 1 || d == 2 || d == 4) || zd.dbuf == nullptr || st.dbuf == nullptr ||
        (Z.variant == 5 && (zd.dbuf2 == nullptr || st.dbuf2 == nullptr)))
        return false;
    const int j = Z.n;
    if (j == 0) Z.first[0] = T.first[0] = 0;
    const bool i16 = zd.img_type == kStoreI16;
    const int esz = i16 ? 2 : 4;
    const int fsw = FTX + 2 * (16 / esz);  // S box: 16 bytes of x halo each side
    const CUtensorMapDataType it = i16 ? tma_type<int16_t>() : tma_type<float>();
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint32_t tbox[4] = {(cuuint32_t)FTX, (cuuint32_t)FTY, (cuuint32_t)(d + 2 * FZR), 3u};
    const cuuint32_t dbox[4] = {(cuuint32_t)(FTX + 8), (cuuint32_t)(FTY + 2), (cuuint32_t)(d + 2), 1u};
    const cuuint32_t sbox[4] = {(cuuint32_t)fsw, (cuuint32_t)(FTY + 2), (cuuint32_t)(d + 2), 1u};
    const cuuint32_t ubox[4] = {(cuuint32_t)FTX, (cuuint32_t)FTY, (cuuint32_t)d, 3u};
    const cuuint32_t ebox[4] = {(cuuint32_t)FTX, (cuuint32_t)FTY, (cuuint32_t)d, 1u};
    if (!encode4(&Z.tmap[j], f32, zd.u, zd.g, 3, 4, tbox) ||
        !encode4(&T.dmap[j], f32, st.dbuf, st.g, 1, 4, dbox) ||
        !encode4(&T.smap[j], it, st.S, st.g, 1, esz, sbox) ||
        !encode4(&T.umap[j], f32, st.u, st.g, 3, 4, ubox))
        return false;
    if (Z.variant == 5) {
        if (!encode4(&T.emap[j], f32, st.dbuf2, st.g, 1, 4, ebox)) return false;
    } else {
        T.emap[j] = T.umap[j];  // not read
    }
    Z.a[j] = zd;
    T.a[j] = st;
    Z.gx[j] = T.gx[j] = (zd.g.nx + FTX - 1) / FTX;
    Z.gy[j] = T.gy[j] = (zd.g.ny + FTY - 1) / FTY;
    Z.gz[j] = T.gz[j] = (zd.g.nz + d - 1) / d;
    Z.first[j + 1] = T.first[j + 1] = Z.first[j] + Z.gx[j] * Z.gy[j] * Z.gz[j];
    Z.n = T.n = j + 1;
    return true;
}

template <int V, int FTZ, typename TI>
static cudaError_t launch_dg(const ZDGroup& Z, const STGroup& T, cudaStream_t s, bool pdl) {
    constexpr int ZS = ZDGeom<FTZ>::SMEM, TS = STGeom<FTZ, V, TI>::SMEM;
    static KernelSetup zst, tst;  // per instantiation
    cudaError_t e = setup_kernel(zst, force_zd_grouped_kernel<V, FTZ, TI>, ZS);
    if (e == cudaSuccess) e = setup_kernel(tst, force_st_grouped_kernel<V, FTZ, TI>, TS);
    if (e != cudaSuccess) return e;
    e = launch_ex(force_zd_grouped_kernel<V, FTZ, TI>, dim3((unsigned)Z.first[Z.n]),
                  dim3(FTX, FTY, 1), ZS, s, pdl, Z);
    if (e != cudaSuccess) return e;
    return launch_ex(force_st_grouped_kernel<V, FTZ, TI>, dim3((unsigned)T.first[T.n]),
                     dim3(FTX, FTY, 1), TS, s, pdl, T);
}

template <int V, typename TI>
static cudaError_t launch_dg_depth(const ZDGroup& Z, const STGroup& T, cudaStream_t s, bool pdl) {
    switch (Z.depth) {
        case 4: return launch_dg<V, 4, TI>(Z, T, s, pdl);
        case 2: return launch_dg<V, 2, TI>(Z, T, s, pdl);
        case 1: return launch_dg<V, 1, TI>(Z, T, s, pdl);
        default: return cudaErrorInvalidValue;
    }
}

template <typename TI>
static cudaError_t launch_dg_types(const ZDGroup& Z, const STGroup& T, cudaStream_t s, bool pdl) {
    switch (Z.variant) {
        case 2: return launch_dg_depth<2, TI>(Z, T, s, pdl);
        case 3: return launch_dg_depth<3, TI>(Z, T, s, pdl);
        case 4: return launch_dg_depth<4, TI>(Z, T, s, pdl);
        case 5: return launch_dg_depth<5, TI>(Z, T, s, pdl);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_force_d_grouped(int img_type, const ZDGroup& Z, const STGroup& T,
                                   cudaStream_t s, bool pdl) {
    if (Z.n < 1 || Z.n != T.n || Z.first[Z.n] < 1 || Z.variant != T.variant ||
        Z.depth != T.depth)
        return cudaErrorInvalidValue;
    if (img_type == kStoreF32) return launch_dg_types<float>(Z, T, s, pdl);
    if (img_type == kStoreI16) return launch_dg_types<int16_t>(Z, T, s, pdl);
    return cudaErrorInvalidValue;
}

}  // namespace dirk
