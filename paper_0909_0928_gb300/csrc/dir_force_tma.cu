// dir_force_tma.cu -- the force pass of Eqs. (1)-(6) in single precision with
// its streamed operands brought in by TMA (Eqs. 1-2 below; Eqs. 3-6, which
// need the gradient of the warped image, in force_tma_gm_kernel further down).
//
// Same work per voxel as force_kernel (dir_force_kernel.cuh: interp_rel,
// demons_force, the same reductions) on the same 32 x 8 x FTZ bricks, but the
// block fetches its whole brick of u (three components) and of S with a
// one-voxel halo (and of M, for Eq. 2's |grad M|) with one bulk tensor copy
// each, waits once, and then reads them from shared memory; only the gathers
// of M at x + u go through L1/L2.  Thread 0 also asks L2 to prefetch the
// bricks of the block pf_stride positions ahead (one block per SM ahead by
// default; cp.async.bulk.prefetch.tensor), so that later blocks find their
// operands in L2.
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_force_gm.cuh"
#include "dir_force_kernel.cuh"
#include "dir_stencil.cuh"

namespace dirk {


// Image boxes (S, and M for Eq. 2) start 16 bytes before the tile in x (the
// copy's x coordinate must be 16-byte aligned): a halo of 4 floats or 8 int16.
template <int FTZ, int V, typename TI>
struct FTGeom {
    static constexpr int FBX = 16 / (int)sizeof(TI);           // image box x halo
    static constexpr int FSW = FTX + 2 * FBX;                  // image box width
    static constexpr int UBOX = 3 * FTZ * FTY * FTX * 4;       // [3][FTZ][FTY][FTX] floats
    static constexpr int SBOX = (FTZ + 2) * FSH * FSW * (int)sizeof(TI);  // [FTZ+2][FSH][FSW]
    static constexpr int OFF_S = (UBOX + 127) / 128 * 128;
    static constexpr int OFF_M = OFF_S + (SBOX + 127) / 128 * 128;
    static constexpr int OFF_BAR = OFF_M + (V == 1 ? (SBOX + 127) / 128 * 128 : 0);
    static constexpr int SMEM = 128 + OFF_BAR + 64;
};

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, 4)
    force_tma_kernel(const __grid_constant__ CUtensorMap umap,
                     const __grid_constant__ CUtensorMap smap,
                     const __grid_constant__ CUtensorMap mmap, const ForceArgs a) {
    static_assert(V == 0 || V == 1, "no gradient of the warped image");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;  // uniform across the grid
    using F = FTGeom<FTZ, V, TI>;
    constexpr int FBX = F::FBX, FSW = F::FSW;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const float* ub = reinterpret_cast<const float*>(base);          // [3][FTZ][FTY][FTX]
    const TI* sb = reinterpret_cast<const TI*>(base + F::OFF_S);     // [FTZ+2][FSH][FSW]
    const TI* mb = reinterpret_cast<const TI*>(base + F::OFF_M);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + F::OFF_BAR);
    const Grid3 g = a.g;
    const TI* __restrict__ M = static_cast<const TI*>(a.M);
    float* __restrict__ v = static_cast<float*>(a.v);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + FTX * ty;
    const int bx0 = blockIdx.x * FTX, by0 = blockIdx.y * FTY, bz0 = blockIdx.z * FTZ;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)(F::UBOX + F::SBOX + (V == 1 ? F::SBOX : 0)));
        tma_load_4d(base, &umap, bx0, by0, bz0, 0, bar);
        tma_load_4d(base + F::OFF_S, &smap, bx0 - FBX, by0 - 1, bz0 - 1, 0, bar);
        if (V == 1) tma_load_4d(base + F::OFF_M, &mmap, bx0 - FBX, by0 - 1, bz0 - 1, 0, bar);
        // the block pf_stride positions ahead: its bricks into L2
        if (a.pf_stride > 0) {
            const long long gx = gridDim.x, gy = gridDim.y;
            const long long b = blockIdx.x + gx * (blockIdx.y + gy * (long long)blockIdx.z) +
                                a.pf_stride;
            if (b < gx * gy * gridDim.z) {
                const int px = (int)(b % gx) * FTX, py = (int)((b / gx) % gy) * FTY;
                const int pz = (int)(b / (gx * gy)) * FTZ;
                tma_prefetch_4d(&umap, px, py, pz, 0);
                tma_prefetch_4d(&smap, px - FBX, py - 1, pz - 1, 0);
                tma_prefetch_4d(&mmap, px - FBX, py - 1, pz - 1, 0);
            }
        }
    }
    __syncthreads();
    bool ok = true;
    if (tid == 0) ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (__syncthreads_or(!ok)) {
        if (tid == 0 && a.err) atomicOr(a.err, kErrTmaTimeout);
        return;
    }
    (void)mbar_try_wait(bar, 0);

    const int x = bx0 + tx, y = by0 + ty;
    const bool col_valid = (x < g.nx) && (y < g.ny);
    const int xc = min(x, g.nx - 1), yc = min(y, g.ny - 1);
    // shared-memory offsets of this column and of its clamped x / y neighbours
    const int sx = xc - (bx0 - FBX), sxm = max(xc - 1, 0) - (bx0 - FBX);
    const int sxp = min(xc + 1, g.nx - 1) - (bx0 - FBX);
    const int sy = yc - (by0 - 1), sym = max(yc - 1, 0) - (by0 - 1);
    const int syp = min(yc + 1, g.ny - 1) - (by0 - 1);
    const Interp ip(g);
    const int cs = (int)g.cs;
    float sd2 = 0.0f, sdu = 0.0f, su = 0.0f;
    CorrSums<float> corr_s;  // with a.corr: the correlation sums
    if (col_valid) {
#pragma unroll
        for (int k = 0; k < FTZ; ++k) {
            const int z = bz0 + k;
            if (z < g.nz) {
                // S planes of the box: plane p holds z = bz0 - 1 + p; the clamped
                // neighbours z - 1 and z + 1 are planes k and k + 2 unless they
                // fall outside the volume
                const int pc = k + 1;
                const int pm = max(z - 1, 0) - (bz0 - 1), pp = min(z + 1, g.nz - 1) - (bz0 - 1);
                const TI* Sc = sb + pc * (FSH * FSW);
                const float s0 = (float)Sc[sy * FSW + sx];
                const float gsx = 0.5f * ((float)Sc[sy * FSW + sxp] - (float)Sc[sy * FSW + sxm]);
                const float gsy = 0.5f * ((float)Sc[syp * FSW + sx] - (float)Sc[sym * FSW + sx]);
                const float gsz = 0.5f * ((float)sb[pp * (FSH * FSW) + sy * FSW + sx] -
                                          (float)sb[pm * (FSH * FSW) + sy * FSW + sx]);
                const int ui = (k * FTY + ty) * FTX + tx;
                const float ux = ub[ui], uy = ub[ui + FTZ * FTY * FTX],
                            uz = ub[ui + 2 * FTZ * FTY * FTX];
                float bm = 0.0f;
                if (V == 1) {
                    const TI* Mc = mb + pc * (FSH * FSW);
                    const float mx = 0.5f * ((float)Mc[sy * FSW + sxp] - (float)Mc[sy * FSW + sxm]);
                    const float my = 0.5f * ((float)Mc[syp * FSW + sx] - (float)Mc[sym * FSW + sx]);
                    const float mz = 0.5f * ((float)mb[pp * (FSH * FSW) + sy * FSW + sx] -
                                             (float)mb[pm * (FSH * FSW) + sy * FSW + sx]);
                    bm = r_sqrt(mx * mx + my * my + mz * mz);
                }
                const float d = interp_rel(M, ip, x, ux, y, uy, z, uz, s0);  // W - S
                if (a.corr) corr_s.add(s0, d);
                float dx, dy, dz;
                demons_force<float, V>(d, gsx, gsy, gsz, 0.0f, 0.0f, 0.0f, bm, 0.0f, dx, dy, dz);
                dx = -dx;
                dy = -dy;
                dz = -dz;
                sd2 += d * d;
                sdu += r_norm_fast(dx * dx + dy * dy + dz * dz);
                su += r_norm_fast(ux * ux + uy * uy + uz * uz);
                const int o = offs(g, x, y, z);
                v[o] = ux + dx;
                v[o + cs] = uy + dy;
                v[o + 2 * cs] = uz + dz;
            }
        }
    }
    block_reduce3_atomic<FNT, float>(sd2, sdu, su, a.red);
    if (a.corr) block_reduce4_atomic<FNT, float>(corr_s, a.corr);
}

template <typename TI>
static bool make_force_maps(CUtensorMap* umap, CUtensorMap* smap, CUtensorMap* mmap,
                            const ForceArgs& a, int ftz) {
    constexpr int FSW = FTGeom<1, 0, TI>::FSW;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const Grid3& g = a.g;
    const cuuint64_t udims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
    const cuuint64_t idims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 1};
    const cuuint64_t ustr[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                (cuuint64_t)g.cs * 4};
    const cuuint64_t istr[3] = {(cuuint64_t)g.px * sizeof(TI), (cuuint64_t)g.plane * sizeof(TI),
                                (cuuint64_t)g.cs * sizeof(TI)};
    const cuuint32_t ubox[4] = {(cuuint32_t)FTX, (cuuint32_t)FTY, (cuuint32_t)ftz, 3u};
    const cuuint32_t ibox[4] = {(cuuint32_t)FSW, (cuuint32_t)FSH, (cuuint32_t)(ftz + 2), 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    auto enc4 = [&](CUtensorMap* m, CUtensorMapDataType t, const void* p, const cuuint64_t* d,
                    const cuuint64_t* st, const cuuint32_t* b) {
        return enc(m, t, 4, const_cast<void*>(p), d, st, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    return enc4(umap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.u, udims, ustr, ubox) &&
           enc4(smap, tma_type<TI>(), a.S, idims, istr, ibox) &&
           enc4(mmap, tma_type<TI>(), a.M, idims, istr, ibox);
}

template <int V, int FTZ, typename TI>
static cudaError_t launch_ft(const ForceArgs& a, cudaStream_t s) {
    using F = FTGeom<FTZ, V, TI>;
    CUtensorMap umap, smap, mmap;
    if (!make_force_maps<TI>(&umap, &smap, &mmap, a, FTZ)) return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    const cudaError_t e = setup_kernel(setup, force_tma_kernel<V, FTZ, TI>, F::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.g.nx + FTX - 1) / FTX, (a.g.ny + FTY - 1) / FTY, (a.g.nz + FTZ - 1) / FTZ);
    force_tma_kernel<V, FTZ, TI><<<grid, dim3(FTX, FTY, 1), F::SMEM, s>>>(umap, smap, mmap, a);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Eqs. (3)-(6): the force needs the gradient of the warped image, so the block
// first forms D = W - S (Eq. 6: D_m + D_s, and d = D_m - D_s on the brick) on
// the brick plus a one-voxel halo in shared memory, as force_kernel does, but
// reads u (with its halo) and S from TMA boxes instead of global memory.  The
// brick depth is at most 4 so that four blocks fit per SM.
// ---------------------------------------------------------------------------

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, 4)
    force_tma_gm_kernel(const __grid_constant__ CUtensorMap umap,
                        const __grid_constant__ CUtensorMap smap,
                        const __grid_constant__ CUtensorMap mmap, const ForceArgs a) {
    static_assert(V >= 2 && V <= 5, "Eqs. 3-6");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;  // uniform across the grid
    using F = FGGeom<FTZ, V, TI>;
    constexpr int FBX = F::FBX;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const float* ub = reinterpret_cast<const float*>(base);       // [3][UD][UH][UW]
    const TI* sb = reinterpret_cast<const TI*>(base + F::OFF_S);  // [UD][FSH][FSW]
    float* wt = reinterpret_cast<float*>(base + F::OFF_W);        // [HZ][HY][HX]
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + F::OFF_BAR);
    const int tid = threadIdx.x + FTX * threadIdx.y;
    const int bx0 = blockIdx.x * FTX, by0 = blockIdx.y * FTY, bz0 = blockIdx.z * FTZ;
    const int ux0 = bx0 - 4, uy0 = by0 - 1, uz0 = bz0 - 1;     // u box origin
    const int sx0 = bx0 - FBX, sy0 = by0 - 1, sz0 = bz0 - 1;   // S box origin
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)(F::UBOX + F::SBOX));
        tma_load_4d(base, &umap, ux0, uy0, uz0, 0, bar);
        tma_load_4d(base + F::OFF_S, &smap, sx0, sy0, sz0, 0, bar);
        if (a.pf_stride > 0) {  // the block pf_stride positions ahead: its boxes into L2
            const long long gx = gridDim.x, gy = gridDim.y;
            const long long b = blockIdx.x + gx * (blockIdx.y + gy * (long long)blockIdx.z) +
                                a.pf_stride;
            if (b < gx * gy * gridDim.z) {
                const int px = (int)(b % gx) * FTX, py = (int)((b / gx) % gy) * FTY;
                const int pz = (int)(b / (gx * gy)) * FTZ;
                tma_prefetch_4d(&umap, px - 4, py - 1, pz - 1, 0);
                tma_prefetch_4d(&smap, px - FBX, py - 1, pz - 1, 0);
                tma_prefetch_4d(&mmap, px - FBX, py - 1, pz - 1, 0);
            }
        }
    }
    __syncthreads();
    bool ok = true;
    if (tid == 0) ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (__syncthreads_or(!ok)) {
        if (tid == 0 && a.err) atomicOr(a.err, kErrTmaTimeout);
        return;
    }
    (void)mbar_try_wait(bar, 0);
    gm_force_body<V, FTZ, TI, F::UD * F::UH * F::UW>(a, ub, sb, wt, BlockPos::of_grid());
}

template <typename TI>
static bool make_gm_maps(CUtensorMap* umap, CUtensorMap* smap, CUtensorMap* mmap,
                         const ForceArgs& a, int ftz) {
    constexpr int FSW = FTGeom<1, 0, TI>::FSW;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const Grid3& g = a.g;
    const cuuint64_t udims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
    const cuuint64_t idims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 1};
    const cuuint64_t ustr[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                (cuuint64_t)g.cs * 4};
    const cuuint64_t istr[3] = {(cuuint64_t)g.px * sizeof(TI), (cuuint64_t)g.plane * sizeof(TI),
                                (cuuint64_t)g.cs * sizeof(TI)};
    const cuuint32_t ubox[4] = {(cuuint32_t)(FTX + 8), (cuuint32_t)(FTY + 2), (cuuint32_t)(ftz + 2),
                                3u};
    const cuuint32_t ibox[4] = {(cuuint32_t)FSW, (cuuint32_t)FSH, (cuuint32_t)(ftz + 2), 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    auto enc4 = [&](CUtensorMap* m, CUtensorMapDataType t, const void* p, const cuuint64_t* d,
                    const cuuint64_t* st, const cuuint32_t* b) {
        return enc(m, t, 4, const_cast<void*>(p), d, st, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    return enc4(umap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.u, udims, ustr, ubox) &&
           enc4(smap, tma_type<TI>(), a.S, idims, istr, ibox) &&
           enc4(mmap, tma_type<TI>(), a.M, idims, istr, ibox);
}

template <int V, int FTZ, typename TI>
static cudaError_t launch_fg(const ForceArgs& a, cudaStream_t s) {
    using F = FGGeom<FTZ, V, TI>;
    CUtensorMap umap, smap, mmap;
    if (!make_gm_maps<TI>(&umap, &smap, &mmap, a, FTZ)) return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    const cudaError_t e = setup_kernel(setup, force_tma_gm_kernel<V, FTZ, TI>, F::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.g.nx + FTX - 1) / FTX, (a.g.ny + FTY - 1) / FTY, (a.g.nz + FTZ - 1) / FTZ);
    force_tma_gm_kernel<V, FTZ, TI><<<grid, dim3(FTX, FTY, 1), F::SMEM, s>>>(umap, smap, mmap, a);
    return cudaGetLastError();
}

template <int V, typename TI>
static cudaError_t launch_fg_depth(const ForceArgs& a, cudaStream_t s) {
    switch (a.depth) {
        case 8:
        case 4: return launch_fg<V, 4, TI>(a, s);  // at most 4 deep (four blocks per SM)
        case 2: return launch_fg<V, 2, TI>(a, s);
        case 1: return launch_fg<V, 1, TI>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename TI>
static cudaError_t launch_fg_types(int variant, const ForceArgs& a, cudaStream_t s) {
    switch (variant) {
        case 2: return launch_fg_depth<2, TI>(a, s);
        case 3: return launch_fg_depth<3, TI>(a, s);
        case 4: return launch_fg_depth<4, TI>(a, s);
        case 5: return launch_fg_depth<5, TI>(a, s);
        default: return cudaErrorNotSupported;
    }
}

template <typename TI>
static cudaError_t launch_ft_types(int variant, const ForceArgs& a, cudaStream_t s) {
    switch (a.depth) {
        case 8: return variant ? launch_ft<1, 8, TI>(a, s) : launch_ft<0, 8, TI>(a, s);
        case 4: return variant ? launch_ft<1, 4, TI>(a, s) : launch_ft<0, 4, TI>(a, s);
        case 2: return variant ? launch_ft<1, 2, TI>(a, s) : launch_ft<0, 2, TI>(a, s);
        case 1: return variant ? launch_ft<1, 1, TI>(a, s) : launch_ft<0, 1, TI>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

// Eqs. (1)-(6) in single precision with a float field and float or int16
// images; returns cudaErrorNotSupported for anything else (the caller then
// uses force_kernel)
cudaError_t launch_force_tma(int variant, const ForceArgs& a, cudaStream_t s) {
    if (variant < 0 || variant > 5) return cudaErrorNotSupported;
    if (a.field_type != kStoreF32) return cudaErrorNotSupported;
    if (variant >= 2) {
        if (a.img_type == kStoreF32) return launch_fg_types<float>(variant, a, s);
        if (a.img_type == kStoreI16) return launch_fg_types<int16_t>(variant, a, s);
        return cudaErrorNotSupported;
    }
    if (a.img_type == kStoreF32) return launch_ft_types<float>(variant, a, s);
    if (a.img_type == kStoreI16) return launch_ft_types<int16_t>(variant, a, s);
    return cudaErrorNotSupported;
}

}  // namespace dirk
