// dir_force_zs.cu -- the force pass of Eqs. (1)-(2) with the last pass of the
// smoothing folded in (single precision).
//
// One iteration of Sec. 2.1 is u = G_sigma * v (Thirion's smoothing of the
// total field), then v = u - dr(u).  The Gaussian is separable (x, then y,
// then z), and the Eqs. 1-2 force needs u only at the voxel itself, so the
// iteration splits cleanly after the y pass: smooth_xy_kernel writes
// t = G_y * G_x * v plane by plane, and this kernel forms u = G_z * t down
// its own z columns before the force work.  Each thread already owns the
// FTZ voxels of one (x, y) column of its brick, so the z pass needs the brick
// of t with R planes more above and below (one bulk tensor copy of all three
// components, edges replicated in shared memory) and no exchange between
// threads.  Unlike the marching smoothing kernel, no z halo of x and y work
// is redone per block, which is what the small pyramid levels paid for.
//
// Per voxel the arithmetic is that of smooth2_kernel's z pass (taps oldest
// plane first, fused multiply-adds from zero) followed by force_tma_kernel's
// force, update and reductions, so the field is bit for bit the one of the
// smoothing + force schedule.
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_force_gm.cuh"
#include "dir_force_kernel.cuh"
#include "dir_stencil.cuh"

namespace dirk {

constexpr int FZR = 3;           // Gaussian radius compiled here (sigma = 1 voxel)
constexpr int FZSH = FTY + 2;    // image box rows: y0 - 1 .. y0 + 8

template <int FTZ, int V, typename TI>
struct FZGeom {
    static constexpr int NPZ = FTZ + 2 * FZR;                  // t planes bz0 - R .. bz0 + FTZ - 1 + R
    static constexpr int FBX = 16 / (int)sizeof(TI);           // image box x halo
    static constexpr int FSW = FTX + 2 * FBX;                  // image box width
    static constexpr int TBOX = 3 * NPZ * FTY * FTX * 4;       // [3][NPZ][FTY][FTX] floats
    static constexpr int SBOX = (FTZ + 2) * FZSH * FSW * (int)sizeof(TI);  // [FTZ+2][FZSH][FSW]
    static constexpr int OFF_S = (TBOX + 127) / 128 * 128;
    static constexpr int OFF_M = OFF_S + (SBOX + 127) / 128 * 128;
    static constexpr int OFF_BAR = OFF_M + (V == 1 ? (SBOX + 127) / 128 * 128 : 0);
    static constexpr int SMEM = 128 + OFF_BAR + 64;
};

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, 4)
    force_zs_kernel(const __grid_constant__ CUtensorMap tmap,
                    const __grid_constant__ CUtensorMap smap,
                    const __grid_constant__ CUtensorMap mmap, const ForceArgs a, const Taps taps) {
    static_assert(V == 0 || V == 1, "no gradient of the warped image");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;  // uniform across the grid
    using F = FZGeom<FTZ, V, TI>;
    constexpr int R = FZR, NPZ = F::NPZ, FBX = F::FBX, FSW = F::FSW;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    float* tb = reinterpret_cast<float*>(base);                      // [3][NPZ][FTY][FTX]
    const TI* sb = reinterpret_cast<const TI*>(base + F::OFF_S);     // [FTZ+2][FZSH][FSW]
    const TI* mb = reinterpret_cast<const TI*>(base + F::OFF_M);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + F::OFF_BAR);
    const Grid3 g = a.g;
    const TI* __restrict__ M = static_cast<const TI*>(a.M);
    float* __restrict__ v = static_cast<float*>(a.v);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + FTX * ty;
    // bricks from the top plane down: smooth_xy_kernel wrote t bottom up, so
    // the first bricks find the planes it wrote last still in L2, and the next
    // x/y pass (bottom up) finds the v this kernel wrote last
    const int bx0 = blockIdx.x * FTX, by0 = blockIdx.y * FTY;
    const int bz0 = (gridDim.z - 1 - blockIdx.z) * FTZ;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)(F::TBOX + F::SBOX + (V == 1 ? F::SBOX : 0)));
        // planes outside the volume arrive zero-filled; replicated below
        tma_load_4d(base, &tmap, bx0, by0, bz0 - R, 0, bar);
        tma_load_4d(base + F::OFF_S, &smap, bx0 - FBX, by0 - 1, bz0 - 1, 0, bar);
        if (V == 1) tma_load_4d(base + F::OFF_M, &mmap, bx0 - FBX, by0 - 1, bz0 - 1, 0, bar);
        if (a.pf_stride > 0) {  // the block pf_stride positions ahead: its boxes into L2
            const long long gx = gridDim.x, gy = gridDim.y;
            const long long b = blockIdx.x + gx * (blockIdx.y + gy * (long long)blockIdx.z) +
                                a.pf_stride;
            if (b < gx * gy * gridDim.z) {
                const int px = (int)(b % gx) * FTX, py = (int)((b / gx) % gy) * FTY;
                const int pz = (int)(gridDim.z - 1 - b / (gx * gy)) * FTZ;
                tma_prefetch_4d(&tmap, px, py, pz - R, 0);
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
    float sd2 = 0.0f, sdu = 0.0f, su = 0.0f;
    CorrSums<float> corr_s;  // with a.corr: the correlation sums
    if (col_valid) {
        // z pass of the Gaussian down this thread's column (only this thread
        // reads or writes it, so no barrier): u[c][k] at z = bz0 + k
        float w[R + 1];
#pragma unroll
        for (int t = 0; t <= R; ++t) w[t] = taps.wf[t];
        float* tcol = tb + tid;  // plane j of component c at tcol[(c * NPZ + j) * FNT]
        const int zlo = bz0 - R;
        if (zlo < 0 || zlo + NPZ > g.nz) {  // replicate the edge planes into the zero fill
            const int jlo = max(0, -zlo), jhi = min(NPZ - 1, g.nz - 1 - zlo);
            for (int c = 0; c < 3; ++c) {
                float* tc = tcol + c * NPZ * FNT;
                const float lo = tc[jlo * FNT], hi = tc[jhi * FNT];
                for (int j = 0; j < jlo; ++j) tc[j * FNT] = lo;
                for (int j = jhi + 1; j < NPZ; ++j) tc[j * FNT] = hi;
            }
        }
        // u overwrites t in place (planes R .. R + FTZ - 1 of the column),
        // which keeps the force loop's registers those of force_tma_kernel
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float cv[NPZ];
#pragma unroll
            for (int j = 0; j < NPZ; ++j) cv[j] = tcol[(c * NPZ + j) * FNT];
#pragma unroll
            for (int k = 0; k < FTZ; ++k) {
                float acc = 0.0f;
#pragma unroll
                for (int t = 0; t < 2 * R + 1; ++t) acc = fmaf(w[t <= R ? t : 2 * R - t], cv[k + t], acc);
                tcol[(c * NPZ + R + k) * FNT] = acc;
            }
        }

        const int xc = x, yc = y;
        const int sx = xc - (bx0 - FBX), sxm = max(xc - 1, 0) - (bx0 - FBX);
        const int sxp = min(xc + 1, g.nx - 1) - (bx0 - FBX);
        const int sy = yc - (by0 - 1), sym = max(yc - 1, 0) - (by0 - 1);
        const int syp = min(yc + 1, g.ny - 1) - (by0 - 1);
        const Interp ip(g);
        const int cs = (int)g.cs;
#pragma unroll
        for (int k = 0; k < FTZ; ++k) {
            const int z = bz0 + k;
            if (z < g.nz) {
                const int pc = k + 1;
                const int pm = max(z - 1, 0) - (bz0 - 1), pp = min(z + 1, g.nz - 1) - (bz0 - 1);
                const TI* Sc = sb + pc * (FZSH * FSW);
                const float s0 = (float)Sc[sy * FSW + sx];
                const float gsx = 0.5f * ((float)Sc[sy * FSW + sxp] - (float)Sc[sy * FSW + sxm]);
                const float gsy = 0.5f * ((float)Sc[syp * FSW + sx] - (float)Sc[sym * FSW + sx]);
                const float gsz = 0.5f * ((float)sb[pp * (FZSH * FSW) + sy * FSW + sx] -
                                          (float)sb[pm * (FZSH * FSW) + sy * FSW + sx]);
                const float ux = tcol[(R + k) * FNT], uy = tcol[(NPZ + R + k) * FNT],
                            uz = tcol[(2 * NPZ + R + k) * FNT];
                float bm = 0.0f;
                if (V == 1) {
                    const TI* Mc = mb + pc * (FZSH * FSW);
                    const float mx = 0.5f * ((float)Mc[sy * FSW + sxp] - (float)Mc[sy * FSW + sxm]);
                    const float my = 0.5f * ((float)Mc[syp * FSW + sx] - (float)Mc[sym * FSW + sx]);
                    const float mz = 0.5f * ((float)mb[pp * (FZSH * FSW) + sy * FSW + sx] -
                                             (float)mb[pm * (FZSH * FSW) + sy * FSW + sx]);
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

// ---------------------------------------------------------------------------
// Eqs. (3)-(6) split the same way.  Their force needs the gradient of the
// warped image, so u is needed on the brick plus a one-voxel halo: the block
// copies t over the u box of force_tma_gm_kernel (x0 - 4 .. x0 + 35,
// y0 - 1 .. y0 + 8) with R + 1 extra planes below and above, forms
// u = G_z * t in place on the 34 x 10 columns the force reads (one thread per
// column, a column read and written only by its thread), and then runs the
// Eqs. 3-6 force work of dir_force_gm.cuh on that u.
// ---------------------------------------------------------------------------
template <int FTZ, int V, typename TI>
struct GZGeom {
    using G = FGGeom<FTZ, V, TI>;
    static constexpr int NPZ = G::UD + 2 * FZR;   // t planes z0 - 1 - R .. z0 + FTZ + R
    static constexpr int PL = G::UH * G::UW;      // floats per plane of the box
    static constexpr int TBOX = 3 * NPZ * PL * 4;
    static constexpr int OFF_S = (TBOX + 127) / 128 * 128;
    static constexpr int OFF_W = OFF_S + (G::SBOX + 127) / 128 * 128;
    static constexpr int OFF_BAR = OFF_W + (G::WT + 127) / 128 * 128;
    static constexpr int SMEM = 128 + OFF_BAR + 64;
};

template <int V, int FTZ, typename TI>
__global__ void __launch_bounds__(FNT, FTZ >= 2 ? 3 : 4)
    force_gzs_kernel(const __grid_constant__ CUtensorMap tmap,
                     const __grid_constant__ CUtensorMap smap,
                     const __grid_constant__ CUtensorMap mmap, const ForceArgs a, const Taps taps) {
    static_assert(V >= 2 && V <= 5, "Eqs. 3-6");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;  // uniform across the grid
    using F = FGGeom<FTZ, V, TI>;
    using Z = GZGeom<FTZ, V, TI>;
    constexpr int R = FZR, NPZ = Z::NPZ, PL = Z::PL, UD = F::UD, FBX = F::FBX;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    float* tb = reinterpret_cast<float*>(base);                   // [3][NPZ][UH][UW]
    const TI* sb = reinterpret_cast<const TI*>(base + Z::OFF_S);  // [UD][FSH][FSW]
    float* wt = reinterpret_cast<float*>(base + Z::OFF_W);        // [HZ][HY][HX]
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + Z::OFF_BAR);
    const Grid3 g = a.g;
    const int tid = threadIdx.x + FTX * threadIdx.y;
    const int bx0 = blockIdx.x * FTX, by0 = blockIdx.y * FTY, bz0 = blockIdx.z * FTZ;
    const int zlo = bz0 - 1 - R;  // global plane of box plane 0
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)(Z::TBOX + F::SBOX));
        tma_load_4d(base, &tmap, bx0 - 4, by0 - 1, zlo, 0, bar);
        tma_load_4d(base + Z::OFF_S, &smap, bx0 - FBX, by0 - 1, bz0 - 1, 0, bar);
        if (a.pf_stride > 0) {  // the block pf_stride positions ahead: its boxes into L2
            const long long gx = gridDim.x, gy = gridDim.y;
            const long long b = blockIdx.x + gx * (blockIdx.y + gy * (long long)blockIdx.z) +
                                a.pf_stride;
            if (b < gx * gy * gridDim.z) {
                const int px = (int)(b % gx) * FTX, py = (int)((b / gx) % gy) * FTY;
                const int pz = (int)(b / (gx * gy)) * FTZ;
                tma_prefetch_4d(&tmap, px - 4, py - 1, pz - 1 - R, 0);
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

    // z pass on the columns x0 - 1 .. x0 + 32 (box columns 3 .. 36), all rows;
    // planes outside the volume arrive zero-filled and are replicated first
    float w[R + 1];
#pragma unroll
    for (int t = 0; t <= R; ++t) w[t] = taps.wf[t];
    constexpr int NCX = FTX + 2, NCOL = NCX * F::UH;
    const bool zedge = zlo < 0 || zlo + NPZ > g.nz;
    const int jlo = max(0, -zlo), jhi = min(NPZ - 1, g.nz - 1 - zlo);
    for (int col = tid; col < NCOL; col += FNT) {
        float* tcol = tb + (col / NCX) * F::UW + 3 + (col % NCX);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float* tc = tcol + c * NPZ * PL;
            if (zedge) {
                const float lo = tc[jlo * PL], hi = tc[jhi * PL];
                for (int j = 0; j < jlo; ++j) tc[j * PL] = lo;
                for (int j = jhi + 1; j < NPZ; ++j) tc[j * PL] = hi;
            }
            float cv[NPZ];
#pragma unroll
            for (int j = 0; j < NPZ; ++j) cv[j] = tc[j * PL];
#pragma unroll
            for (int k = 0; k < UD; ++k) {
                float acc = 0.0f;
#pragma unroll
                for (int t = 0; t < 2 * R + 1; ++t) acc = fmaf(w[t <= R ? t : 2 * R - t], cv[k + t], acc);
                tc[(R + k) * PL] = acc;
            }
        }
    }
    __syncthreads();
    gm_force_body<V, FTZ, TI, NPZ * PL>(a, tb + R * PL, sb, wt);
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
    force_zs_kernel<V, FTZ, TI><<<grid, dim3(FTX, FTY, 1), F::SMEM, s>>>(tmap, smap, mmap, a, taps);
    return cudaGetLastError();
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
    force_gzs_kernel<V, FTZ, TI><<<grid, dim3(FTX, FTY, 1), Z::SMEM, s>>>(tmap, smap, mmap, a, taps);
    return cudaGetLastError();
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
