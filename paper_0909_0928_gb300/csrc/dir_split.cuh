// dir_split.cuh -- the block functions of the split iteration schedule
// (Sec. 2.1 smoothing of the total field, split at its last pass): the z +
// force pass of Eqs. (1)-(2) and of Eqs. (3)-(6), one brick per call, shared by
// the one-volume kernels (dir_force_zs.cu) and the grouped kernels over several
// volumes (dir_grouped.cu).  Each call handles the block at BlockPos bp of its
// own volume's grid.
//
// Launched with programmatic dependent launch (coarse levels, no stop test),
// a block starts while the kernel before still runs: it sets up its barriers
// and copies the static images, then waits (pdl_wait) before it reads the
// field the kernel before wrote or writes one that kernel reads.  The stop
// flag is read before that wait, which is sound only because such launches
// are made without a stop test, when the flag does not change during a
// registration.
//
// One iteration of Sec. 2.1 is u = G_sigma * v (Thirion's smoothing of the
// total field), then v = u - dr(u).  The Gaussian is separable (x, then y,
// then z), and the Eqs. 1-2 force needs u only at the voxel itself, so the
// iteration splits cleanly after the y pass: the x/y block (sxy_block) writes
// t = G_y * G_x * v plane by plane, and the z + force block forms u = G_z * t
// down its own z columns before the force work.  Each thread already owns the
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
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_force_gm.cuh"
#include "dir_force_kernel.cuh"
#include "dir_smooth2.cuh"
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

// One brick of the z + force pass (every thread of the block calls it).
template <int V, int FTZ, typename TI>
__device__ __forceinline__ void zs_block(const CUtensorMap* tmap, const CUtensorMap* smap,
                                         const CUtensorMap* mmap, const ForceArgs& a,
                                         const Taps& taps, const BlockPos bp) {
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
    const int bx0 = bp.x * FTX, by0 = bp.y * FTY;
    const int bz0 = (bp.gz - 1 - bp.z) * FTZ;
    pdl_trigger();
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)(F::TBOX + F::SBOX + (V == 1 ? F::SBOX : 0)));
        // the static images first: they do not depend on the kernel before
        tma_load_4d(base + F::OFF_S, smap, bx0 - FBX, by0 - 1, bz0 - 1, 0, bar);
        if (V == 1) tma_load_4d(base + F::OFF_M, mmap, bx0 - FBX, by0 - 1, bz0 - 1, 0, bar);
        pdl_wait();
        // planes outside the volume arrive zero-filled; replicated below
        tma_load_4d(base, tmap, bx0, by0, bz0 - R, 0, bar);
        if (a.pf_stride > 0) {  // the block pf_stride positions ahead: its boxes into L2
            const long long gx = bp.gx, gy = bp.gy;
            const long long b = bp.x + gx * (bp.y + gy * (long long)bp.z) +
                                a.pf_stride;
            if (b < gx * gy * bp.gz) {
                const int px = (int)(b % gx) * FTX, py = (int)((b / gx) % gy) * FTY;
                const int pz = (int)(bp.gz - 1 - b / (gx * gy)) * FTZ;
                tma_prefetch_4d(tmap, px, py, pz - R, 0);
                tma_prefetch_4d(smap, px - FBX, py - 1, pz - 1, 0);
                tma_prefetch_4d(mmap, px - FBX, py - 1, pz - 1, 0);
            }
        }
    }
    pdl_wait();  // every thread: v is written below, which the kernel before reads
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

// One brick of the Eqs. 3-6 z + force pass (every thread of the block calls it).
template <int V, int FTZ, typename TI>
__device__ __forceinline__ void gzs_block(const CUtensorMap* tmap, const CUtensorMap* smap,
                                          const CUtensorMap* mmap, const ForceArgs& a,
                                          const Taps& taps, const BlockPos bp) {
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
    const int bx0 = bp.x * FTX, by0 = bp.y * FTY, bz0 = bp.z * FTZ;
    const int zlo = bz0 - 1 - R;  // global plane of box plane 0
    pdl_trigger();
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)(Z::TBOX + F::SBOX));
        tma_load_4d(base + Z::OFF_S, smap, bx0 - FBX, by0 - 1, bz0 - 1, 0, bar);  // static
        pdl_wait();
        tma_load_4d(base, tmap, bx0 - 4, by0 - 1, zlo, 0, bar);
        if (a.pf_stride > 0) {  // the block pf_stride positions ahead: its boxes into L2
            const long long gx = bp.gx, gy = bp.gy;
            const long long b = bp.x + gx * (bp.y + gy * (long long)bp.z) +
                                a.pf_stride;
            if (b < gx * gy * bp.gz) {
                const int px = (int)(b % gx) * FTX, py = (int)((b / gx) % gy) * FTY;
                const int pz = (int)(b / (gx * gy)) * FTZ;
                tma_prefetch_4d(tmap, px - 4, py - 1, pz - 1 - R, 0);
                tma_prefetch_4d(smap, px - FBX, py - 1, pz - 1, 0);
                tma_prefetch_4d(mmap, px - FBX, py - 1, pz - 1, 0);
            }
        }
    }
    pdl_wait();  // every thread: v is written below, which the kernel before reads
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
    gm_force_body<V, FTZ, TI, NPZ * PL>(a, tb + R * PL, sb, wt, bp);
}

// ---------------------------------------------------------------------------
// The x and y passes of the split schedule (see smooth_xy_kernel in
// dir_smooth.cu): one z chunk of one component of a 32 x TY tile per call.
// ---------------------------------------------------------------------------
constexpr int SXYSTAGES = 4;

template <int R, int TY>
struct SXYSmem {
    using G = S2Geom<R, TY>;
    static constexpr int SMEM = 128 + SXYSTAGES * G::SLOT_STRIDE + G::TXP_STRIDE + 64;
};

// One z chunk of one component of one tile (every thread of the block calls it).
template <int R, int TY>
__device__ __forceinline__ void sxy_block(const CUtensorMap* tmap, const SmoothArgs& a, int zchunk,
                                          const BlockPos bp) {
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    using G = S2Geom<R, TY>;
    constexpr int H = G::H, HA = G::HA, WB = G::WB, NT = G::NTG;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    f32x2* txp = reinterpret_cast<f32x2*>(base + SXYSTAGES * G::SLOT_STRIDE);
    float* txf = reinterpret_cast<float*>(txp);
    uint64_t* full =
        reinterpret_cast<uint64_t*>(base + SXYSTAGES * G::SLOT_STRIDE + G::TXP_STRIDE);
    const Grid3 g = a.g;
    float w[R + 1];
    f32x2 wp[R + 1];
#pragma unroll
    for (int t = 0; t <= R; ++t) {
        w[t] = a.taps.wf[t];
        wp[t] = f2_pack(w[t], w[t]);
    }
    const int tid = threadIdx.x;
    const int lx = tid & 31, q = tid >> 5;
    const int comp = bp.z % a.ncomp;
    const int x0 = bp.x * S2X, y0 = bp.y * TY;
    const int z0 = (bp.z / a.ncomp) * zchunk;
    const int nsteps = min(z0 + zchunk, g.nz) - z0;  // planes z0 .. z0 + nsteps - 1
    const int bx = x0 - HA, by = y0 - R;
    const bool edge = (bx < 0) || (bx + WB > g.nx) || (by < 0) || (by + H > g.ny);
    float* __restrict__ out = static_cast<float*>(a.out) + (long long)comp * g.cs;

    auto issue = [&](int step) {
        const int sl = step % SXYSTAGES;
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[sl], (uint32_t)G::SLOT);
        tma_load_4d(base + sl * G::SLOT_STRIDE, tmap, bx, by, z0 + step, comp, &full[sl]);
    };
    pdl_trigger();
    if (tid == 0) {
        for (int sl = 0; sl < SXYSTAGES; ++sl) mbar_init(&full[sl], 1);
        fence_mbar_init();
        fence_proxy_async();
        pdl_wait();
        for (int st = 0; st < SXYSTAGES - 1 && st < nsteps; ++st) issue(st);
    }
    pdl_wait();  // every thread: t is written below, which the kernel before reads
    __syncthreads();

    const int x = x0 + lx;
    const int ya = y0 + 2 * q;  // rows ya, ya + 1 (lane 0) and ya + TY/2, ya + TY/2 + 1 (lane 1)
    const int px = (int)g.px;
    const int rows_left = x < g.nx ? g.ny - ya : 0;  // 0: this thread stores nothing
    for (int step = 0; step < nsteps; ++step) {
        if (tid == 0 && step + SXYSTAGES - 1 < nsteps) issue(step + SXYSTAGES - 1);
        const int sl = step % SXYSTAGES;
        const uint32_t parity = (uint32_t)((step / SXYSTAGES) & 1);
        bool ok = true;
        if (tid == 0) ok = mbar_wait_bounded(&full[sl], parity, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && a.err) atomicOr(a.err, kErrTmaTimeout);
            return;
        }
        (void)mbar_try_wait(&full[sl], parity);
        float* slot = reinterpret_cast<float*>(base + sl * G::SLOT_STRIDE);  // [H][WB]
        if (edge) s2_edge_fix<R, TY>(slot, G::SLOT_STRIDE / 4, 1, bx, by, g, tid, NT);
        s2_xpass<R, TY>(slot, txf, tid, w);
        __syncthreads();
        f32x2 r0, r1;
        s2_y_pair<R>(txp, q, lx, wp, r0, r1);
        float a0, b0, a1, b1;
        f2_unpack(r0, a0, b0);
        f2_unpack(r1, a1, b1);
        float* o = out + offs(g, x < g.nx ? x : 0, ya, z0 + step);
        if (rows_left > 0) o[0] = a0;
        if (rows_left > 1) o[px] = a1;
        if (rows_left > TY / 2) o[(TY / 2) * px] = b0;
        if (rows_left > TY / 2 + 1) o[(TY / 2 + 1) * px] = b1;
        // the next step's __syncthreads_or orders this step's reads of the
        // pair rows before the next x pass rewrites them
    }
}

}  // namespace dirk
