// dir_split_d.cuh -- the Eqs. (3)-(6) iteration split once more, after the
// difference image: D = W - S is formed once per voxel instead of once per
// voxel of every block footprint that reaches it.
//
// The force of Eqs. 3-6 needs the gradient of the warped image, so a block of
// the one-pass form (dir_force_gm.cuh) interpolates W on its brick plus a
// one-voxel halo: about twice per voxel at 32 x 8 x 4 bricks, four times for
// Eq. 6, which also warps S backwards.  Here one iteration is three kernels:
//   x/y pass   t = G_y G_x v                     (sxy_block, unchanged)
//   z + D pass u = G_z t down each thread's own column, then per voxel
//              D = W - S (Eq. 6: D_m + D_s and d = D_m - D_s); writes u and D
//   force pass the gradients of S and of W (= D + S) from shared-memory boxes
//              of D and S with a one-voxel halo, the force, v = u - dr(u) and
//              the reductions: a stencil with no gathers
// The arithmetic is that of gm_force_body voxel by voxel (D by interp_rel with
// the same operands, the same clamped neighbours, the same force call), so the
// field is bit for bit the one of the other schedules.  The default for Eqs.
// 3-6 on every pyramid level: the one-pass blocks were bound by issue and by
// the latency of their footprint gathers, not by memory, so the 36 B per voxel
// of u and D written here and read back by the force pass cost less than the
// gathers and instructions they remove.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_force_kernel.cuh"
#include "dir_split.cuh"

namespace dirk {

// z + D pass: the brick of t with R planes above and below (as FZGeom).
template <int FTZ>
struct ZDGeom {
    static constexpr int NPZ = FTZ + 2 * FZR;
    static constexpr int TBOX = 3 * NPZ * FTY * FTX * 4;  // [3][NPZ][FTY][FTX] floats
    static constexpr int OFF_BAR = (TBOX + 127) / 128 * 128;
    static constexpr int SMEM = 128 + OFF_BAR + 64;
};

// One brick of the z + D pass (every thread of the block calls it).  a.u: t,
// a.v: u out; a.dbuf: D out (Eq. 6: D_m + D_s), a.dbuf2: Eq. 6's d out.
template <int V, int FTZ, typename TI>
__device__ __forceinline__ void zd_block(const CUtensorMap* tmap, const ForceArgs& a,
                                         const Taps& taps, const BlockPos bp) {
    static_assert(V >= 2 && V <= 5, "Eqs. 3-6");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;  // uniform across the grid
    constexpr bool IC = (V == 5);
    using Z = ZDGeom<FTZ>;
    constexpr int R = FZR, NPZ = Z::NPZ;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    float* tb = reinterpret_cast<float*>(base);  // [3][NPZ][FTY][FTX]
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + Z::OFF_BAR);
    const Grid3 g = a.g;
    const TI* __restrict__ S = static_cast<const TI*>(a.S);
    const TI* __restrict__ M = static_cast<const TI*>(a.M);
    float* __restrict__ uo = static_cast<float*>(a.v);
    float* __restrict__ Do = static_cast<float*>(a.dbuf);
    float* __restrict__ do2 = static_cast<float*>(a.dbuf2);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + FTX * ty;
    // bricks from the top plane down, as zs_block (t was written bottom up)
    const int bx0 = bp.x * FTX, by0 = bp.y * FTY;
    const int bz0 = (bp.gz - 1 - bp.z) * FTZ;
    const int x = bx0 + tx, y = by0 + ty;
    const bool col_valid = (x < g.nx) && (y < g.ny);
    pdl_trigger();
    // S at this thread's voxels (static: read before the wait)
    float s0[FTZ];
#pragma unroll
    for (int k = 0; k < FTZ; ++k)
        s0[k] = (col_valid && bz0 + k < g.nz) ? ldg_as<float>(S + offs(g, x, y, bz0 + k)) : 0.0f;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)Z::TBOX);
        pdl_wait();
        tma_load_4d(base, tmap, bx0, by0, bz0 - R, 0, bar);  // planes outside: zero fill
        if (a.pf_stride > 0) {  // the block pf_stride positions ahead: its t box into L2
            const long long gx = bp.gx, gy = bp.gy;
            const long long b = bp.x + gx * (bp.y + gy * (long long)bp.z) + a.pf_stride;
            if (b < gx * gy * bp.gz) {
                const int px = (int)(b % gx) * FTX, py = (int)((b / gx) % gy) * FTY;
                const int pz = (int)(bp.gz - 1 - b / (gx * gy)) * FTZ;
                tma_prefetch_4d(tmap, px, py, pz - R, 0);
            }
        }
    }
    pdl_wait();  // every thread: u and D are written below, which the previous
                 // iteration's force pass reads (finished before the kernel before)
    __syncthreads();
    bool ok = true;
    if (tid == 0) ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (__syncthreads_or(!ok)) {
        if (tid == 0 && a.err) atomicOr(a.err, kErrTmaTimeout);
        return;
    }
    (void)mbar_try_wait(bar, 0);
    if (!col_valid) return;  // no barrier below

    // z pass down this thread's column, as zs_block: edge planes replicated
    // into the zero fill, u[c][k] written over t planes R .. R + FTZ - 1
    float w[R + 1];
#pragma unroll
    for (int t = 0; t <= R; ++t) w[t] = taps.wf[t];
    float* tcol = tb + tid;  // plane j of component c at tcol[(c * NPZ + j) * FNT]
    const int zlo = bz0 - R;
    if (zlo < 0 || zlo + NPZ > g.nz) {
        const int jlo = max(0, -zlo), jhi = min(NPZ - 1, g.nz - 1 - zlo);
        for (int c = 0; c < 3; ++c) {
            float* tc = tcol + c * NPZ * FNT;
            const float lo = tc[jlo * FNT], hi = tc[jhi * FNT];
            for (int j = 0; j < jlo; ++j) tc[j * FNT] = lo;
            for (int j = jhi + 1; j < NPZ; ++j) tc[j * FNT] = hi;
        }
    }
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

    // D per voxel: the interpolations of gm_force_body's d_at at the voxel itself
    const Interp ip(g);
    const int cs = (int)g.cs;
#pragma unroll
    for (int k = 0; k < FTZ; ++k) {
        const int z = bz0 + k;
        if (z < g.nz) {
            const float ux = tcol[(R + k) * FNT], uy = tcol[(NPZ + R + k) * FNT],
                        uz = tcol[(2 * NPZ + R + k) * FNT];
            const float wm = interp_rel(M, ip, x, ux, y, uy, z, uz, s0[k]);
            const int o = offs(g, x, y, z);
            uo[o] = ux;
            uo[o + cs] = uy;
            uo[o + 2 * cs] = uz;
            if (IC) {
                const float ws = interp_rel(S, ip, x, -ux, y, -uy, z, -uz, s0[k]);
                Do[o] = wm + ws;
                do2[o] = wm - ws;
            } else {
                Do[o] = wm;
            }
        }
    }
}

// Force pass: D with a one-voxel halo over the columns x0 - 4 .. x0 + 35 (a
// 16-byte aligned start), S with the halo of FGGeom, u (and Eq. 6's d) on the
// brick.
template <int FTZ, int V, typename TI>
struct STGeom {
    static constexpr bool IC = (V == 5);
    static constexpr int FBX = 16 / (int)sizeof(TI);
    static constexpr int FSW = FTX + 2 * FBX;
    static constexpr int DW = FTX + 8, DH = FTY + 2, DD = FTZ + 2;
    static constexpr int DBOX = DD * DH * DW * 4;                    // [DD][DH][DW] floats
    static constexpr int SBOX = DD * FSH * FSW * (int)sizeof(TI);   // [DD][FSH][FSW]
    static constexpr int UBOX = 3 * FTZ * FTY * FTX * 4;            // [3][FTZ][FTY][FTX]
    static constexpr int EBOX = IC ? FTZ * FTY * FTX * 4 : 0;       // [FTZ][FTY][FTX]
    static constexpr int OFF_S = (DBOX + 127) / 128 * 128;
    static constexpr int OFF_U = OFF_S + (SBOX + 127) / 128 * 128;
    static constexpr int OFF_E = OFF_U + (UBOX + 127) / 128 * 128;
    static constexpr int OFF_BAR = OFF_E + (EBOX + 127) / 128 * 128;
    static constexpr int SMEM = 128 + OFF_BAR + 64;
};

// One brick of the force pass (every thread of the block calls it).  a.u: u,
// a.v: v out; a.dbuf: D, a.dbuf2: Eq. 6's d.
template <int V, int FTZ, typename TI>
__device__ __forceinline__ void st_block(const CUtensorMap* dmap, const CUtensorMap* smap,
                                         const CUtensorMap* umap, const CUtensorMap* emap,
                                         const ForceArgs& a, const BlockPos bp) {
    static_assert(V >= 2 && V <= 5, "Eqs. 3-6");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;  // uniform across the grid
    using F = STGeom<FTZ, V, TI>;
    constexpr int FSW = F::FSW, DW = F::DW, DH = F::DH, FBX = F::FBX;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const float* db = reinterpret_cast<const float*>(base);             // [DD][DH][DW]
    const TI* sb = reinterpret_cast<const TI*>(base + F::OFF_S);        // [DD][FSH][FSW]
    const float* ub = reinterpret_cast<const float*>(base + F::OFF_U);  // [3][FTZ][FTY][FTX]
    const float* eb = reinterpret_cast<const float*>(base + F::OFF_E);  // [FTZ][FTY][FTX]
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + F::OFF_BAR);
    const Grid3 g = a.g;
    float* __restrict__ v = static_cast<float*>(a.v);
    const float alpha2 = (float)a.alpha2;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + FTX * ty;
    const int bx0 = bp.x * FTX, by0 = bp.y * FTY, bz0 = bp.z * FTZ;
    const int dx0 = bx0 - 4, dy0 = by0 - 1, dz0 = bz0 - 1;      // D box origin
    const int sx0 = bx0 - FBX, sy0 = by0 - 1, sz0 = bz0 - 1;    // S box origin
    pdl_trigger();
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)(F::DBOX + F::SBOX + F::UBOX + F::EBOX));
        tma_load_4d(base + F::OFF_S, smap, sx0, sy0, sz0, 0, bar);  // static
        pdl_wait();
        tma_load_4d(base, dmap, dx0, dy0, dz0, 0, bar);
        tma_load_4d(base + F::OFF_U, umap, bx0, by0, bz0, 0, bar);
        if (F::IC) tma_load_4d(base + F::OFF_E, emap, bx0, by0, bz0, 0, bar);
        if (a.pf_stride > 0) {  // the block pf_stride positions ahead: its boxes into L2
            const long long gx = bp.gx, gy = bp.gy;
            const long long b = bp.x + gx * (bp.y + gy * (long long)bp.z) + a.pf_stride;
            if (b < gx * gy * bp.gz) {
                const int px = (int)(b % gx) * FTX, py = (int)((b / gx) % gy) * FTY;
                const int pz = (int)(b / (gx * gy)) * FTZ;
                tma_prefetch_4d(dmap, px - 4, py - 1, pz - 1, 0);
                tma_prefetch_4d(smap, px - FBX, py - 1, pz - 1, 0);
                tma_prefetch_4d(umap, px, py, pz, 0);
            }
        }
    }
    pdl_wait();  // every thread: v is written below, which this iteration's x/y
                 // pass read (finished before the kernel before)
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
        // the clamped neighbours of gm_force_body's footprint, in box indices
        const int sx = x - sx0, sxm = max(x - 1, 0) - sx0, sxp = min(x + 1, g.nx - 1) - sx0;
        const int sy = y - sy0, sym = max(y - 1, 0) - sy0, syp = min(y + 1, g.ny - 1) - sy0;
        const int cx = x - dx0, cxm = max(x - 1, 0) - dx0, cxp = min(x + 1, g.nx - 1) - dx0;
        const int cy = y - dy0, cym = max(y - 1, 0) - dy0, cyp = min(y + 1, g.ny - 1) - dy0;
        const int cs = (int)g.cs;
#pragma unroll
        for (int k = 0; k < FTZ; ++k) {
            const int z = bz0 + k;
            if (z < g.nz) {
                const int pc = k + 1;
                const int pm = max(z - 1, 0) - sz0, pp = min(z + 1, g.nz - 1) - sz0;
                const TI* Sc = sb + pc * (FSH * FSW);
                const float gsx = 0.5f * ((float)Sc[sy * FSW + sxp] - (float)Sc[sy * FSW + sxm]);
                const float gsy = 0.5f * ((float)Sc[syp * FSW + sx] - (float)Sc[sym * FSW + sx]);
                const float gsz = 0.5f * ((float)sb[pp * (FSH * FSW) + sy * FSW + sx] -
                                          (float)sb[pm * (FSH * FSW) + sy * FSW + sx]);
                // grad W = grad D + grad S (Eq. 6: grad(D_m + D_s) + 2 grad S)
                const float ns = F::IC ? 2.0f : 1.0f;
                const float* Dc = db + pc * (DH * DW);
                const float dcen = Dc[cy * DW + cx];
                const float gmx = r_fma(ns, gsx, 0.5f * (Dc[cy * DW + cxp] - Dc[cy * DW + cxm]));
                const float gmy = r_fma(ns, gsy, 0.5f * (Dc[cyp * DW + cx] - Dc[cym * DW + cx]));
                const float gmz = r_fma(ns, gsz, 0.5f * (db[pp * (DH * DW) + cy * DW + cx] -
                                                         db[pm * (DH * DW) + cy * DW + cx]));
                const int bi = (k * FTY + ty) * FTX + tx;
                const float d = F::IC ? eb[bi] : dcen;
                if (a.corr) {  // reference: S (Eq. 6: the warped static image S + D_s)
                    float bref = (float)Sc[sy * FSW + sx];
                    if (F::IC) bref += 0.5f * (dcen - d);
                    corr_s.add(bref, d);
                }
                constexpr int UC = FTZ * FTY * FTX;
                const float ux = ub[bi], uy = ub[bi + UC], uz = ub[bi + 2 * UC];
                float dx, dy, dz;
                demons_force<float, V>(d, gsx, gsy, gsz, gmx, gmy, gmz, 0.0f, alpha2, dx, dy, dz);
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

}  // namespace dirk
