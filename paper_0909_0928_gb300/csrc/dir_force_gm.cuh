// dir_force_gm.cuh -- the force work of Eqs. (3)-(6) on a brick whose u
// (with a one-voxel halo) and S (with its halo) already sit in shared memory:
// D = W - S (Eq. 6: D_m + D_s, and d = D_m - D_s) on the brick plus a
// one-voxel halo, the gradient of the warped image from it, the force, the
// update and the reductions.  Shared by the TMA-fed force kernel (u copied
// from the field) and the split kernel (u formed by the Gaussian's z pass).
#pragma once

#include <cuda_runtime.h>

#include "dir_force_kernel.cuh"

namespace dirk {

constexpr int FSH = FTY + 2;           // image box rows: y0 - 1 .. y0 + 8

// Shared-memory geometry: the u box spans x0 - 4 .. x0 + 35 (a 16-byte
// aligned start), y0 - 1 .. y0 + 8 and z0 - 1 .. z0 + FTZ; S the same rows and
// planes with FBX columns of x halo; D the brick plus a one-voxel halo.
template <int FTZ, int V, typename TI>
struct FGGeom {
    static constexpr bool IC = (V == 5);
    static constexpr int FBX = 16 / (int)sizeof(TI);
    static constexpr int FSW = FTX + 2 * FBX;
    static constexpr int UW = FTX + 8, UH = FTY + 2, UD = FTZ + 2;  // u box: x0-4 .. x0+35
    static constexpr int UBOX = 3 * UD * UH * UW * 4;             // [3][UD][UH][UW] floats
    static constexpr int SBOX = UD * FSH * FSW * (int)sizeof(TI);  // [UD][FSH][FSW]
    static constexpr int HX = FTX + 2, HY = FTY + 2, HZ = FTZ + 2;
    static constexpr int WT = HZ * HY * HX * 4;                    // D on brick + halo
    static constexpr int DT = 0;                                   // d stays in registers
    static constexpr int OFF_S = (UBOX + 127) / 128 * 128;
    static constexpr int OFF_W = OFF_S + (SBOX + 127) / 128 * 128;
    static constexpr int OFF_D = OFF_W + (WT + 127) / 128 * 128;
    static constexpr int OFF_BAR = OFF_D + (DT + 127) / 128 * 128;
    static constexpr int SMEM = 128 + OFF_BAR + 64;
};

// After the block's boxes have arrived: ub points at plane z0 - 1, row y0 - 1,
// column x0 - 4 of component 0 of u, components UC floats apart; rows of UW
// floats and planes of UH rows as in FGGeom.  sb is the S box, wt the D tile.
// Every thread of the block calls it (one barrier inside).
template <int V, int FTZ, typename TI, int UC>
__device__ __forceinline__ void gm_force_body(const ForceArgs& a, const float* __restrict__ ub,
                                              const TI* __restrict__ sb, float* __restrict__ wt,
                                              const BlockPos bp) {
    using F = FGGeom<FTZ, V, TI>;
    constexpr int FSW = F::FSW, UW = F::UW, UH = F::UH;
    constexpr int HX = F::HX, HY = F::HY, HZ = F::HZ;
    const Grid3 g = a.g;
    const TI* __restrict__ S = static_cast<const TI*>(a.S);
    const TI* __restrict__ M = static_cast<const TI*>(a.M);
    float* __restrict__ v = static_cast<float*>(a.v);
    const float alpha2 = (float)a.alpha2;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + FTX * ty;
    const int bx0 = bp.x * FTX, by0 = bp.y * FTY, bz0 = bp.z * FTZ;
    const int ux0 = bx0 - 4, uy0 = by0 - 1, uz0 = bz0 - 1;     // u box origin
    const int sx0 = bx0 - F::FBX, sy0 = by0 - 1, sz0 = bz0 - 1;  // S box origin
    const Interp ip(g);

    // D (= W - S) at one clamped position of the brick + halo footprint; all
    // reads from the boxes (every clamped position lies inside them)
    auto d_at = [&](int gx, int gy, int gz, float& dd) -> float {
        const int ui = ((gz - uz0) * UH + (gy - uy0)) * UW + (gx - ux0);
        const float ux = ub[ui], uy = ub[ui + UC], uz = ub[ui + 2 * UC];
        const float sref = (float)sb[((gz - sz0) * FSH + (gy - sy0)) * FSW + (gx - sx0)];
        const float wm = interp_rel(M, ip, gx, ux, gy, uy, gz, uz, sref);
        if (F::IC) {
            const float ws = interp_rel(S, ip, gx, -ux, gy, -uy, gz, -uz, sref);
            dd = wm - ws;
            return wm + ws;
        }
        dd = wm;
        return wm;
    };
    const int x = bx0 + tx, y = by0 + ty;
    const bool col_valid = (x < g.nx) && (y < g.ny);
    const int xc = min(x, g.nx - 1), yc = min(y, g.ny - 1);
    // this thread's own column, planes bz0-1 .. bz0+FTZ: D kept in registers
    // (for the z gradient and d) and written to the tile for the neighbours
    float dcol[FTZ + 2];  // D (Eq. 6: D_m + D_s)
    float dd[FTZ];        // d at the brick's planes (Eq. 6: D_m - D_s)
#pragma unroll
    for (int h = 0; h < FTZ + 2; ++h) {
        float t;
        dcol[h] = d_at(xc, yc, clampi(bz0 + h - 1, 0, g.nz - 1), t);
        if (h >= 1 && h <= FTZ) dd[h - 1] = t;
        wt[(h * HY + (ty + 1)) * HX + (tx + 1)] = dcol[h];
    }
    // the 2 (HX + HY) - 4 = 84 border columns of the footprint, FTZ + 2 planes
    // each, spread over all threads
    constexpr int NB = 2 * (HX + HY) - 4;
    for (int q = tid; q < NB * HZ; q += FNT) {
        const int hz = q / NB, b = q - hz * NB;
        int hx, hy;
        if (b < HX) {
            hx = b;
            hy = 0;
        } else if (b < 2 * HX) {
            hx = b - HX;
            hy = HY - 1;
        } else if (b < 2 * HX + (HY - 2)) {
            hx = 0;
            hy = 1 + (b - 2 * HX);
        } else {
            hx = HX - 1;
            hy = 1 + (b - 2 * HX - (HY - 2));
        }
        float t;
        wt[(hz * HY + hy) * HX + hx] =
            d_at(clampi(bx0 + hx - 1, 0, g.nx - 1), clampi(by0 + hy - 1, 0, g.ny - 1),
                 clampi(bz0 + hz - 1, 0, g.nz - 1), t);
    }
    __syncthreads();

    const int sx = xc - sx0, sxm = max(xc - 1, 0) - sx0, sxp = min(xc + 1, g.nx - 1) - sx0;
    const int sy = yc - sy0, sym = max(yc - 1, 0) - sy0, syp = min(yc + 1, g.ny - 1) - sy0;
    const int cs = (int)g.cs;
    float sd2 = 0.0f, sdu = 0.0f, su = 0.0f;
    CorrSums<float> corr_s;  // with a.corr: the correlation sums
    if (col_valid) {
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
                // grad W = grad D + grad S (Eq. 6: grad(D_m + D_s) + 2 grad S); the
                // footprint's clamped positions make the neighbours of an edge
                // voxel the clamped ones, as in force_kernel
                const float ns = F::IC ? 2.0f : 1.0f;
                const float* W1 = wt + ((k + 1) * HY + (ty + 1)) * HX + (tx + 1);
                const float gmx = r_fma(ns, gsx, 0.5f * (W1[1] - W1[-1]));
                const float gmy = r_fma(ns, gsy, 0.5f * (W1[HX] - W1[-HX]));
                const float gmz = r_fma(ns, gsz, 0.5f * (dcol[k + 2] - dcol[k]));
                const float d = dd[k];
                if (a.corr) {  // reference: S (Eq. 6: the warped static image S + D_s)
                    float bref = (float)Sc[sy * FSW + sx];
                    if (F::IC) bref += 0.5f * (dcol[k + 1] - d);
                    corr_s.add(bref, d);
                }
                const int ui = (((k + 1) * UH) + (ty + 1)) * UW + (tx + 4);
                const float ux = ub[ui], uy = ub[ui + UC], uz = ub[ui + 2 * UC];
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
