// dir_force_kernel.cuh -- the fused warp + gradient + force + update +
// reduction kernel (Sec. 2.5 interpolation, gradient and displacement kernels
// of the paper in one pass, plus the Sec. 2.4 reductions):
//   W(x)  = M(x + u(x))                    trilinear, clamped (Sec. 2.5)
//   d     = W - S                          (Eq. 6: M(x + h) - S(x - h))
//   grad W = grad(W - S) + grad S          (Eqs. 3-6; same clamped indices)
//   dr    = force law of Eqs. (1)-(6)      each fraction 0 where its denominator is 0
//   v     = u - dr                         total field, smoothed afterwards
//   red  += {sum d^2, sum |du|, sum |u|}   per-warp partial sums, FP64 across blocks
//
// A block of 32 x 8 threads owns a 32 x 8 x FTZ brick; each thread handles the
// FTZ voxels of its (x, y) column (FTZ = 8 for large levels, down to 1 for
// small ones so that enough blocks run).  Loads of different voxels are
// independent, so many are in flight per warp.  The static gradient uses the
// thread's column of S in registers plus x/y neighbours through L1.  Variants
// that need the gradient of the warped image (Eqs. 3-6) first compute D = W - S
// on the brick plus a one-voxel halo into shared memory (every D once per
// block), then difference it there and add the static gradient.  The warped
// image is only ever formed relative to S at the same grid point (see
// trilinear), which keeps single-precision rounding at the size of the
// intensity difference instead of the intensity.
//
// Templates: Real is the arithmetic (float, or double for verification); TI
// the image storage (float, int16 HU, double); TF the field storage (float,
// bf16, double).  Each storage combination is instantiated in its own
// translation unit (dir_force_*.cu) so that they compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "dir_common.cuh"
#include "dir_force_law.cuh"
#include "dir_launch.h"

namespace dirk {

constexpr int FTX = 32, FTY = 8, FNT = FTX * FTY;
constexpr int HX = FTX + 2, HY = FTY + 2;


// Interpolation constants of one level for the force kernel's gathers (Sec. 2.5
// software trilinear, clamped): the upper corner is one element to the right
// along x and sy / sz elements further along y / z, with sy or sz 0 on an axis
// of one voxel.  On an x axis of one voxel the weight of the right neighbour is
// 0 and that neighbour is row padding (zero in the image pool), so the read is
// harmless.
struct Interp {
    int nx1, ny1, nz1;     // n - 1
    int nxm2, nym2, nzm2;  // max(n - 2, 0): largest lower corner
    int px, pl, sy, sz;
    __device__ __forceinline__ explicit Interp(const Grid3& g)
        : nx1(g.nx - 1), ny1(g.ny - 1), nz1(g.nz - 1), nxm2(max(g.nx - 2, 0)),
          nym2(max(g.ny - 2, 0)), nzm2(max(g.nz - 2, 0)), px(g.px), pl((int)g.plane),
          sy(g.ny > 1 ? g.px : 0), sz(g.nz > 1 ? (int)g.plane : 0) {}
};

// Lower corner and weight along one axis at p = base + off: p clamped to
// [0, n-1] in offset form (exact: the bounds are small integers), corner
// floor(p) kept <= n-2 (weight 1 at the upper clamp).
template <typename Real>
__device__ __forceinline__ int ax_corner(int base, Real off, int nm1, int nm2, Real& f) {
    const Real c = r_clamp(off, Real(-base), Real(nm1 - base));
    const Real fl = r_floor(c);
    int i = base + (int)fl;
    f = c - fl;
    if (i > nm2) {
        i = nm2;
        f = Real(1);
    }
    return i;
}

// I(x + o) - ref, corners taken relative to ref (see trilinear in
// dir_common.cuh for why), lerped along x, then y, then z.
template <typename Real, typename T>
__device__ __forceinline__ Real interp_rel(const T* __restrict__ I, const Interp& q, int x, Real ox,
                                           int y, Real oy, int z, Real oz, Real ref) {
    Real fx, fy, fz;
    const int ix = ax_corner(x, ox, q.nx1, q.nxm2, fx);
    const int iy = ax_corner(y, oy, q.ny1, q.nym2, fy);
    const int iz = ax_corner(z, oz, q.nz1, q.nzm2, fz);
    const T* p0 = I + (ix + q.px * iy + q.pl * iz);
    const T* p1 = p0 + q.sy;
    const T* p2 = p0 + q.sz;
    const T* p3 = p2 + q.sy;
    const Real c000 = ldg_as<Real>(p0) - ref, c100 = ldg_as<Real>(p0 + 1) - ref;
    const Real c010 = ldg_as<Real>(p1) - ref, c110 = ldg_as<Real>(p1 + 1) - ref;
    const Real c001 = ldg_as<Real>(p2) - ref, c101 = ldg_as<Real>(p2 + 1) - ref;
    const Real c011 = ldg_as<Real>(p3) - ref, c111 = ldg_as<Real>(p3 + 1) - ref;
    const Real gx = Real(1) - fx, gy = Real(1) - fy, gz = Real(1) - fz;
    const Real v00 = r_fma(c100, fx, c000 * gx);
    const Real v10 = r_fma(c110, fx, c010 * gx);
    const Real v01 = r_fma(c101, fx, c001 * gx);
    const Real v11 = r_fma(c111, fx, c011 * gx);
    const Real v0 = r_fma(v10, fy, v00 * gy);
    const Real v1 = r_fma(v11, fy, v01 * gy);
    return r_fma(v1, fz, v0 * gz);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Prefetch into L2 the rows of the brick that block `b` (linear block index)
// will read: u (three components) over its FTZ planes, S and M over the planes
// one below to one above.  Issued for the block pf_stride positions ahead, so
// that its loads of u and S (and M near its voxels) hit L2 instead of HBM.
template <int FTZ, typename TI, typename TF>
__device__ __forceinline__ void prefetch_brick(const ForceArgs& a, long long b, int tid, int nt) {
    const Grid3& g = a.g;
    const long long gx = gridDim.x, gy = gridDim.y, total = gx * gy * gridDim.z;
    if (b >= total) return;
    const int bx = (int)(b % gx), by = (int)((b / gx) % gy), bz = (int)(b / (gx * gy));
    const int x0 = bx * FTX;
    constexpr int NU = 3 * FTZ * FTY, NS = (FTZ + 2) * FTY;
    for (int t = tid; t < NU + 2 * NS; t += nt) {
        if (t < NU) {
            const int c = t / (FTZ * FTY), r = t % (FTZ * FTY);
            const int y = by * FTY + r % FTY, z = bz * FTZ + r / FTY;
            if (y < g.ny && z < g.nz)
                prefetch_l2(static_cast<const TF*>(a.u) + (long long)c * g.cs + offs(g, x0, y, z));
        } else {
            const int r = (t - NU) % NS;
            const int y = by * FTY + r % FTY, z = clampi(bz * FTZ - 1 + r / FTY, 0, g.nz - 1);
            const TI* img = static_cast<const TI*>(t - NU < NS ? a.S : a.M);
            if (y < g.ny) prefetch_l2(img + offs(g, x0, y, z));
        }
    }
}

template <int V>
struct VT {
    static constexpr bool GM = (V == 2 || V == 3 || V == 4 || V == 5);  // warped gradient
    static constexpr bool GS = true;  // static gradient: a force term, or part of grad W
    static constexpr bool IC = (V == 5);
    static constexpr bool EV = (V == 1);
};

template <typename Real, int V, int FTZ, typename TI, typename TF>
__global__ void __launch_bounds__(FNT, 4) force_kernel(const ForceArgs a) {
    constexpr int HZ = FTZ + 2;
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;  // uniform across the grid
    using T = VT<V>;
    const Grid3 g = a.g;
    const TI* __restrict__ S = static_cast<const TI*>(a.S);
    const TI* __restrict__ M = static_cast<const TI*>(a.M);
    const TF* __restrict__ u = static_cast<const TF*>(a.u);
    TF* __restrict__ v = static_cast<TF*>(a.v);
    const Real alpha2 = (Real)a.alpha2;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + FTX * ty;
    const int bx0 = blockIdx.x * FTX, by0 = blockIdx.y * FTY, bz0 = blockIdx.z * FTZ;
    const int x = bx0 + tx, y = by0 + ty;
    const bool col_valid = (x < g.nx) && (y < g.ny);
    if (a.pf_stride > 0)
        prefetch_brick<FTZ, TI, TF>(
            a, blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z) +
                   a.pf_stride,
            tid, FNT);
    const int xc = min(x, g.nx - 1), yc = min(y, g.ny - 1);
    const int xm = max(xc - 1, 0), xp = min(xc + 1, g.nx - 1);
    const int ym = max(yc - 1, 0), yp = min(yc + 1, g.ny - 1);
    const int cs = (int)g.cs;
    const Interp ip(g);

    // D = W - S (Eq. 6: D_m + D_s with D_m = W_m - S, D_s = W_s - S) on the brick
    // plus halo; Eq. 6 also d = D_m - D_s on the brick
    __shared__ Real Wt[T::GM ? HZ : 1][T::GM ? HY : 1][T::GM ? HX : 1];
    __shared__ Real Dt[T::IC ? FTZ : 1][T::IC ? FTY : 1][T::IC ? FTX : 1];
    if constexpr (T::GM) {
#pragma unroll 2
        for (int q = tid; q < HX * HY * HZ; q += FNT) {
            const int hz = q / (HX * HY);
            const int r = q - hz * (HX * HY);
            const int hy = r / HX, hx = r - hy * HX;
            const int gx = clampi(bx0 + hx - 1, 0, g.nx - 1);
            const int gy = clampi(by0 + hy - 1, 0, g.ny - 1);
            const int gz = clampi(bz0 + hz - 1, 0, g.nz - 1);
            const int o = offs(g, gx, gy, gz);
            const Real ux = ldg_as<Real>(u + o), uy = ldg_as<Real>(u + o + cs), uz = ldg_as<Real>(u + o + 2 * cs);
            const Real sref = ldg_as<Real>(S + o);
            const Real wm = interp_rel(M, ip, gx, ux, gy, uy, gz, uz, sref);
            if (T::IC) {
                const Real ws = interp_rel(S, ip, gx, -ux, gy, -uy, gz, -uz, sref);
                Wt[hz][hy][hx] = wm + ws;
                if (hx >= 1 && hx <= FTX && hy >= 1 && hy <= FTY && hz >= 1 && hz <= FTZ)
                    Dt[T::IC ? hz - 1 : 0][hy - 1][hx - 1] = wm - ws;
            } else {
                Wt[hz][hy][hx] = wm;
            }
        }
        __syncthreads();
    }

    // this thread's column of S (and M for Eq. 2), planes bz0-1 .. bz0+FTZ, clamped
    Real scol[FTZ + 2];
    Real mcol[T::EV ? FTZ + 2 : 1];
    if (T::GS) {
#pragma unroll
        for (int k = 0; k < FTZ + 2; ++k)
            scol[k] = ldg_as<Real>(S + offs(g, xc, yc, clampi(bz0 + k - 1, 0, g.nz - 1)));
    }
    if (T::EV) {
#pragma unroll
        for (int k = 0; k < FTZ + 2; ++k)
            mcol[k] = ldg_as<Real>(M + offs(g, xc, yc, clampi(bz0 + k - 1, 0, g.nz - 1)));
    }

    Real sd2 = 0, sdu = 0, su = 0;  // per-thread partial sums
    CorrSums<Real> corr_s;          // with a.corr: the correlation sums
    if (col_valid) {
#pragma unroll
        for (int k = 0; k < FTZ; ++k) {
            const int z = bz0 + k;
            if (z < g.nz) {
                const int o = offs(g, x, y, z);
                const Real ux = ldg_as<Real>(u + o), uy = ldg_as<Real>(u + o + cs), uz = ldg_as<Real>(u + o + 2 * cs);
                Real gsx = 0, gsy = 0, gsz = 0, gmx = 0, gmy = 0, gmz = 0, bm = 0, d;
                if (T::GS) {
                    const int ro = offs(g, 0, y, z);
                    gsx = Real(0.5) * (ldg_as<Real>(S + ro + xp) - ldg_as<Real>(S + ro + xm));
                    gsy = Real(0.5) * (ldg_as<Real>(S + offs(g, x, yp, z)) - ldg_as<Real>(S + offs(g, x, ym, z)));
                    gsz = Real(0.5) * (scol[k + 2] - scol[k]);
                }
                if (T::EV) {
                    const int ro = offs(g, 0, y, z);
                    const Real mx = Real(0.5) * (ldg_as<Real>(M + ro + xp) - ldg_as<Real>(M + ro + xm));
                    const Real my =
                        Real(0.5) * (ldg_as<Real>(M + offs(g, x, yp, z)) - ldg_as<Real>(M + offs(g, x, ym, z)));
                    const Real mz = Real(0.5) * (mcol[k + 2] - mcol[k]);
                    bm = r_sqrt(mx * mx + my * my + mz * mz);
                }
                if constexpr (T::GM) {
                    // grad W = grad D + grad S (Eq. 6: grad(W_m + W_s) = grad(D_m + D_s) + 2 grad S)
                    const Real ns = T::IC ? Real(2) : Real(1);
                    gmx = r_fma(ns, gsx, Real(0.5) * (Wt[k + 1][ty + 1][tx + 2] - Wt[k + 1][ty + 1][tx]));
                    gmy = r_fma(ns, gsy, Real(0.5) * (Wt[k + 1][ty + 2][tx + 1] - Wt[k + 1][ty][tx + 1]));
                    gmz = r_fma(ns, gsz, Real(0.5) * (Wt[k + 2][ty + 1][tx + 1] - Wt[k][ty + 1][tx + 1]));
                    if (T::IC)
                        d = Dt[T::IC ? k : 0][ty][tx];
                    else
                        d = Wt[k + 1][ty + 1][tx + 1];
                } else {
                    d = interp_rel(M, ip, x, ux, y, uy, z, uz, scol[k + 1]);
                }
                if (a.corr) {  // reference: S (Eq. 6: the warped static image S + D_s)
                    Real bref = scol[k + 1];
                    if constexpr (T::IC) bref += Real(0.5) * (Wt[k + 1][ty + 1][tx + 1] - d);
                    corr_s.add(bref, d);
                }
                Real dx, dy, dz;
                demons_force<Real, V>(d, gsx, gsy, gsz, gmx, gmy, gmz, bm, alpha2, dx, dy, dz);
                dx = -dx;
                dy = -dy;
                dz = -dz;
                sd2 += d * d;
                sdu += r_norm_fast(dx * dx + dy * dy + dz * dz);
                su += r_norm_fast(ux * ux + uy * uy + uz * uz);
                v[o] = st_as<TF>(ux + dx);
                v[o + cs] = st_as<TF>(uy + dy);
                v[o + 2 * cs] = st_as<TF>(uz + dz);
            }
        }
    }
    block_reduce3_atomic<FNT, Real>(sd2, sdu, su, a.red);
    if (a.corr) block_reduce4_atomic<FNT, Real>(corr_s, a.corr);
}

template <typename Real, typename TI, typename TF, int FTZ>
static cudaError_t launch_z(int variant, const ForceArgs& a, cudaStream_t s) {
    const dim3 block(FTX, FTY, 1);
    const dim3 grid((a.g.nx + FTX - 1) / FTX, (a.g.ny + FTY - 1) / FTY, (a.g.nz + FTZ - 1) / FTZ);
    switch (variant) {
        case 0: force_kernel<Real, 0, FTZ, TI, TF><<<grid, block, 0, s>>>(a); break;
        case 1: force_kernel<Real, 1, FTZ, TI, TF><<<grid, block, 0, s>>>(a); break;
        case 2: force_kernel<Real, 2, FTZ, TI, TF><<<grid, block, 0, s>>>(a); break;
        case 3: force_kernel<Real, 3, FTZ, TI, TF><<<grid, block, 0, s>>>(a); break;
        case 4: force_kernel<Real, 4, FTZ, TI, TF><<<grid, block, 0, s>>>(a); break;
        case 5: force_kernel<Real, 5, FTZ, TI, TF><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename Real, typename TI, typename TF>
static cudaError_t launch_force_types(int variant, const ForceArgs& a, cudaStream_t s) {
    switch (a.depth) {
        case 8: return launch_z<Real, TI, TF, 8>(variant, a, s);
        case 4: return launch_z<Real, TI, TF, 4>(variant, a, s);
        case 2: return launch_z<Real, TI, TF, 2>(variant, a, s);
        case 1: return launch_z<Real, TI, TF, 1>(variant, a, s);
        default: return cudaErrorInvalidValue;
    }
}

// one per translation unit
cudaError_t launch_force_tma(int variant, const ForceArgs& a, cudaStream_t s);   // Eqs. 1-2, f32
cudaError_t launch_force_f32(int variant, const ForceArgs& a, cudaStream_t s);   // f32 / f32
cudaError_t launch_force_f64(int variant, const ForceArgs& a, cudaStream_t s);   // f64 / f64
cudaError_t launch_force_i16(int variant, const ForceArgs& a, cudaStream_t s);   // i16 / f32, i16 / bf16
cudaError_t launch_force_bf16(int variant, const ForceArgs& a, cudaStream_t s);  // f32 / bf16

}  // namespace dirk
