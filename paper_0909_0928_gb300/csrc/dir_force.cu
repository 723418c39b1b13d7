// dir_force.cu -- fused warp + gradient + force + update + reduction kernel.
//
// One launch performs the paper's interpolation, gradient and displacement
// kernels (Sec. 2.5) for one iteration at one level, plus the comparison
// reductions of Sec. 2.4:
//   W(x)  = M(x + u(x))                    trilinear, clamped (Sec. 2.5)
//   d     = W - S                          (Eq. 6: M(x + h) - S(x - h))
//   dr    = force law of Eqs. (1)-(6)      each fraction 0 where its denominator is 0
//   v     = u - dr                         total field, smoothed afterwards
//   red  += {sum d^2, sum |du|, sum |u|}   FP64 atomics, one per block
//
// A block of 32 x 8 threads owns a 32 x 8 x FTZ brick; each thread handles the
// FTZ voxels of its (x, y) column (FTZ = 8 for large levels, down to 1 for
// small ones so that enough blocks run).  Loads of different voxels are independent,
// so many are in flight per warp.  The static gradient uses the thread's
// column of S in registers plus x/y neighbours through L1.  Variants that need
// the gradient of the warped image (Eqs. 3-6) first compute W on the brick
// plus a one-voxel halo into shared memory (every W once per block), then
// difference it there.
#include <cuda_runtime.h>

#include "dir_common.cuh"
#include "dir_force_law.cuh"
#include "dir_launch.h"

namespace dirk {

constexpr int FTX = 32, FTY = 8, FNT = FTX * FTY;
constexpr int HX = FTX + 2, HY = FTY + 2;

template <int V>
struct VT {
    static constexpr bool GS = (V == 0 || V == 1 || V == 3 || V == 4);  // static gradient
    static constexpr bool GM = (V == 2 || V == 3 || V == 4 || V == 5);  // warped gradient
    static constexpr bool IC = (V == 5);
    static constexpr bool EV = (V == 1);
};

template <typename Real, int V, int FTZ>
__global__ void __launch_bounds__(FNT, 4) force_kernel(const ForceArgs a) {
    constexpr int HZ = FTZ + 2;
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;  // uniform across the grid
    using T = VT<V>;
    const Grid3 g = a.g;
    const Real* __restrict__ S = static_cast<const Real*>(a.S);
    const Real* __restrict__ M = static_cast<const Real*>(a.M);
    const Real* __restrict__ u = static_cast<const Real*>(a.u);
    Real* __restrict__ v = static_cast<Real*>(a.v);
    const Real alpha2 = (Real)a.alpha2;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + FTX * ty;
    const int bx0 = blockIdx.x * FTX, by0 = blockIdx.y * FTY, bz0 = blockIdx.z * FTZ;
    const int x = bx0 + tx, y = by0 + ty;
    const bool col_valid = (x < g.nx) && (y < g.ny);
    const int xc = min(x, g.nx - 1), yc = min(y, g.ny - 1);
    const int xm = max(xc - 1, 0), xp = min(xc + 1, g.nx - 1);
    const int ym = max(yc - 1, 0), yp = min(yc + 1, g.ny - 1);
    const int cs = (int)g.cs;

    // W (Eq. 6: W_m + W_s) on the brick plus halo; Eq. 6 also W_m - W_s on the brick
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
            const Real ux = __ldg(u + o), uy = __ldg(u + o + cs), uz = __ldg(u + o + 2 * cs);
            const Real wm = trilinear(M, g, gx, ux, gy, uy, gz, uz);
            if (T::IC) {
                const Real ws = trilinear(S, g, gx, -ux, gy, -uy, gz, -uz);
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
            scol[k] = __ldg(S + offs(g, xc, yc, clampi(bz0 + k - 1, 0, g.nz - 1)));
    }
    if (T::EV) {
#pragma unroll
        for (int k = 0; k < FTZ + 2; ++k)
            mcol[k] = __ldg(M + offs(g, xc, yc, clampi(bz0 + k - 1, 0, g.nz - 1)));
    }

    Real sd2 = 0, sdu = 0, su = 0;  // per-thread partial sums
    if (col_valid) {
#pragma unroll
        for (int k = 0; k < FTZ; ++k) {
            const int z = bz0 + k;
            if (z < g.nz) {
                const int o = offs(g, x, y, z);
                const Real ux = __ldg(u + o), uy = __ldg(u + o + cs), uz = __ldg(u + o + 2 * cs);
                Real gsx = 0, gsy = 0, gsz = 0, gmx = 0, gmy = 0, gmz = 0, bm = 0, d;
                if (T::GS) {
                    const int ro = offs(g, 0, y, z);
                    gsx = Real(0.5) * (__ldg(S + ro + xp) - __ldg(S + ro + xm));
                    gsy = Real(0.5) * (__ldg(S + offs(g, x, yp, z)) - __ldg(S + offs(g, x, ym, z)));
                    gsz = Real(0.5) * (scol[k + 2] - scol[k]);
                }
                if (T::EV) {
                    const int ro = offs(g, 0, y, z);
                    const Real mx = Real(0.5) * (__ldg(M + ro + xp) - __ldg(M + ro + xm));
                    const Real my =
                        Real(0.5) * (__ldg(M + offs(g, x, yp, z)) - __ldg(M + offs(g, x, ym, z)));
                    const Real mz = Real(0.5) * (mcol[k + 2] - mcol[k]);
                    bm = r_sqrt(mx * mx + my * my + mz * mz);
                }
                if constexpr (T::GM) {
                    gmx = Real(0.5) * (Wt[k + 1][ty + 1][tx + 2] - Wt[k + 1][ty + 1][tx]);
                    gmy = Real(0.5) * (Wt[k + 1][ty + 2][tx + 1] - Wt[k + 1][ty][tx + 1]);
                    gmz = Real(0.5) * (Wt[k + 2][ty + 1][tx + 1] - Wt[k][ty + 1][tx + 1]);
                    if (T::IC)
                        d = Dt[T::IC ? k : 0][ty][tx];
                    else
                        d = Wt[k + 1][ty + 1][tx + 1] - (T::GS ? scol[k + 1] : __ldg(S + o));
                } else {
                    const Real w = trilinear(M, g, x, ux, y, uy, z, uz);
                    d = w - scol[k + 1];
                }
                Real dx, dy, dz;
                demons_force<Real, V>(d, gsx, gsy, gsz, gmx, gmy, gmz, bm, alpha2, dx, dy, dz);
                dx = -dx;
                dy = -dy;
                dz = -dz;
                sd2 += d * d;
                sdu += r_norm_fast(dx * dx + dy * dy + dz * dz);
                su += r_norm_fast(ux * ux + uy * uy + uz * uz);
                v[o] = ux + dx;
                v[o + cs] = uy + dy;
                v[o + 2 * cs] = uz + dz;
            }
        }
    }
    block_reduce3_atomic<FNT, Real>(sd2, sdu, su, a.red);
}

template <typename Real, int FTZ>
static cudaError_t launch_z(int variant, const ForceArgs& a, cudaStream_t s) {
    const dim3 block(FTX, FTY, 1);
    const dim3 grid((a.g.nx + FTX - 1) / FTX, (a.g.ny + FTY - 1) / FTY, (a.g.nz + FTZ - 1) / FTZ);
    switch (variant) {
        case 0: force_kernel<Real, 0, FTZ><<<grid, block, 0, s>>>(a); break;
        case 1: force_kernel<Real, 1, FTZ><<<grid, block, 0, s>>>(a); break;
        case 2: force_kernel<Real, 2, FTZ><<<grid, block, 0, s>>>(a); break;
        case 3: force_kernel<Real, 3, FTZ><<<grid, block, 0, s>>>(a); break;
        case 4: force_kernel<Real, 4, FTZ><<<grid, block, 0, s>>>(a); break;
        case 5: force_kernel<Real, 5, FTZ><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Brick depth: the deepest of 8, 4, 2, 1 that still gives at least `waves`
// waves of resident blocks (4 per SM), so small levels spread over the GPU.
int force_brick_depth(const Grid3& g, int num_sms, int waves) {
    const long long bxy = (long long)((g.nx + FTX - 1) / FTX) * ((g.ny + FTY - 1) / FTY);
    const long long want = (long long)waves * 4 * num_sms;
    for (int d = 8; d > 1; d /= 2)
        if (bxy * ((g.nz + d - 1) / d) >= want) return d;
    return 1;
}

template <typename Real>
static cudaError_t launch_t(int variant, const ForceArgs& a, cudaStream_t s) {
    switch (a.depth) {
        case 8: return launch_z<Real, 8>(variant, a, s);
        case 4: return launch_z<Real, 4>(variant, a, s);
        case 2: return launch_z<Real, 2>(variant, a, s);
        case 1: return launch_z<Real, 1>(variant, a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_force(int variant, bool fp64, const ForceArgs& a, cudaStream_t s) {
    return fp64 ? launch_t<double>(variant, a, s) : launch_t<float>(variant, a, s);
}

}  // namespace dirk
