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
// A block owns a 32 x 8 column tile in (x, y) and marches through a chunk of z
// planes.  Static gradients use a rolling z window in registers and x/y
// neighbours through L1.  Variants that need the gradient of the warped image
// (Eqs. 3-6) compute W for the next plane on the tile plus a one-voxel halo
// into a double-buffered shared-memory plane, so every W is computed once per
// block and plane; z neighbours roll through registers.
#include <cuda_runtime.h>

#include "dir_common.cuh"
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

__device__ __forceinline__ void term(float d, float gx, float gy, float gz, float den, float& ox,
                                     float& oy, float& oz) {
    if (den == 0.0f) {
        ox = oy = oz = 0.0f;
    } else {
        const float c = d / den;
        ox = c * gx;
        oy = c * gy;
        oz = c * gz;
    }
}

// dr of Eqs. (1)-(6).  gs: static gradient, gm: warped-image gradient (for
// Eq. 6 the gradient of W_m + W_s), b: |grad M| on the grid (Eq. 2).
template <int V>
__device__ __forceinline__ void demons_force(float d, float gsx, float gsy, float gsz, float gmx,
                                             float gmy, float gmz, float b, float alpha2,
                                             float& dx, float& dy, float& dz) {
    const float d2 = d * d;
    if (V == 0) {
        term(d, gsx, gsy, gsz, d2 + (gsx * gsx + gsy * gsy + gsz * gsz), dx, dy, dz);
    } else if (V == 1) {
        const float gs2 = gsx * gsx + gsy * gsy + gsz * gsz;
        const float a = sqrtf(gs2);
        const float s = a * a + b * b;
        const float den = (2.0f * d2 + s) * s;
        if (den == 0.0f) {
            dx = dy = dz = 0.0f;
        } else {
            const float c = 4.0f * d * a * b / den;
            dx = c * gsx;
            dy = c * gsy;
            dz = c * gsz;
        }
    } else if (V == 2 || V == 5) {
        term(d, gmx, gmy, gmz, d2 + (gmx * gmx + gmy * gmy + gmz * gmz), dx, dy, dz);
    } else {
        const float ad2 = (V == 4) ? alpha2 * d2 : d2;
        float px, py, pz, qx, qy, qz;
        term(d, gsx, gsy, gsz, ad2 + (gsx * gsx + gsy * gsy + gsz * gsz), px, py, pz);
        term(d, gmx, gmy, gmz, ad2 + (gmx * gmx + gmy * gmy + gmz * gmz), qx, qy, qz);
        dx = px + qx;
        dy = py + qy;
        dz = pz + qz;
    }
}

template <int V>
__global__ void __launch_bounds__(FNT) force_kernel(const ForceArgs a) {
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;  // uniform across the grid
    using T = VT<V>;
    const Grid3 g = a.g;
    const float* __restrict__ S = a.S;
    const float* __restrict__ M = a.M;
    const float* __restrict__ u = a.u;
    float* __restrict__ v = a.v;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + FTX * ty;
    const int bx0 = blockIdx.x * FTX, by0 = blockIdx.y * FTY;
    const int x = bx0 + tx, y = by0 + ty;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nz);
    const bool valid = (x < g.nx) && (y < g.ny);
    const int xc = min(x, g.nx - 1), yc = min(y, g.ny - 1);
    const int xm = max(xc - 1, 0), xp = min(xc + 1, g.nx - 1);
    const int ym = max(yc - 1, 0), yp = min(yc + 1, g.ny - 1);
    const long long cs = g.cs;

    float sd2 = 0.0f, sdu = 0.0f, su = 0.0f;

    // rolling z windows (centre column of this thread)
    float s_m1 = 0.f, s_0 = 0.f, s_p1 = 0.f;  // static image, for grad S
    float m_m1 = 0.f, m_0 = 0.f, m_p1 = 0.f;  // moving image on the grid, for |grad M|
    if (T::GS) {
        s_m1 = __ldg(S + offs(g, xc, yc, max(z0 - 1, 0)));
        s_0 = __ldg(S + offs(g, xc, yc, z0));
    }
    if (T::EV) {
        m_m1 = __ldg(M + offs(g, xc, yc, max(z0 - 1, 0)));
        m_0 = __ldg(M + offs(g, xc, yc, z0));
    }

    if constexpr (T::GM) {
        __shared__ float Wp[2][HY][HX];               // W (Eq. 6: W_m + W_s), tile + halo
        __shared__ float Dp[T::IC ? 2 : 1][FTY][FTX];  // Eq. 6: W_m - W_s at the tile
        auto fill = [&](int zz, int buf) {
            const int zcl = clampi(zz, 0, g.nz - 1);
            for (int q = tid; q < HX * HY; q += FNT) {
                const int hy = q / HX, hx = q - hy * HX;
                const int gx = clampi(bx0 + hx - 1, 0, g.nx - 1);
                const int gy = clampi(by0 + hy - 1, 0, g.ny - 1);
                const long long o = offs(g, gx, gy, zcl);
                const float ux = __ldg(u + o), uy = __ldg(u + o + cs), uz = __ldg(u + o + 2 * cs);
                const float wm = trilinear(M, g, gx + ux, gy + uy, zcl + uz);
                if (T::IC) {
                    const float ws = trilinear(S, g, gx - ux, gy - uy, zcl - uz);
                    Wp[buf][hy][hx] = wm + ws;
                    if (hx >= 1 && hx <= FTX && hy >= 1 && hy <= FTY)
                        Dp[T::IC ? buf : 0][hy - 1][hx - 1] = wm - ws;
                } else {
                    Wp[buf][hy][hx] = wm;
                }
            }
        };
        fill(z0 - 1, 1);
        __syncthreads();
        float w_m1 = Wp[1][ty + 1][tx + 1];
        fill(z0, 0);
        __syncthreads();
        float w_0 = Wp[0][ty + 1][tx + 1];
        int b = 0;
        for (int z = z0; z < z1; ++z) {
            const int zn = min(z + 1, g.nz - 1);
            if (T::GS) s_p1 = __ldg(S + offs(g, xc, yc, zn));
            fill(z + 1, b ^ 1);
            __syncthreads();
            const float w_p1 = Wp[b ^ 1][ty + 1][tx + 1];
            if (valid) {
                const long long o = offs(g, x, y, z);
                const float ux = __ldg(u + o), uy = __ldg(u + o + cs), uz = __ldg(u + o + 2 * cs);
                const float gmx = 0.5f * (Wp[b][ty + 1][tx + 2] - Wp[b][ty + 1][tx]);
                const float gmy = 0.5f * (Wp[b][ty + 2][tx + 1] - Wp[b][ty][tx + 1]);
                const float gmz = 0.5f * (w_p1 - w_m1);
                float gsx = 0.f, gsy = 0.f, gsz = 0.f;
                if (T::GS) {
                    const long long ro = offs(g, 0, yc, z);
                    gsx = 0.5f * (__ldg(S + ro + xp) - __ldg(S + ro + xm));
                    gsy = 0.5f * (__ldg(S + offs(g, xc, yp, z)) - __ldg(S + offs(g, xc, ym, z)));
                    gsz = 0.5f * (s_p1 - s_m1);
                }
                float d;
                if (T::IC) {
                    d = Dp[T::IC ? b : 0][ty][tx];
                } else {
                    d = w_0 - (T::GS ? s_0 : __ldg(S + o));
                }
                float dx, dy, dz;
                demons_force<V>(d, gsx, gsy, gsz, gmx, gmy, gmz, 0.0f, a.alpha2, dx, dy, dz);
                dx = -dx;
                dy = -dy;
                dz = -dz;
                sd2 += d * d;
                sdu += sqrtf(dx * dx + dy * dy + dz * dz);
                su += sqrtf(ux * ux + uy * uy + uz * uz);
                v[o] = ux + dx;
                v[o + cs] = uy + dy;
                v[o + 2 * cs] = uz + dz;
            }
            __syncthreads();
            w_m1 = w_0;
            w_0 = w_p1;
            if (T::GS) {
                s_m1 = s_0;
                s_0 = s_p1;
            }
            b ^= 1;
        }
    } else {
        for (int z = z0; z < z1; ++z) {
            const int zn = min(z + 1, g.nz - 1);
            s_p1 = __ldg(S + offs(g, xc, yc, zn));
            if (T::EV) m_p1 = __ldg(M + offs(g, xc, yc, zn));
            if (valid) {
                const long long o = offs(g, x, y, z);
                const float ux = __ldg(u + o), uy = __ldg(u + o + cs), uz = __ldg(u + o + 2 * cs);
                const float w = trilinear(M, g, x + ux, y + uy, z + uz);
                const long long ro = offs(g, 0, y, z);
                const float gsx = 0.5f * (__ldg(S + ro + xp) - __ldg(S + ro + xm));
                const float gsy = 0.5f * (__ldg(S + offs(g, x, yp, z)) - __ldg(S + offs(g, x, ym, z)));
                const float gsz = 0.5f * (s_p1 - s_m1);
                float bm = 0.0f;
                if (T::EV) {
                    const float mx = 0.5f * (__ldg(M + ro + xp) - __ldg(M + ro + xm));
                    const float my = 0.5f * (__ldg(M + offs(g, x, yp, z)) - __ldg(M + offs(g, x, ym, z)));
                    const float mz = 0.5f * (m_p1 - m_m1);
                    bm = sqrtf(mx * mx + my * my + mz * mz);
                }
                const float d = w - s_0;
                float dx, dy, dz;
                demons_force<V>(d, gsx, gsy, gsz, 0.f, 0.f, 0.f, bm, a.alpha2, dx, dy, dz);
                dx = -dx;
                dy = -dy;
                dz = -dz;
                sd2 += d * d;
                sdu += sqrtf(dx * dx + dy * dy + dz * dz);
                su += sqrtf(ux * ux + uy * uy + uz * uz);
                v[o] = ux + dx;
                v[o + cs] = uy + dy;
                v[o + 2 * cs] = uz + dz;
            }
            s_m1 = s_0;
            s_0 = s_p1;
            if (T::EV) {
                m_m1 = m_0;
                m_0 = m_p1;
            }
        }
    }
    block_reduce3_atomic<FNT>(sd2, sdu, su, a.red);
}

int force_zchunk(int variant, const Grid3& g, int num_sms) {
    const long long bxy = (long long)((g.nx + FTX - 1) / FTX) * ((g.ny + FTY - 1) / FTY);
    const long long target = 8LL * num_sms;  // resident blocks of 256 threads, about
    long long chunks = (target + bxy - 1) / bxy;
    if (chunks < 1) chunks = 1;
    int zc = (int)((g.nz + chunks - 1) / chunks);
    const bool gm = (variant >= 2);
    const int zmin = gm ? 8 : 4;
    if (zc < zmin) zc = zmin;
    if (zc > g.nz) zc = g.nz;
    return zc < 1 ? 1 : zc;
}

cudaError_t launch_force(int variant, const ForceArgs& a, cudaStream_t s) {
    const dim3 block(FTX, FTY, 1);
    const dim3 grid((a.g.nx + FTX - 1) / FTX, (a.g.ny + FTY - 1) / FTY,
                    (a.g.nz + a.zchunk - 1) / a.zchunk);
    switch (variant) {
        case 0: force_kernel<0><<<grid, block, 0, s>>>(a); break;
        case 1: force_kernel<1><<<grid, block, 0, s>>>(a); break;
        case 2: force_kernel<2><<<grid, block, 0, s>>>(a); break;
        case 3: force_kernel<3><<<grid, block, 0, s>>>(a); break;
        case 4: force_kernel<4><<<grid, block, 0, s>>>(a); break;
        case 5: force_kernel<5><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dirk
