// dir_force_law.cuh -- the demons force of Eqs. (1)-(6), per voxel, shared by
// the force kernel and the fused iteration kernel.
#pragma once

#include "dir_common.cuh"

namespace dirk {

template <typename Real>
__device__ __forceinline__ void term(Real d, Real gx, Real gy, Real gz, Real den, Real& ox,
                                     Real& oy, Real& oz) {
    if (den == Real(0)) {
        ox = oy = oz = Real(0);
    } else {
        const Real c = r_div(d, den);
        ox = c * gx;
        oy = c * gy;
        oz = c * gz;
    }
}

// dr of Eqs. (1)-(6).  gs: static gradient, gm: warped-image gradient (for
// Eq. 6 the gradient of W_m + W_s), b: |grad M| on the grid (Eq. 2).
template <typename Real, int V>
__device__ __forceinline__ void demons_force(Real d, Real gsx, Real gsy, Real gsz, Real gmx,
                                             Real gmy, Real gmz, Real b, Real alpha2, Real& dx,
                                             Real& dy, Real& dz) {
    // every a * b + c below is an explicit fused multiply-add (r_fma, r_sq3), so
    // that all kernels round the force identically
    const Real d2 = d * d;
    if (V == 0) {
        term(d, gsx, gsy, gsz, d2 + r_sq3(gsx, gsy, gsz), dx, dy, dz);
    } else if (V == 1) {
        const Real gs2 = r_sq3(gsx, gsy, gsz);
        const Real a = r_sqrt(gs2);
        const Real s = r_fma(b, b, a * a);
        const Real den = r_fma(Real(2), d2, s) * s;
        if (den == Real(0)) {
            dx = dy = dz = Real(0);
        } else {
            const Real c = r_div(Real(4) * d * a * b, den);
            dx = c * gsx;
            dy = c * gsy;
            dz = c * gsz;
        }
    } else if (V == 2 || V == 5) {
        term(d, gmx, gmy, gmz, d2 + r_sq3(gmx, gmy, gmz), dx, dy, dz);
    } else {
        const Real ad2 = (V == 4) ? alpha2 * d2 : d2;
        Real px, py, pz, qx, qy, qz;
        term(d, gsx, gsy, gsz, ad2 + r_sq3(gsx, gsy, gsz), px, py, pz);
        term(d, gmx, gmy, gmz, ad2 + r_sq3(gmx, gmy, gmz), qx, qy, qz);
        dx = px + qx;
        dy = py + qy;
        dz = pz + qz;
    }
}

}  // namespace dirk
