// dir_fused.cu -- one demons iteration in one pass, for the force laws that
// need no gradient of the warped image (Eq. 1 passive, Eq. 2 evolved passive).
//
// Iteration k keeps v_k = u_k + du_k in memory instead of u_k: the kernel reads
// v_{k-1}, smooths it on the fly into u_k = G_sigma * v_{k-1} (Sec. 2.1: the
// total field is smoothed), then warps M by u_k, applies the force and writes
// v_k, with the reductions of Sec. 2.4 on the way.  The first iteration of a
// level (u_0 given) uses the plain force kernel and the last v is smoothed
// once more by the smoothing kernel, so the arithmetic and its order are those
// of the two-kernel schedule while each iteration moves about 32 bytes per
// voxel instead of 56.
//
// Layout: the TMA plane pipeline of dir_stencil.cuh smooths the three field
// components of a 32 x 8 column tile plane by plane; the smoothed plane goes
// through shared memory to the 256 force threads (one voxel each), which
// gather M through L1/L2 and keep a rolling z window of S (and M for Eq. 2).
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_common.cuh"
#include "dir_force_law.cuh"
#include "dir_launch.h"
#include "dir_stencil.cuh"

namespace dirk {

constexpr int FUSED_NT = STX * STY;  // 256: one force voxel per thread and plane

template <typename Real, int R>
struct FusedGeom {
    using G = StencilGeom<Real, R, 3>;
    static constexpr int UTILE_BYTES = 3 * STY * STX * (int)sizeof(Real);
    static constexpr int SMEM = G::BASE_SMEM + UTILE_BYTES;
};

template <typename Real, int R, int V>
__global__ void __launch_bounds__(FUSED_NT, R <= 4 ? 2 : 1)
    fused_kernel(const __grid_constant__ CUtensorMap tmap, const FusedArgs a, int zchunk) {
    static_assert(V == 0 || V == 1, "fused iteration needs no warped-image gradient");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    using G = StencilGeom<Real, R, 3>;
    constexpr int K = G::K;
    extern __shared__ unsigned char smem_raw[];
    const Grid3 g = a.g;
    const Real* __restrict__ S = static_cast<const Real*>(a.S);
    const Real* __restrict__ M = static_cast<const Real*>(a.M);
    Real* __restrict__ vout = static_cast<Real*>(a.v);
    Real w[K];
#pragma unroll
    for (int t = 0; t < K; ++t) w[t] = tap<Real>(a.taps, t);

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * STX, y0 = blockIdx.y * STY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    // smoothing role (first G::YT threads): column, component, row group
    const bool smoother = tid < G::YT;
    const int lx = tid % STX;
    const int c_own = (tid / STX) % 3;
    const int q_own = (tid / STX) / 3;
    // force role (all threads): one voxel of the tile
    const int fx = tid % STX, fy = tid / STX;
    const int x = x0 + fx, y = y0 + fy;
    const bool valid = (x < g.nx) && (y < g.ny);
    const int xc = min(x, g.nx - 1), yc = min(y, g.ny - 1);
    const int xm = max(xc - 1, 0), xp = min(xc + 1, g.nx - 1);
    const int ym = max(yc - 1, 0), yp = min(yc + 1, g.ny - 1);

    PlanePipe<Real, R, 3> pipe;
    pipe.setup(smem_raw, g, x0, y0, z0, z1);
    Real* utile = reinterpret_cast<Real*>(pipe.extra());  // [3][STY][STX]
    pipe.start(&tmap, g, tid);

    Real ring[K][YW];
#pragma unroll
    for (int t = 0; t < K; ++t)
#pragma unroll
        for (int r = 0; r < YW; ++r) ring[t][r] = Real(0);

    // rolling z windows of S (and M for Eq. 2) at this thread's force voxel
    Real s_m1 = __ldg(S + offs(g, xc, yc, max(z0 - 1, 0)));
    Real s_0 = __ldg(S + offs(g, xc, yc, z0));
    Real m_m1 = 0, m_0 = 0;
    if (V == 1) {
        m_m1 = __ldg(M + offs(g, xc, yc, max(z0 - 1, 0)));
        m_0 = __ldg(M + offs(g, xc, yc, z0));
    }
    Real sd2 = 0, sdu = 0, su = 0;  // per-thread partial sums

    for (int step = 0; step < pipe.nsteps; ++step) {
        if (!pipe.template xpass<FUSED_NT>(&tmap, g, step, tid, w, a.err)) {
            return;
        }
        const bool out_plane = step >= 2 * R;
        if (smoother) {
            pipe.ypass(c_own, q_own, lx, w, ring);
            if (out_plane) {
#pragma unroll
                for (int r = 0; r < YW; ++r)
                    utile[(c_own * STY + q_own * YW + r) * STX + lx] = zpass<Real, R>(w, ring, r);
            }
        }
        __syncthreads();
        if (out_plane) {
            const int zo = z0 + step - 2 * R;
            const int zn = min(zo + 1, g.nz - 1);
            const Real s_p1 = __ldg(S + offs(g, xc, yc, zn));
            Real m_p1 = 0;
            if (V == 1) m_p1 = __ldg(M + offs(g, xc, yc, zn));
            if (valid) {
                const int o = offs(g, x, y, zo);
                const Real ux = utile[(0 * STY + fy) * STX + fx];
                const Real uy = utile[(1 * STY + fy) * STX + fx];
                const Real uz = utile[(2 * STY + fy) * STX + fx];
                const Real d = trilinear(M, g, x, ux, y, uy, zo, uz, s_0);  // W - S
                const int ro = offs(g, 0, y, zo);
                const Real gsx = Real(0.5) * (__ldg(S + ro + xp) - __ldg(S + ro + xm));
                const Real gsy =
                    Real(0.5) * (__ldg(S + offs(g, x, yp, zo)) - __ldg(S + offs(g, x, ym, zo)));
                const Real gsz = Real(0.5) * (s_p1 - s_m1);
                Real bm = 0;
                if (V == 1) {
                    const Real mx = Real(0.5) * (__ldg(M + ro + xp) - __ldg(M + ro + xm));
                    const Real my = Real(0.5) *
                                    (__ldg(M + offs(g, x, yp, zo)) - __ldg(M + offs(g, x, ym, zo)));
                    const Real mz = Real(0.5) * (m_p1 - m_m1);
                    bm = r_sqrt(mx * mx + my * my + mz * mz);
                }
                Real dx, dy, dz;
                demons_force<Real, V>(d, gsx, gsy, gsz, Real(0), Real(0), Real(0), bm, Real(0), dx,
                                      dy, dz);
                dx = -dx;
                dy = -dy;
                dz = -dz;
                sd2 += d * d;
                sdu += r_norm_fast(dx * dx + dy * dy + dz * dz);
                su += r_norm_fast(ux * ux + uy * uy + uz * uz);
                vout[o] = ux + dx;
                vout[o + (int)g.cs] = uy + dy;
                vout[o + 2 * (int)g.cs] = uz + dz;
            }
            s_m1 = s_0;
            s_0 = s_p1;
            if (V == 1) {
                m_m1 = m_0;
                m_0 = m_p1;
            }
        }
    }
    block_reduce3_atomic<FUSED_NT, Real>(sd2, sdu, su, a.red);
}

template <typename Real, int R, int V>
static cudaError_t launch_rv(const FusedArgs& a, int num_sms, cudaStream_t s) {
    using F = FusedGeom<Real, R>;
    CUtensorMap map;
    if (!make_plane_map<Real, R, 3>(&map, a.vin, a.g, 3)) return cudaErrorInvalidValue;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(
            fused_kernel<Real, R, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, F::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel<Real, R, V>, FUSED_NT,
                                                  F::SMEM);
    const int zc = stencil_zchunk(a.g, per_sm, num_sms);
    const dim3 grid((a.g.nx + STX - 1) / STX, (a.g.ny + STY - 1) / STY, (a.g.nz + zc - 1) / zc);
    fused_kernel<Real, R, V><<<grid, dim3(FUSED_NT, 1, 1), F::SMEM, s>>>(map, a, zc);
    return cudaGetLastError();
}

template <typename Real, int R>
static cudaError_t launch_r(int variant, const FusedArgs& a, int num_sms, cudaStream_t s) {
    return variant == 1 ? launch_rv<Real, R, 1>(a, num_sms, s) : launch_rv<Real, R, 0>(a, num_sms, s);
}

template <typename Real>
static cudaError_t launch_t(int variant, const FusedArgs& a, int num_sms, cudaStream_t s) {
    switch (a.taps.R) {
        case 1: return launch_r<Real, 1>(variant, a, num_sms, s);
        case 2: return launch_r<Real, 2>(variant, a, num_sms, s);
        case 3: return launch_r<Real, 3>(variant, a, num_sms, s);
        case 4: return launch_r<Real, 4>(variant, a, num_sms, s);
        case 5: return launch_r<Real, 5>(variant, a, num_sms, s);
        case 6: return launch_r<Real, 6>(variant, a, num_sms, s);
        case 7: return launch_r<Real, 7>(variant, a, num_sms, s);
        case 8: return launch_r<Real, 8>(variant, a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

bool fused_supported(int variant) { return variant == 0 || variant == 1; }

cudaError_t launch_fused(int variant, bool fp64, const FusedArgs& a, int num_sms, cudaStream_t s) {
    if (!fused_supported(variant)) return cudaErrorInvalidValue;
    return fp64 ? launch_t<double>(variant, a, num_sms, s) : launch_t<float>(variant, a, num_sms, s);
}

}  // namespace dirk
