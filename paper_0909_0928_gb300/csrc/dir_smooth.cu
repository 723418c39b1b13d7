// dir_smooth.cu -- separable 3-D Gaussian low-pass filter (Sec. 2.5).
//
// out = G_sigma * in, applied along x, then y, then z, with replicated edges,
// on 1 or 3 components: the TMA-fed plane pipeline of dir_stencil.cuh.  A
// block smooths one component of a 32 x 8 column tile over a z chunk, one
// thread per (column, 4-row group) for the y and z passes, so the three
// components run as independent blocks (three times the marching chains per
// SM).  Every input voxel is read from HBM about once per launch (plus the
// 2R-plane halo of each z chunk).
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_common.cuh"
#include "dir_launch.h"
#include "dir_stencil.cuh"

namespace dirk {

template <typename Real, int R, typename TIN, typename TOUT>
__global__ void __launch_bounds__(StencilGeom<Real, R, 1, 8, TIN>::YT)
    smooth_kernel(const __grid_constant__ CUtensorMap tmap, const SmoothArgs a, int zchunk) {
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    constexpr int NC = 1;
    using G = StencilGeom<Real, R, NC, 8, TIN>;
    constexpr int K = G::K, NT = G::YT;
    extern __shared__ unsigned char smem_raw[];
    const Grid3 g = a.g;
    TOUT* __restrict__ out = static_cast<TOUT*>(a.out);
    Real w[K];
#pragma unroll
    for (int t = 0; t < K; ++t) w[t] = tap<Real>(a.taps, t);

    const int tid = threadIdx.x;
    const int lx = tid % STX;          // y/z role: column, row group
    const int q_own = tid / STX;
    const int comp = blockIdx.z % a.ncomp;
    const int x0 = blockIdx.x * STX, y0 = blockIdx.y * STY;
    const int x = x0 + lx;
    const int z0 = (blockIdx.z / a.ncomp) * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    out += (long long)comp * g.cs;

    PlanePipe<Real, R, NC, 8, TIN> pipe;
    pipe.setup(smem_raw, g, x0, y0, z0, z1, comp);
    pipe.start(&tmap, g, tid);

    Real ring[K][YW];
#pragma unroll
    for (int t = 0; t < K; ++t)
#pragma unroll
        for (int r = 0; r < YW; ++r) ring[t][r] = Real(0);

    for (int step = 0; step < pipe.nsteps; ++step) {
        if (!pipe.template xpass<NT>(&tmap, g, step, tid, w, a.err)) return;
        pipe.ypass(0, q_own, lx, w, ring);
        if (step >= 2 * R && x < g.nx) {
            const int zo = z0 + step - 2 * R;
#pragma unroll
            for (int r = 0; r < YW; ++r) {
                const int y = y0 + q_own * YW + r;
                if (y < g.ny) out[offs(g, x, y, zo)] = st_as<TOUT>(zpass<Real, R>(w, ring, r));
            }
        }
        // no barrier here: the next step's __syncthreads_or orders these reads
        // of the x-pass rows before they are rewritten
    }
}

template <typename Real, int R, typename TIN, typename TOUT>
static cudaError_t launch_rt(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    using G = StencilGeom<Real, R, 1, 8, TIN>;
    CUtensorMap map;
    if (!make_plane_map<Real, R, 1, TIN>(&map, a.in, a.g, a.ncomp)) return cudaErrorInvalidValue;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(smooth_kernel<Real, R, TIN, TOUT>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   G::BASE_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smooth_kernel<Real, R, TIN, TOUT>,
                                                  G::YT, G::BASE_SMEM);
    int zc = a.zchunk > 0 ? a.zchunk : stencil_zchunk(a.g, per_sm, num_sms, a.ncomp);
    if (zc > a.g.nz) zc = a.g.nz;
    const int chunks = (a.g.nz + zc - 1) / zc;
    const dim3 grid((a.g.nx + STX - 1) / STX, (a.g.ny + STY - 1) / STY, chunks * a.ncomp);
    smooth_kernel<Real, R, TIN, TOUT><<<grid, dim3(G::YT, 1, 1), G::BASE_SMEM, s>>>(map, a, zc);
    return cudaGetLastError();
}

template <typename Real, typename TIN, typename TOUT>
static cudaError_t launch_types(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    switch (a.taps.R) {
        case 1: return launch_rt<Real, 1, TIN, TOUT>(a, num_sms, s);
        case 2: return launch_rt<Real, 2, TIN, TOUT>(a, num_sms, s);
        case 3: return launch_rt<Real, 3, TIN, TOUT>(a, num_sms, s);
        case 4: return launch_rt<Real, 4, TIN, TOUT>(a, num_sms, s);
        case 5: return launch_rt<Real, 5, TIN, TOUT>(a, num_sms, s);
        case 6: return launch_rt<Real, 6, TIN, TOUT>(a, num_sms, s);
        case 7: return launch_rt<Real, 7, TIN, TOUT>(a, num_sms, s);
        case 8: return launch_rt<Real, 8, TIN, TOUT>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_smooth(bool fp64, const SmoothArgs& a, int num_sms, cudaStream_t s) {
    if (a.ncomp != 1 && a.ncomp != 3) return cudaErrorInvalidValue;
    if (fp64) {
        if (a.in_type != kStoreF64 || a.out_type != kStoreF64) return cudaErrorInvalidValue;
        return launch_types<double, double, double>(a, num_sms, s);
    }
    if (a.in_type == kStoreF32 && a.out_type == kStoreF32)
        return launch_types<float, float, float>(a, num_sms, s);
    if (a.in_type == kStoreI16 && a.out_type == kStoreF32)
        return launch_types<float, int16_t, float>(a, num_sms, s);
    if (a.in_type == kStoreBF16 && a.out_type == kStoreBF16)
        return launch_types<float, bf16, bf16>(a, num_sms, s);
    return cudaErrorInvalidValue;
}

}  // namespace dirk
