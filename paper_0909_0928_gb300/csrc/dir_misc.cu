// dir_misc.cu -- once-per-level and once-per-registration kernels:
// pyramid decimation and field up-sampling (Sec. 2.3), the final warp
// (Sec. 2.5 interpolation), the inverse-consistent output field (Eq. 6), field
// import/export, and the relative-norm stop test (Sec. 2.4).
#include <cuda_runtime.h>
#include <math.h>

#include "dir_common.cuh"
#include "dir_launch.h"

namespace dirk {

constexpr int MTX = 32, MTY = 8;

static dim3 grid_for(const Grid3& g) {
    return dim3((g.nx + MTX - 1) / MTX, (g.ny + MTY - 1) / MTY, g.nz);
}

template <typename Real>
__global__ void decimate_kernel(const Real* __restrict__ in, Grid3 gi, Real* __restrict__ out,
                                Grid3 go) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= go.nx || y >= go.ny) return;
    out[offs(go, x, y, z)] = __ldg(in + offs(gi, 2 * x, 2 * y, 2 * z));
}

template <typename Real, typename TF>
__global__ void upsample_kernel(const TF* __restrict__ coarse, Grid3 gc, TF* __restrict__ fine,
                                Grid3 gf) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= gf.nx || y >= gf.ny) return;
    // coarse position x / 2 = (x >> 1) + (x & 1) / 2, exact
    const Real hx = Real(0.5) * (x & 1), hy = Real(0.5) * (y & 1), hz = Real(0.5) * (z & 1);
    const long long o = (long long)offs(gf, x, y, z);
#pragma unroll
    for (int c = 0; c < 3; ++c)
        fine[o + c * gf.cs] = st_as<TF>(
            Real(2) * trilinear<Real>(coarse + c * gc.cs, gc, x >> 1, hx, y >> 1, hy, z >> 1, hz));
}

template <typename Real, typename TF>
__global__ void warp_kernel(const Real* __restrict__ img, const TF* __restrict__ u, Grid3 g,
                            float* __restrict__ out) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long o = (long long)offs(g, x, y, z);
    const Real w = trilinear<Real>(img, g, x, ldg_as<Real>(u + o), y, ldg_as<Real>(u + o + g.cs),
                                   z, ldg_as<Real>(u + o + 2 * g.cs));
    out[(long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z)] = (float)w;
}

template <typename Real, typename TF>
__global__ void ic_invert_kernel(const TF* __restrict__ h, TF* __restrict__ u, Grid3 g,
                                 int steps) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const TF* hx = h;
    const TF* hy = h + g.cs;
    const TF* hz = h + 2 * g.cs;
    // x* = y + a with a = h(x*), iterated from a = 0; once a step returns its
    // input exactly, every later step would too, so the loop may stop there
    Real ax = 0, ay = 0, az = 0;
    for (int s = 0; s < steps; ++s) {
        const Real nx_ = trilinear<Real>(hx, g, x, ax, y, ay, z, az);
        const Real ny_ = trilinear<Real>(hy, g, x, ax, y, ay, z, az);
        const Real nz_ = trilinear<Real>(hz, g, x, ax, y, ay, z, az);
        const bool fixed = (nx_ == ax) && (ny_ == ay) && (nz_ == az);
        ax = nx_;
        ay = ny_;
        az = nz_;
        if (fixed) break;
    }
    const long long o = (long long)offs(g, x, y, z);
    u[o] = st_as<TF>(Real(2) * trilinear<Real>(hx, g, x, ax, y, ay, z, az));
    u[o + g.cs] = st_as<TF>(Real(2) * trilinear<Real>(hy, g, x, ax, y, ay, z, az));
    u[o + 2 * g.cs] = st_as<TF>(Real(2) * trilinear<Real>(hz, g, x, ax, y, ay, z, az));
}

template <typename Real, typename TF, typename Out>
__global__ void export_kernel(const TF* __restrict__ f, Grid3 g, double sx, double sy, double sz,
                              Out* __restrict__ dense) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long o = (long long)offs(g, x, y, z);
    const long long d = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
    dense[d] = (Out)((Real)sx * ld_as<Real>(f + o));
    dense[d + n] = (Out)((Real)sy * ld_as<Real>(f + o + g.cs));
    dense[d + 2 * n] = (Out)((Real)sz * ld_as<Real>(f + o + 2 * g.cs));
}

template <typename Real, typename TF>
__global__ void import_kernel(const float* __restrict__ dense, TF* __restrict__ f, Grid3 g,
                              int ncomp) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long o = (long long)offs(g, x, y, z);
    const long long d = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
    for (int c = 0; c < ncomp; ++c) f[o + c * g.cs] = st_as<TF>((Real)dense[d + c * n]);
}

// Sec. 2.4: l(t) = sum|du| / sum|u|; stop the level after iteration t when
// |l(t) - l(t - window)| <= eps (both defined).  One thread.
__global__ void stop_test_kernel(const double* __restrict__ red, const double* __restrict__ corr,
                                 double n, double* lhist, int t, int level_first, int window,
                                 double eps, int* stop_iter, int iter_in_level) {
    if (*stop_iter < iter_in_level) return;
    const double B = red[3 * t + 2];
    const double l = corr ? correlation_from_sums(red[3 * t], corr + 4 * t, n)
                          : (B > 0.0 ? red[3 * t + 1] / B : nan(""));
    lhist[t] = l;
    if (iter_in_level >= window && t - window >= level_first) {
        const double lp = lhist[t - window];
        if (!isnan(l) && !isnan(lp) && fabs(l - lp) <= eps) *stop_iter = iter_in_level;
    }
}

// Dispatch on (arithmetic, field storage): double/double, float/float,
// float/bf16.  `CALL` sees the types as Real and TF.
#define DIR_DISPATCH_F(fp64, ftype, CALL)                      \
    do {                                                       \
        if (fp64) {                                            \
            if (ftype != kStoreF64) return cudaErrorInvalidValue; \
            using Real = double;                               \
            using TF = double;                                 \
            CALL;                                              \
        } else if (ftype == kStoreBF16) {                      \
            using Real = float;                                \
            using TF = bf16;                                   \
            CALL;                                              \
        } else if (ftype == kStoreF32) {                       \
            using Real = float;                                \
            using TF = float;                                  \
            CALL;                                              \
        } else {                                               \
            return cudaErrorInvalidValue;                      \
        }                                                      \
    } while (0)

cudaError_t launch_decimate(bool fp64, const void* in, const Grid3& gin, void* out,
                            const Grid3& gout, cudaStream_t s) {
    if (fp64)
        decimate_kernel<double><<<grid_for(gout), dim3(MTX, MTY), 0, s>>>(
            static_cast<const double*>(in), gin, static_cast<double*>(out), gout);
    else
        decimate_kernel<float><<<grid_for(gout), dim3(MTX, MTY), 0, s>>>(
            static_cast<const float*>(in), gin, static_cast<float*>(out), gout);
    return cudaGetLastError();
}

cudaError_t launch_upsample(bool fp64, int ftype, const void* coarse, const Grid3& gc, void* fine,
                            const Grid3& gf, cudaStream_t s) {
    DIR_DISPATCH_F(fp64, ftype, (upsample_kernel<Real, TF><<<grid_for(gf), dim3(MTX, MTY), 0, s>>>(
                                    static_cast<const TF*>(coarse), gc, static_cast<TF*>(fine), gf)));
    return cudaGetLastError();
}

cudaError_t launch_warp(bool fp64, int ftype, const void* img, const void* u, const Grid3& g,
                        float* out_dense, cudaStream_t s) {
    DIR_DISPATCH_F(fp64, ftype, (warp_kernel<Real, TF><<<grid_for(g), dim3(MTX, MTY), 0, s>>>(
                                    static_cast<const Real*>(img), static_cast<const TF*>(u), g,
                                    out_dense)));
    return cudaGetLastError();
}

cudaError_t launch_ic_invert(bool fp64, int ftype, const void* h, void* u, const Grid3& g,
                             int steps, cudaStream_t s) {
    DIR_DISPATCH_F(fp64, ftype, (ic_invert_kernel<Real, TF><<<grid_for(g), dim3(MTX, MTY), 0, s>>>(
                                    static_cast<const TF*>(h), static_cast<TF*>(u), g, steps)));
    return cudaGetLastError();
}

cudaError_t launch_export_field(bool fp64, int ftype, const void* field, const Grid3& g, double sx,
                                double sy, double sz, void* dense, bool out_fp64, cudaStream_t s) {
    if (out_fp64) {
        DIR_DISPATCH_F(fp64, ftype,
                       (export_kernel<Real, TF, double><<<grid_for(g), dim3(MTX, MTY), 0, s>>>(
                           static_cast<const TF*>(field), g, sx, sy, sz,
                           static_cast<double*>(dense))));
    } else {
        DIR_DISPATCH_F(fp64, ftype,
                       (export_kernel<Real, TF, float><<<grid_for(g), dim3(MTX, MTY), 0, s>>>(
                           static_cast<const TF*>(field), g, sx, sy, sz,
                           static_cast<float*>(dense))));
    }
    return cudaGetLastError();
}

cudaError_t launch_import(bool fp64, int out_type, const float* dense, void* pitched,
                          const Grid3& g, int ncomp, cudaStream_t s) {
    DIR_DISPATCH_F(fp64, out_type, (import_kernel<Real, TF><<<grid_for(g), dim3(MTX, MTY), 0, s>>>(
                                       dense, static_cast<TF*>(pitched), g, ncomp)));
    return cudaGetLastError();
}

// One thread waits, bounded, on an mbarrier that nothing arrives on (the
// failure path of the TMA waits), then records that it gave up.
__global__ void wait_probe_kernel(int* err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(err, kErrTmaTimeout);
}

cudaError_t launch_wait_probe(int* err, unsigned long long limit_ns, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(err, limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_stop_test(const double* red, const double* corr, double n, double* lhist,
                             int t, int level_first, int window, double eps, int* stop_iter,
                             int iter_in_level, cudaStream_t s) {
    stop_test_kernel<<<1, 1, 0, s>>>(red, corr, n, lhist, t, level_first, window, eps, stop_iter,
                                     iter_in_level);
    return cudaGetLastError();
}

}  // namespace dirk
