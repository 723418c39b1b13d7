// dir_misc.cu -- once-per-level and once-per-registration kernels:
// pyramid decimation and field up-sampling (Sec. 2.3), the final warp
// (Sec. 2.5 interpolation), the inverse-consistent output field (Eq. 6), field
// export, and the relative-norm stop test (Sec. 2.4).
#include <cuda_runtime.h>
#include <math.h>

#include "dir_common.cuh"
#include "dir_launch.h"

namespace dirk {

constexpr int MTX = 32, MTY = 8;

static dim3 grid_for(const Grid3& g) {
    return dim3((g.nx + MTX - 1) / MTX, (g.ny + MTY - 1) / MTY, g.nz);
}

__global__ void decimate_kernel(const float* __restrict__ in, Grid3 gi, float* __restrict__ out,
                                Grid3 go) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= go.nx || y >= go.ny) return;
    out[offs(go, x, y, z)] = __ldg(in + offs(gi, 2 * x, 2 * y, 2 * z));
}

__global__ void upsample_kernel(const float* __restrict__ coarse, Grid3 gc,
                                float* __restrict__ fine, Grid3 gf) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= gf.nx || y >= gf.ny) return;
    const float cx = 0.5f * x, cy = 0.5f * y, cz = 0.5f * z;
    const long long o = offs(gf, x, y, z);
#pragma unroll
    for (int c = 0; c < 3; ++c) fine[o + c * gf.cs] = 2.0f * trilinear(coarse + c * gc.cs, gc, cx, cy, cz);
}

__global__ void warp_kernel(const float* __restrict__ img, const float* __restrict__ u, Grid3 g,
                            float* __restrict__ out) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long o = offs(g, x, y, z);
    const float w = trilinear(img, g, x + __ldg(u + o), y + __ldg(u + o + g.cs),
                              z + __ldg(u + o + 2 * g.cs));
    out[(long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z)] = w;
}

__global__ void ic_invert_kernel(const float* __restrict__ h, float* __restrict__ u, Grid3 g,
                                 int steps) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const float* hx = h;
    const float* hy = h + g.cs;
    const float* hz = h + 2 * g.cs;
    float px = (float)x, py = (float)y, pz = (float)z;
    for (int s = 0; s < steps; ++s) {
        const float ax = trilinear(hx, g, px, py, pz);
        const float ay = trilinear(hy, g, px, py, pz);
        const float az = trilinear(hz, g, px, py, pz);
        px = x + ax;
        py = y + ay;
        pz = z + az;
    }
    const long long o = offs(g, x, y, z);
    u[o] = 2.0f * trilinear(hx, g, px, py, pz);
    u[o + g.cs] = 2.0f * trilinear(hy, g, px, py, pz);
    u[o + 2 * g.cs] = 2.0f * trilinear(hz, g, px, py, pz);
}

__global__ void export_kernel(const float* __restrict__ f, Grid3 g, float sx, float sy, float sz,
                              float* __restrict__ dense) {
    const int x = blockIdx.x * MTX + threadIdx.x, y = blockIdx.y * MTY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long o = offs(g, x, y, z);
    const long long d = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
    dense[d] = sx * f[o];
    dense[d + n] = sy * f[o + g.cs];
    dense[d + 2 * n] = sz * f[o + 2 * g.cs];
}

// Sec. 2.4: l(t) = sum|du| / sum|u|; stop the level after iteration t when
// |l(t) - l(t - window)| <= eps (both defined).  One thread.
__global__ void stop_test_kernel(const double* __restrict__ red, double* lhist, int t,
                                 int level_first, int window, double eps, int* stop_iter,
                                 int iter_in_level) {
    if (*stop_iter < iter_in_level) return;
    const double B = red[3 * t + 2];
    const double l = B > 0.0 ? red[3 * t + 1] / B : nan("");
    lhist[t] = l;
    if (iter_in_level >= window && t - window >= level_first) {
        const double lp = lhist[t - window];
        if (!isnan(l) && !isnan(lp) && fabs(l - lp) <= eps) *stop_iter = iter_in_level;
    }
}

cudaError_t launch_decimate(const float* in, const Grid3& gin, float* out, const Grid3& gout,
                            cudaStream_t s) {
    decimate_kernel<<<grid_for(gout), dim3(MTX, MTY), 0, s>>>(in, gin, out, gout);
    return cudaGetLastError();
}

cudaError_t launch_upsample(const float* coarse, const Grid3& gc, float* fine, const Grid3& gf,
                            cudaStream_t s) {
    upsample_kernel<<<grid_for(gf), dim3(MTX, MTY), 0, s>>>(coarse, gc, fine, gf);
    return cudaGetLastError();
}

cudaError_t launch_warp(const float* img, const float* u, const Grid3& g, float* out_dense,
                        cudaStream_t s) {
    warp_kernel<<<grid_for(g), dim3(MTX, MTY), 0, s>>>(img, u, g, out_dense);
    return cudaGetLastError();
}

cudaError_t launch_ic_invert(const float* h, float* u, const Grid3& g, int steps, cudaStream_t s) {
    ic_invert_kernel<<<grid_for(g), dim3(MTX, MTY), 0, s>>>(h, u, g, steps);
    return cudaGetLastError();
}

cudaError_t launch_export_field(const float* field, const Grid3& g, float sx, float sy, float sz,
                                float* dense, cudaStream_t s) {
    export_kernel<<<grid_for(g), dim3(MTX, MTY), 0, s>>>(field, g, sx, sy, sz, dense);
    return cudaGetLastError();
}

cudaError_t launch_stop_test(const double* red, double* lhist, int t, int level_first, int window,
                             double eps, int* stop_iter, int iter_in_level, cudaStream_t s) {
    stop_test_kernel<<<1, 1, 0, s>>>(red, lhist, t, level_first, window, eps, stop_iter,
                                     iter_in_level);
    return cudaGetLastError();
}

}  // namespace dirk
