// dir_smooth.cu -- separable 3-D Gaussian low-pass filter (Sec. 2.5).
//
// out = G_sigma * in, applied along x, then y, then z, with replicated edges,
// on 1 or 3 components.  The paper stages data in shared memory so that the
// strided y and z passes stay coalesced; here a block owns a 32 x 8 column tile
// and marches through a chunk of z planes: each input plane (tile plus an R
// halo in x and y) is staged in shared memory, the x and y passes run there,
// and the z pass is a rolling window of 2R+1 y-filtered planes held in
// registers, so every input voxel is read from HBM about once.
#include <cuda_runtime.h>

#include "dir_common.cuh"
#include "dir_launch.h"

namespace dirk {

constexpr int STX = 32, STY = 8, SNT = STX * STY;

template <int R, int NC>
__global__ void __launch_bounds__(SNT) smooth_kernel(const SmoothArgs a) {
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    constexpr int W = STX + 2 * R, H = STY + 2 * R, K = 2 * R + 1;
    __shared__ float tin[NC][H][W];
    __shared__ float txp[NC][H][STX];
    const Grid3 g = a.g;
    const float* __restrict__ in = a.in;
    float* __restrict__ out = a.out;
    float w[K];
#pragma unroll
    for (int t = 0; t < K; ++t) w[t] = a.taps.w[t];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + STX * ty;
    const int x0 = blockIdx.x * STX, y0 = blockIdx.y * STY;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = (x < g.nx) && (y < g.ny);
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nz);

    float ring[K][NC];
#pragma unroll
    for (int t = 0; t < K; ++t)
#pragma unroll
        for (int c = 0; c < NC; ++c) ring[t][c] = 0.0f;

    for (int p = z0 - R; p < z1 + R; ++p) {
        const int pc = clampi(p, 0, g.nz - 1);
        for (int q = tid; q < W * H; q += SNT) {
            const int hy = q / W, hx = q - hy * W;
            const int gx = clampi(x0 + hx - R, 0, g.nx - 1);
            const int gy = clampi(y0 + hy - R, 0, g.ny - 1);
            const long long o = offs(g, gx, gy, pc);
#pragma unroll
            for (int c = 0; c < NC; ++c) tin[c][hy][hx] = __ldg(in + o + c * g.cs);
        }
        __syncthreads();
        for (int q = tid; q < STX * H; q += SNT) {
            const int r = q / STX, cc = q - r * STX;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float acc = 0.0f;
#pragma unroll
                for (int t = 0; t < K; ++t) acc += w[t] * tin[c][r][cc + t];
                txp[c][r][cc] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < K - 1; ++t)
#pragma unroll
            for (int c = 0; c < NC; ++c) ring[t][c] = ring[t + 1][c];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            float acc = 0.0f;
#pragma unroll
            for (int t = 0; t < K; ++t) acc += w[t] * txp[c][ty + t][tx];
            ring[K - 1][c] = acc;
        }
        if (p >= z0 + R && valid) {
            const long long o = offs(g, x, y, p - R);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float acc = 0.0f;
#pragma unroll
                for (int t = 0; t < K; ++t) acc += w[t] * ring[t][c];
                out[o + c * g.cs] = acc;
            }
        }
    }
}

int smooth_zchunk(const Grid3& g, int radius, int num_sms) {
    const long long bxy = (long long)((g.nx + STX - 1) / STX) * ((g.ny + STY - 1) / STY);
    const long long target = 4LL * num_sms;
    long long chunks = (target + bxy - 1) / bxy;
    if (chunks < 1) chunks = 1;
    int zc = (int)((g.nz + chunks - 1) / chunks);
    const int zmin = 4 * radius;  // keep the 2R-plane halo small against the chunk
    if (zc < zmin) zc = zmin;
    if (zc > g.nz) zc = g.nz;
    return zc < 1 ? 1 : zc;
}

template <int R>
static cudaError_t launch_r(const SmoothArgs& a, dim3 grid, dim3 block, cudaStream_t s) {
    if (a.ncomp == 3)
        smooth_kernel<R, 3><<<grid, block, 0, s>>>(a);
    else
        smooth_kernel<R, 1><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_smooth(const SmoothArgs& a, cudaStream_t s) {
    if (a.ncomp != 1 && a.ncomp != 3) return cudaErrorInvalidValue;
    const dim3 block(STX, STY, 1);
    const dim3 grid((a.g.nx + STX - 1) / STX, (a.g.ny + STY - 1) / STY,
                    (a.g.nz + a.zchunk - 1) / a.zchunk);
    switch (a.taps.R) {
        case 1: return launch_r<1>(a, grid, block, s);
        case 2: return launch_r<2>(a, grid, block, s);
        case 3: return launch_r<3>(a, grid, block, s);
        case 4: return launch_r<4>(a, grid, block, s);
        case 5: return launch_r<5>(a, grid, block, s);
        case 6: return launch_r<6>(a, grid, block, s);
        case 7: return launch_r<7>(a, grid, block, s);
        case 8: return launch_r<8>(a, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dirk
