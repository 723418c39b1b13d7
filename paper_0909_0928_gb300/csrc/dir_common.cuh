// dir_common.cuh -- device-side layout and helpers shared by the library's kernels.
//
// Internal volumes are pitched: voxel (i, j, k) of a level lives at
// i + px * j + plane * k with px >= nx a multiple of 32 floats and
// plane = px * ny, so every row starts on a 128-byte boundary.  A field stores
// its three components cs floats apart (cs a multiple of 64).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dirk {

struct Grid3 {
    int nx, ny, nz;   // voxels per axis
    int px;           // row pitch in floats
    long long plane;  // px * ny
    long long cs;     // component stride of a field, floats
};

struct Taps {
    int R;         // radius: 2R+1 taps
    float w[17];   // w[t + R] for t = -R..R
};

constexpr int kMaxRadius = 8;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ long long offs(const Grid3& g, int i, int j, int k) {
    return (long long)i + (long long)g.px * j + g.plane * k;
}

// One axis of the trilinear setup (Sec. 2.5 interpolation, clamped
// coordinates): lower corner floor(p) kept <= n-2 so the upper corner exists.
__device__ __forceinline__ void axis_setup(float p, int n, int& i0, int& i1, float& f) {
    p = fminf(fmaxf(p, 0.0f), (float)(n - 1));
    int lo = (int)floorf(p);
    lo = min(lo, n - 2);
    lo = max(lo, 0);
    i0 = lo;
    i1 = (n > 1) ? lo + 1 : lo;
    f = p - (float)lo;
}

// Software trilinear interpolation of a pitched volume at a continuous voxel
// position (x, y, z); lerps along x, then y, then z.
__device__ __forceinline__ float trilinear(const float* __restrict__ I, const Grid3& g, float x,
                                           float y, float z) {
    int x0, x1, y0, y1, z0, z1;
    float fx, fy, fz;
    axis_setup(x, g.nx, x0, x1, fx);
    axis_setup(y, g.ny, y0, y1, fy);
    axis_setup(z, g.nz, z0, z1, fz);
    const float* p00 = I + (long long)g.px * y0 + g.plane * z0;
    const float* p10 = I + (long long)g.px * y1 + g.plane * z0;
    const float* p01 = I + (long long)g.px * y0 + g.plane * z1;
    const float* p11 = I + (long long)g.px * y1 + g.plane * z1;
    const float c000 = __ldg(p00 + x0), c100 = __ldg(p00 + x1);
    const float c010 = __ldg(p10 + x0), c110 = __ldg(p10 + x1);
    const float c001 = __ldg(p01 + x0), c101 = __ldg(p01 + x1);
    const float c011 = __ldg(p11 + x0), c111 = __ldg(p11 + x1);
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float v00 = c000 * gx + c100 * fx;
    const float v10 = c010 * gx + c110 * fx;
    const float v01 = c001 * gx + c101 * fx;
    const float v11 = c011 * gx + c111 * fx;
    const float v0 = v00 * gy + v10 * fy;
    const float v1 = v01 * gy + v11 * fy;
    return v0 * gz + v1 * fz;
}

// Block-wide sum of three per-thread values in double, then one FP64 atomic
// per value.  Every thread of the block must call it.
template <int NT>
__device__ __forceinline__ void block_reduce3_atomic(float a, float b, float c, double* out) {
    static_assert(NT % 32 == 0, "block size must be whole warps");
    __shared__ double red_s[3][NT / 32];
    double da = a, db = b, dc = c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        da += __shfl_down_sync(0xffffffffu, da, o);
        db += __shfl_down_sync(0xffffffffu, db, o);
        dc += __shfl_down_sync(0xffffffffu, dc, o);
    }
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        red_s[0][warp] = da;
        red_s[1][warp] = db;
        red_s[2][warp] = dc;
    }
    __syncthreads();
    if (warp == 0) {
        da = lane < NT / 32 ? red_s[0][lane] : 0.0;
        db = lane < NT / 32 ? red_s[1][lane] : 0.0;
        dc = lane < NT / 32 ? red_s[2][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            da += __shfl_down_sync(0xffffffffu, da, o);
            db += __shfl_down_sync(0xffffffffu, db, o);
            dc += __shfl_down_sync(0xffffffffu, dc, o);
        }
        if (lane == 0) {
            atomicAdd(out + 0, da);
            atomicAdd(out + 1, db);
            atomicAdd(out + 2, dc);
        }
    }
}

}  // namespace dirk
