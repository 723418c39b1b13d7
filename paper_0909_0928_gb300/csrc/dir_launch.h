// dir_launch.h -- host-side launchers of the library's kernels (internal).
// Each returns the cudaError_t of its launch.
#pragma once

#include <cuda_runtime.h>

#include "dir_common.cuh"

namespace dirk {

// Force + update + reductions of one demons iteration at one level
// (Sec. 2.5 interpolation, gradient and displacement kernels fused):
//   v = u - dr(u),  red[0..2] += {sum d^2, sum |du|, sum |u|}.
// Skips all work when *stop_iter < iter (device-side stop test).
struct ForceArgs {
    const float* S;      // static image of the level (pitched)
    const float* M;      // moving image of the level (pitched)
    const float* u;      // field in (3 components)
    float* v;            // field out, u + du
    Grid3 g;
    int zchunk;          // planes per block
    float alpha2;        // alpha^2 for Eq. (5)
    double* red;         // 3 doubles, accumulated with atomics
    const int* stop_iter;
    int iter;
};
cudaError_t launch_force(int variant, const ForceArgs& a, cudaStream_t s);
int force_zchunk(int variant, const Grid3& g, int num_sms);

// Separable Gaussian (Sec. 2.5 low-pass filter), x then y then z, replicate
// edges, ncomp components cs apart.  Skips when *stop_iter < iter.
struct SmoothArgs {
    const float* in;
    float* out;
    Grid3 g;
    int ncomp;           // 1 or 3
    int zchunk;
    Taps taps;
    const int* stop_iter;
    int iter;
};
cudaError_t launch_smooth(const SmoothArgs& a, cudaStream_t s);
int smooth_zchunk(const Grid3& g, int radius, int num_sms);

// out(i, j, k) = in(2i, 2j, 2k)   (pyramid decimation, Sec. 2.3)
cudaError_t launch_decimate(const float* in, const Grid3& gin, float* out, const Grid3& gout,
                            cudaStream_t s);
// fine(x) = 2 * trilinear(coarse, x / 2), per component (Sec. 2.3)
cudaError_t launch_upsample(const float* coarse, const Grid3& gc, float* fine, const Grid3& gf,
                            cudaStream_t s);
// out(x) = img(x + u(x)); out written dense (x-contiguous, no pitch)
cudaError_t launch_warp(const float* img, const float* u, const Grid3& g, float* out_dense,
                        cudaStream_t s);
// u(y) = 2 h(x*), x* = y + h(x*) by `steps` fixed-point steps (Eq. 6 output)
cudaError_t launch_ic_invert(const float* h, float* u, const Grid3& g, int steps, cudaStream_t s);
// dense[c*N + i + nx*(j + ny*k)] = scale[c] * field[c*cs + pitched(i,j,k)]
cudaError_t launch_export_field(const float* field, const Grid3& g, float sx, float sy, float sz,
                                float* dense, cudaStream_t s);
// relative-norm stop test of Sec. 2.4 for iteration t of a level
cudaError_t launch_stop_test(const double* red, double* lhist, int t, int level_first, int window,
                             double eps, int* stop_iter, int iter_in_level, cudaStream_t s);

}  // namespace dirk
