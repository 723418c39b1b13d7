// dir_launch.h -- host-side launchers of the library's kernels (internal).
// Pointers are untyped: `fp64` selects the element type (double) or float.
// Each launcher returns the cudaError_t of its launch.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>

#include "dir_common.cuh"

namespace dirk {

// storage types of images and fields on the device
constexpr int kStoreF32 = 0, kStoreI16 = 1, kStoreBF16 = 3, kStoreF64 = 4;

// Force + update + reductions of one demons iteration at one level
// (Sec. 2.5 interpolation, gradient and displacement kernels fused):
//   v = u - dr(u),  red[0..2] += {sum d^2, sum |du|, sum |u|}.
// Skips all work when *stop_iter < iter (device-side stop test).
struct ForceArgs {
    const void* S;       // static image of the level (pitched)
    const void* M;       // moving image of the level (pitched)
    const void* u;       // field in (3 components)
    void* v;             // field out, u + du
    Grid3 g;
    double alpha2;       // alpha^2 for Eq. (5)
    double* red;         // 3 doubles, accumulated with atomics
    const int* stop_iter;
    int iter;
    int depth;           // voxels per thread along z: 1, 2, 4 or 8
    int img_type;        // storage of S and M at this level (kStore*)
    int field_type;      // storage of u and v (kStore*)
    int pf_stride = 0;   // > 0: each block prefetches into L2 the brick of the block
                         // this many linear indices ahead
    int* err = nullptr;  // device error word (kErr* bits) for bounded waits
    double* corr = nullptr;  // non-null: += {Sum b, Sum b^2, Sum d, Sum b d} of the
                             // correlation of the warped image with its reference
    bool pdl = false;        // launch as a programmatic dependent launch (split
                             // kernels only; only without a stop test: they read the
                             // stop flag before waiting for the kernel before)
    void* dbuf = nullptr;    // Eqs. 3-6 split with the difference image: D = W - S
                             // (Eq. 6: D_m + D_s), one float per voxel, pitched as a
                             // field component
    void* dbuf2 = nullptr;   // Eq. 6 only: d = D_m - D_s, likewise
};
// plain = true: the plain-load force_kernel even where a TMA-fed kernel exists
// (the same per-voxel arithmetic without the tiling; a cross-check of it)
cudaError_t launch_force(int variant, bool fp64, const ForceArgs& a, cudaStream_t s,
                         bool plain = false);
int force_brick_depth(const Grid3& g, int min_blocks);

// Separable Gaussian (Sec. 2.5 low-pass filter), x then y then z, replicate
// edges, ncomp components cs apart, fed by TMA.  Skips when *stop_iter < iter.
struct SmoothArgs {
    const void* in;
    void* out;
    Grid3 g;
    int ncomp;           // 1 or 3
    Taps taps;
    const int* stop_iter;
    int iter;
    int* err;            // device error word (kErr* bits)
    int in_type;         // storage of in (kStore*)
    int out_type;        // storage of out
    int zchunk;          // planes per block; 0 = one wave of resident blocks
    bool pdl = false;    // as ForceArgs::pdl (the x/y kernel)
};
// plain = true: the 32 x 8 tile kernel (smooth_kernel) for every storage type
// instead of the packed single-precision kernels
cudaError_t launch_smooth(bool fp64, const SmoothArgs& a, int num_sms, cudaStream_t s,
                          bool plain = false);

// The x and y passes of the Gaussian alone, plane by plane (single precision,
// three components, radius 1..4): out = G_y * G_x * in.  With
// launch_force_zs, which applies G_z, one smoothing + force iteration.
bool smooth_xy_supported(const SmoothArgs& a);
cudaError_t launch_smooth_xy(const SmoothArgs& a, int num_sms, cudaStream_t s);

// Force pass of Eqs. 1-2 whose u is G_z * t, t = a.u the output of
// launch_smooth_xy (single-precision field, float or int16 images, radius 3):
// v = u - dr(u) and the reductions of ForceArgs, the same field bit for bit as
// launch_smooth + launch_force.  Brick depth a.depth (8, 6, 4, 2 or 1).
bool force_zs_supported(int variant, const ForceArgs& a, const Taps& taps);
int force_zs_depth(int variant, const Grid3& g, int num_sms);
cudaError_t launch_force_zs(int variant, const ForceArgs& a, const Taps& taps, cudaStream_t s);

// Eqs. 3-6, the split iteration with the difference image formed once per
// voxel (dir_split_d.cuh): after launch_smooth_xy, the z + D pass (zd: u = t,
// v = the u it writes, dbuf / dbuf2 = the D it writes) and the stencil force
// pass (st: u = that u, v = the field out, dbuf / dbuf2 = that D), each with
// its own brick depth (1, 2, 4 or 8; 6 runs as 4).  force_d_planes: floats per
// voxel of the u + D scratch (4, Eq. 6: 5).
bool force_d_supported(int variant, const ForceArgs& a, const Taps& taps);
int force_d_planes(int variant);
int force_d_depth(const Grid3& g, int num_sms);
cudaError_t launch_force_d(int variant, const ForceArgs& zd, const ForceArgs& st, const Taps& taps,
                           cudaStream_t s);

// Grouped launches of the split schedule: one kernel over the blocks of up to
// kGroupMax volumes (the same pyramid level of several registrations, each
// with its own tensor maps and arguments), so that the fixed latencies of a
// launch are paid once for all of them.  Block b of the launch belongs to job
// j when first[j] <= b < first[j + 1], and is block b - first[j] of that job's
// own grid (gx x gy x gz, x fastest).  Jobs of one launch share the Gaussian
// (radius 3), the force law, the image storage and the brick shape.  The
// structures travel as __grid_constant__ kernel parameters (about 9 KB).
constexpr int kGroupMax = 16;
struct XYGroup {
    CUtensorMap map[kGroupMax];  // each job's plane box of v (x/y kernel layout)
    SmoothArgs a[kGroupMax];
    int first[kGroupMax + 1];
    int gx[kGroupMax], gy[kGroupMax], gz[kGroupMax];
    int n = 0;                   // jobs
    int ty = 0;                  // tile rows, 16 or 32 (all jobs)
    int zchunk = 0;              // planes per block (all jobs)
};
struct ZSGroup {
    CUtensorMap tmap[kGroupMax], smap[kGroupMax], mmap[kGroupMax];
    ForceArgs a[kGroupMax];
    int first[kGroupMax + 1];
    int gx[kGroupMax], gy[kGroupMax], gz[kGroupMax];
    Taps taps;
    int n = 0;
    int variant = 0;             // force law (all jobs)
    int depth = 0;               // brick depth (all jobs)
};
// Shapes for a group of jobs with the given level grids: the x/y kernel's tile
// rows and z chunk, and the z + force kernel's brick depth (the one-volume
// rules applied to the group's total block count).
void group_shapes(int variant, const Grid3* grids, int n, int num_sms, int* ty, int* zchunk,
                  int* depth);
// Add a job (its arguments; a.in / a.u its input field) to a group with
// shapes already set; false if a tensor map cannot be made.
bool xy_group_add(XYGroup& G, const SmoothArgs& a);
bool zs_group_add(ZSGroup& G, const ForceArgs& a);
// pdl: as programmatic dependent launches (the kernels wait for the one
// before them before they touch a field; no stop test in a grouped batch)
cudaError_t launch_smooth_xy_grouped(const XYGroup& G, cudaStream_t s, bool pdl = false);
cudaError_t launch_force_zs_grouped(int variant, int img_type, const ZSGroup& G, cudaStream_t s,
                                    bool pdl = false);

// The Eqs. 3-6 split after the difference image, grouped the same way: the z +
// D kernel (each job's t map and arguments as for launch_force_d's zd) and the
// stencil force kernel (its D, S, u and Eq. 6 d maps and arguments as for
// st); both groups share first / gx / gy / gz and the brick depth (1, 2 or 4).
struct ZDGroup {
    CUtensorMap tmap[kGroupMax];
    ForceArgs a[kGroupMax];
    int first[kGroupMax + 1];
    int gx[kGroupMax], gy[kGroupMax], gz[kGroupMax];
    Taps taps;
    int n = 0;
    int variant = 0;
    int depth = 0;
};
struct STGroup {
    CUtensorMap dmap[kGroupMax], smap[kGroupMax], umap[kGroupMax], emap[kGroupMax];
    ForceArgs a[kGroupMax];
    int first[kGroupMax + 1];
    int gx[kGroupMax], gy[kGroupMax], gz[kGroupMax];
    int n = 0;
    int variant = 0;
    int depth = 0;
};
// Add one job to both groups (variant and depth already set on them)
bool d_group_add(ZDGroup& Z, STGroup& T, const ForceArgs& zd, const ForceArgs& st);
cudaError_t launch_force_d_grouped(int img_type, const ZDGroup& Z, const STGroup& T,
                                   cudaStream_t s, bool pdl = false);

// One fused iteration (Eqs. 1-2 only): u = G_sigma * vin on the fly, then the
// force kernel's work, v = u - dr(u); red as for ForceArgs.
struct FusedArgs {
    const void* S;
    const void* M;
    const void* vin;     // v of the previous iteration (3 components)
    void* v;             // v of this iteration
    Grid3 g;
    Taps taps;
    double* red;
    const int* stop_iter;
    int iter;
    int* err;
    double* corr = nullptr;  // as ForceArgs::corr
};
bool fused_supported(int variant);
// the level is small enough for the all-planes-at-once fused kernel (one block
// per SM covers it); there the fused iteration beats the two-kernel schedule
bool fused_small_level(const Grid3& g, int num_sms);
cudaError_t launch_fused(int variant, bool fp64, const FusedArgs& a, int num_sms, cudaStream_t s);

// out(i, j, k) = in(2i, 2j, 2k)   (pyramid decimation, Sec. 2.3; float or double)
cudaError_t launch_decimate(bool fp64, const void* in, const Grid3& gin, void* out,
                            const Grid3& gout, cudaStream_t s);
// The field kernels below take the field storage type ftype (kStoreF32,
// kStoreBF16 with float arithmetic; kStoreF64 with double).
// fine(x) = 2 * trilinear(coarse, x / 2), per component (Sec. 2.3)
cudaError_t launch_upsample(bool fp64, int ftype, const void* coarse, const Grid3& gc, void* fine,
                            const Grid3& gf, cudaStream_t s);
// out(x) = img(x + u(x)); img in the arithmetic type, out written dense float
cudaError_t launch_warp(bool fp64, int ftype, const void* img, const void* u, const Grid3& g,
                        float* out_dense, cudaStream_t s);
// u(y) = 2 h(x*), x* = y + h(x*) by `steps` fixed-point steps (Eq. 6 output)
cudaError_t launch_ic_invert(bool fp64, int ftype, const void* h, void* u, const Grid3& g,
                             int steps, cudaStream_t s);
// dense[c*N + i + nx*(j + ny*k)] = scale[c] * field[c*cs + pitched(i,j,k)],
// written as float (out_fp64 = false) or double
cudaError_t launch_export_field(bool fp64, int ftype, const void* field, const Grid3& g, double sx,
                                double sy, double sz, void* dense, bool out_fp64, cudaStream_t s);
// pitched[c] = dense float input converted to out_type, for ncomp components
cudaError_t launch_import(bool fp64, int out_type, const float* dense, void* pitched,
                          const Grid3& g, int ncomp, cudaStream_t s);
// one bounded wait on an mbarrier that never completes; sets kErrTmaTimeout
// in *err when it gives up after limit_ns
cudaError_t launch_wait_probe(int* err, unsigned long long limit_ns, cudaStream_t s);
// stop test of Sec. 2.4 for iteration t of a level on the relative norm
// (corr == nullptr) or on the correlation coefficient of the warped image with
// its reference (corr: the four sums of each iteration, n: voxels of the level)
cudaError_t launch_stop_test(const double* red, const double* corr, double n, double* lhist,
                             int t, int level_first, int window, double eps, int* stop_iter,
                             int iter_in_level, cudaStream_t s);
// correlation coefficient from Sum d^2 and the four sums of CorrSums over n voxels
__host__ __device__ inline double correlation_from_sums(double sdd, const double* c, double n) {
    const double sb = c[0], sbb = c[1], sd = c[2], sbd = c[3];
    const double sa = sb + sd, saa = sbb + 2.0 * sbd + sdd, sab = sbb + sbd;
    const double cov = sab - sa * sb / n, va = saa - sa * sa / n, vb = sbb - sb * sb / n;
    return (va > 0.0 && vb > 0.0) ? cov / sqrt(va * vb) : nan("");
}

}  // namespace dirk
