// dir_common.cuh -- device-side layout and helpers shared by the library's kernels.
//
// Internal volumes are pitched: voxel (i, j, k) of a level lives at
// i + px * j + plane * k with px >= nx a multiple of 32 elements and
// plane = px * ny, so every row starts on a 128-byte boundary.  A field stores
// its three components cs elements apart (cs a multiple of 64).
//
// Every kernel is a template on the scalar type Real (float for production,
// double for the verification precision); the arithmetic is written once.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dirk {

struct Grid3 {
    int nx, ny, nz;   // voxels per axis
    int px;           // row pitch in elements
    long long plane;  // px * ny
    long long cs;     // component stride of a field, elements
};

struct Taps {
    int R;          // radius: 2R+1 taps
    double w[17];   // w[t + R] for t = -R..R (normalised)
    float wf[17];   // the same taps rounded for the single-precision path, with
                    // their exact sum kept at 1 (see make_taps in the engine)
};

template <typename Real>
__device__ __forceinline__ Real tap(const Taps& t, int i);
template <>
__device__ __forceinline__ float tap<float>(const Taps& t, int i) { return t.wf[i]; }
template <>
__device__ __forceinline__ double tap<double>(const Taps& t, int i) { return t.w[i]; }

constexpr int kMaxRadius = 8;

// error bits a kernel can raise in the context's device error word
constexpr int kErrTmaTimeout = 1;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// 32-bit element offsets: the engine bounds volumes so that every field
// offset (three components included) stays below 2^31
__device__ __forceinline__ int offs(const Grid3& g, int i, int j, int k) {
    return i + g.px * j + (int)g.plane * k;
}

// Fused multiply-add written out: every kernel that evaluates the same formula
// then rounds it the same way (the compiler's own contraction of a * b + c
// may pick a different product to fuse in different kernels).
__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return fma(a, b, c); }
// |(x, y, z)|^2 as ((x x) + y y) + z z with the two additions fused
template <typename Real>
__device__ __forceinline__ Real r_sq3(Real x, Real y, Real z) {
    return r_fma(z, z, r_fma(y, y, x * x));
}
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float r_floor(float x) { return floorf(x); }
__device__ __forceinline__ double r_floor(double x) { return floor(x); }
__device__ __forceinline__ float r_clamp(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }
// division and vector norm as used by the single-precision path: the CUDA fast
// intrinsics (about 2 ulp); the double-precision path stays exact
__device__ __forceinline__ float r_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double r_div(double a, double b) { return a / b; }
__device__ __forceinline__ float r_norm_fast(float s) { return s > 0.0f ? s * rsqrtf(s) : 0.0f; }
__device__ __forceinline__ double r_norm_fast(double s) { return sqrt(s); }
__device__ __forceinline__ double r_clamp(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

// ---------------------------------------------------------------- storage types
// Images and fields may be stored narrower than the arithmetic: int16 HU
// images (exact), bf16 fields.  Every load widens to Real, every store rounds
// to the storage type (round to nearest even).
typedef __nv_bfloat16 bf16;

template <typename Real, typename T>
__device__ __forceinline__ Real ldg_as(const T* p) { return (Real)__ldg(p); }
template <>
__device__ __forceinline__ float ldg_as<float, bf16>(const bf16* p) { return __bfloat162float(__ldg(p)); }
template <typename Real, typename T>
__device__ __forceinline__ Real ld_as(const T* p) { return (Real)*p; }
template <>
__device__ __forceinline__ float ld_as<float, bf16>(const bf16* p) { return __bfloat162float(*p); }
template <typename T, typename Real>
__device__ __forceinline__ T st_as(Real v) { return (T)v; }
template <>
__device__ __forceinline__ bf16 st_as<bf16, float>(float v) { return __float2bfloat16_rn(v); }

// One axis of the trilinear setup (Sec. 2.5 interpolation, clamped
// coordinates) at p = base + off, base an integer voxel index: clamp p to
// [0, n-1], lower corner floor(p) kept <= n-2 so the upper corner exists,
// weight p - corner.  Splitting p keeps the weight accurate to the precision
// of the offset rather than of base + off (single precision at base = 255
// would otherwise round p to about 3e-5 voxel).
template <typename Real>
__device__ __forceinline__ void axis_setup(int base, Real off, int n, int& i0, int& i1, Real& f) {
    const Real fl = r_floor(r_clamp(off, Real(-1048576), Real(1048576)));
    const int i = base + (int)fl;
    if (n < 2) {
        i0 = i1 = 0;
        f = Real(0);
    } else if (i < 0) {                       // p < 0: clamped to 0
        i0 = 0;
        i1 = 1;
        f = Real(0);
    } else if (i >= n - 1) {                  // p >= n-1: clamped to n-1
        i0 = n - 2;
        i1 = n - 1;
        f = Real(1);
    } else {
        i0 = i;
        i1 = i + 1;
        f = off - fl;
    }
}

// Software trilinear interpolation of a pitched volume at the continuous voxel
// position (bx + ox, by + oy, bz + oz), minus a reference value `ref`; lerps
// along x, then y, then z.  The corners are taken relative to ref before the
// lerps, so the result is rounded to the precision of its own size rather
// than of the image's: with ref = S(x), M(x + u) - S(x) has single-precision
// error of a few ulp of the intensity difference, where interpolating M first
// would leave an error of an ulp of |M| (about 6e-5 HU at -1000 HU), which the
// demons iteration amplifies in homogeneous regions.  Each corner difference
// is exact when the corner is within a factor two of ref.
template <typename Real, typename T>
__device__ __forceinline__ Real trilinear(const T* __restrict__ I, const Grid3& g, int bx,
                                          Real ox, int by, Real oy, int bz, Real oz,
                                          Real ref = Real(0)) {
    int x0, x1, y0, y1, z0, z1;
    Real fx, fy, fz;
    axis_setup(bx, ox, g.nx, x0, x1, fx);
    axis_setup(by, oy, g.ny, y0, y1, fy);
    axis_setup(bz, oz, g.nz, z0, z1, fz);
    const int pl = (int)g.plane;
    const T* p00 = I + (g.px * y0 + pl * z0);
    const T* p10 = I + (g.px * y1 + pl * z0);
    const T* p01 = I + (g.px * y0 + pl * z1);
    const T* p11 = I + (g.px * y1 + pl * z1);
    const Real c000 = ldg_as<Real>(p00 + x0) - ref, c100 = ldg_as<Real>(p00 + x1) - ref;
    const Real c010 = ldg_as<Real>(p10 + x0) - ref, c110 = ldg_as<Real>(p10 + x1) - ref;
    const Real c001 = ldg_as<Real>(p01 + x0) - ref, c101 = ldg_as<Real>(p01 + x1) - ref;
    const Real c011 = ldg_as<Real>(p11 + x0) - ref, c111 = ldg_as<Real>(p11 + x1) - ref;
    const Real gx = Real(1) - fx, gy = Real(1) - fy, gz = Real(1) - fz;
    const Real v00 = r_fma(c100, fx, c000 * gx);
    const Real v10 = r_fma(c110, fx, c010 * gx);
    const Real v01 = r_fma(c101, fx, c001 * gx);
    const Real v11 = r_fma(c111, fx, c011 * gx);
    const Real v0 = r_fma(v10, fy, v00 * gy);
    const Real v1 = r_fma(v11, fy, v01 * gy);
    return r_fma(v1, fz, v0 * gz);
}

// Block-wide sum of three per-thread partial sums, then one FP64 atomic per
// value.  Within a warp the sums stay in the working precision (float for the
// production path: 32 partials of a few voxels each); across warps and blocks
// they are added in double (the global MSE / convergence reduction).  Every
// thread of the block must call it.
template <int NT, typename Real>
__device__ __forceinline__ void block_reduce3_atomic(Real a, Real b, Real c, double* out) {
    static_assert(NT % 32 == 0, "block size must be whole warps");
    __shared__ double red_s[3][NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        red_s[0][warp] = (double)a;
        red_s[1][warp] = (double)b;
        red_s[2][warp] = (double)c;
    }
    __syncthreads();
    if (warp == 0) {
        double da = lane < NT / 32 ? red_s[0][lane] : 0.0;
        double db = lane < NT / 32 ? red_s[1][lane] : 0.0;
        double dc = lane < NT / 32 ? red_s[2][lane] : 0.0;
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

// The sums of the correlation coefficient of the warped image with its
// reference (Secs. 2.4, 3.3): per voxel b (S; Eq. 6: the warped static image)
// and d = W - b; the field's own statistics keep Sum d^2.  Accumulated per
// thread, then reduced like block_reduce3_atomic into out[0..3] =
// {Sum b, Sum b^2, Sum d, Sum b d}.
template <typename Real>
struct CorrSums {
    Real b = 0, bb = 0, d = 0, bd = 0;
    __device__ __forceinline__ void add(Real bv, Real dv) {
        b += bv;
        bb = r_fma(bv, bv, bb);
        d += dv;
        bd = r_fma(bv, dv, bd);
    }
};

template <int NT, typename Real>
__device__ __forceinline__ void block_reduce4_atomic(const CorrSums<Real>& s, double* out) {
    static_assert(NT % 32 == 0, "block size must be whole warps");
    __shared__ double red4_s[4][NT / 32];
    Real v[4] = {s.b, s.bb, s.d, s.bd};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) red4_s[k][warp] = (double)v[k];
    __syncthreads();
    if (warp == 0) {
        double dv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) dv[k] = lane < NT / 32 ? red4_s[k][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 4; ++k) dv[k] += __shfl_down_sync(0xffffffffu, dv[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(out + k, dv[k]);
    }
}

// ------------------------------------------------- packed single precision
// Two float lanes in one 64-bit register (low lane = first float in memory),
// operated on by the f32x2 instructions of sm_100 and later: one instruction
// does two independent single-precision operations, each rounded exactly as
// its scalar counterpart.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {  // a * b + c
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---------------------------------------------------------------- TMA / mbarrier
// Bulk tensor copies (cp.async.bulk.tensor) complete on an mbarrier in shared
// memory; waits are bounded by the global timer so that a copy that never
// lands raises an error instead of hanging the GPU.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete is
// suspended in hardware until it completes (or the hint runs out) instead of
// re-issuing the test, so a waiting warp takes no issue slots from the others.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity,
                                                      uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the barrier; gives up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_suspend(bar, parity, 1000000u)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream serialization attribute may start while the kernel before it in the
// stream still runs.  pdl_trigger lets the next kernel start; pdl_wait blocks
// until the kernels this one depends on have completed and their memory is
// visible.  Both are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Position of a block in its own launch grid: the whole launch, or one job's
// share of a grouped launch over several volumes.
struct BlockPos {
    int x, y, z;     // block coordinates
    int gx, gy, gz;  // grid extent
    __device__ __forceinline__ static BlockPos of_grid() {
        return {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                (int)gridDim.x,  (int)gridDim.y,  (int)gridDim.z};
    }
};

// 4-D tiled tensor load global -> shared, completing on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_u32(bar))
        : "memory");
}

// Ask L2 to fetch the 4-D box at (c0, c1, c2, c3) of a tensor map (no
// shared-memory destination, nothing to wait for).
__device__ __forceinline__ void tma_prefetch_4d(const CUtensorMap* map, int c0, int c1, int c2,
                                                int c3) {
    asm volatile(
        "cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

}  // namespace dirk
