// dir_smooth2.cuh -- building blocks of the packed single-precision Gaussian
// (Sec. 2.5 low-pass filter, applied along x, then y, then z with replicated
// edges), shared by the smoothing kernel and the fused iteration kernel.
//
// Geometry: a block smooths 32 x TY (x, y) tiles plane by plane (TY = 16 by
// default, 32 for the large-level smoothing kernel).  Each input
// plane (tile + halo: H = 16 + 2R rows, WB = 32 + 2 HA columns with the x
// start 16-byte aligned) arrives by TMA.  The x pass (scalar, 4 outputs per
// task from 128-bit shared loads) writes its rows into a pair-interleaved
// buffer in which row m sits beside row m + TY/2, so that the y and z passes
// run on f32x2 pairs (rows y and y + TY/2 of one column; fma.rn.f32x2 does
// both lanes, each rounded as the scalar FMA would be).  A group of 8 TY
// threads owns one component: thread (lx, q) holds column lx and rows
// {2q, 2q+1, 2q+TY/2, 2q+TY/2+1}, filters them in y from 64-bit shared loads,
// keeps the 2R+1
// most recent y-filtered planes in registers and filters them in z.  The y
// and z steps are instantiated per ring position J (the caller switches on
// the plane index modulo 2R+1), so the ring rotates by renaming.
//
// The taps are symmetric (tap t equals tap 2R - t), so only w[0..R] are kept.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_common.cuh"

namespace dirk {

constexpr int S2X = 32, S2Y = 16, S2T = 128;
constexpr int S2TP = S2X + 1;  // pair-row pitch in f32x2 (the pad staggers banks)

template <int R, int TY = S2Y>
struct S2Geom {
    static constexpr int K = 2 * R + 1;
    static constexpr int NTG = 8 * TY;                            // threads per component group
    static constexpr int H = TY + 2 * R;                          // box rows
    static constexpr int HA = (R + 3) / 4 * 4;                    // x halo, 16-byte aligned start
    static constexpr int WB = S2X + 2 * HA;                       // box width
    static constexpr int NPR = TY / 2 + 2 * R;                    // pair rows (m, m + TY/2)
    static constexpr int XLV = (HA - R + 4 + 2 * R + 3) / 4 * 4;  // x-task inputs, whole float4s
    static constexpr int SLOT = H * WB * 4;                       // bytes of one plane box
    static constexpr int SLOT_STRIDE = (SLOT + 127) / 128 * 128;
    static constexpr int TXP = NPR * S2TP * 8;                    // bytes of the pair rows
    static constexpr int TXP_STRIDE = (TXP + 127) / 128 * 128;
    static constexpr int XTASKS = H * (S2X / 4);                  // x tasks per plane
    static_assert(XTASKS > NTG && XTASKS <= 2 * NTG, "x tasks: one or two per thread");
};

template <int R>
__device__ __forceinline__ float s2_w(const float (&w)[R + 1], int t) {
    return w[t <= R ? t : 2 * R - t];
}

// x pass of one task: box row rho, outputs 4 gq .. 4 gq + 3, written to the
// pair rows (as the low lane of pair row rho and the high lane of pair row
// rho - TY/2, where those exist)
template <int R, int TY = S2Y>
__device__ __forceinline__ void s2_xtask(const float* __restrict__ slot, float* __restrict__ txf,
                                         int tk, const float (&w)[R + 1]) {
    using G = S2Geom<R, TY>;
    constexpr int K = 2 * R + 1, HA = G::HA, WB = G::WB, NPR = G::NPR;
    const int gq = tk & 7, rho = tk >> 3;
    const float* src = slot + rho * WB + 4 * gq;
    float in[G::XLV];
#pragma unroll
    for (int v = 0; v < G::XLV / 4; ++v) {
        const float4 t4 = reinterpret_cast<const float4*>(src)[v];
        in[4 * v] = t4.x;
        in[4 * v + 1] = t4.y;
        in[4 * v + 2] = t4.z;
        in[4 * v + 3] = t4.w;
    }
    float o[4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < K; ++t) acc = fmaf(s2_w<R>(w, t), in[HA - R + jj + t], acc);
        o[jj] = acc;
    }
    if (rho < NPR) {
        float* d = txf + 2 * (rho * S2TP + 4 * gq);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) d[2 * jj] = o[jj];
    }
    if (rho >= TY / 2) {
        float* d = txf + 2 * ((rho - TY / 2) * S2TP + 4 * gq) + 1;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) d[2 * jj] = o[jj];
    }
}

// x pass of a whole plane by the 8 TY threads of one group (tid in 0..8 TY-1)
template <int R, int TY = S2Y>
__device__ __forceinline__ void s2_xpass(const float* __restrict__ slot, float* __restrict__ txf,
                                         int tid, const float (&w)[R + 1]) {
    using G = S2Geom<R, TY>;
    s2_xtask<R, TY>(slot, txf, tid, w);
    if (tid < G::XTASKS - G::NTG) s2_xtask<R, TY>(slot, txf, tid + G::NTG, w);
}

// Replicate boundary in a TMA plane box of `nc` components (zero-filled where
// outside the volume): out-of-volume columns first (a thread per row), then
// out-of-volume rows (a thread per column).  bx, by: box origin.  Every thread
// of the block calls it (two barriers).
template <int R, int TY = S2Y>
__device__ __forceinline__ void s2_edge_fix(float* slots, int slot_stride_floats, int nc, int bx,
                                            int by, const Grid3& g, int tid, int nthreads) {
    using G = S2Geom<R, TY>;
    constexpr int H = G::H, WB = G::WB;
    const int lo = max(0, -bx), hi = min(WB, g.nx - bx);
    for (int row = tid; row < nc * H; row += nthreads) {
        float* r = slots + (row / H) * slot_stride_floats + (row % H) * WB;
        const float left = r[lo], right = r[hi - 1];
        for (int hx = 0; hx < lo; ++hx) r[hx] = left;
        for (int hx = hi; hx < WB; ++hx) r[hx] = right;
    }
    __syncthreads();
    const int rlo = max(0, -by), rhi = min(H, g.ny - by);
    for (int col = tid; col < nc * WB; col += nthreads) {
        float* c = slots + (col / WB) * slot_stride_floats + (col % WB);
        const float top = c[rlo * WB], bot = c[(rhi - 1) * WB];
        for (int hy = 0; hy < rlo; ++hy) c[hy * WB] = top;
        for (int hy = rhi; hy < H; ++hy) c[hy * WB] = bot;
    }
    __syncthreads();
}

// y pass of one plane for thread (q, lx): p0 = rows (2q, 2q + TY/2) and
// p1 = rows (2q + 1, 2q + TY/2 + 1) of column lx, from pair rows 2q + t and
// 2q + 1 + t
template <int R>
__device__ __forceinline__ void s2_y_pair(const f32x2* __restrict__ txp, int q, int lx,
                                          const f32x2 (&wp)[R + 1], f32x2& p0, f32x2& p1) {
    constexpr int K = 2 * R + 1;
    f32x2 in2[K + 1];
#pragma unroll
    for (int m = 0; m < K + 1; ++m) in2[m] = txp[(2 * q + m) * S2TP + lx];
    p0 = 0ull;
    p1 = 0ull;
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const f32x2 wt = wp[t <= R ? t : 2 * R - t];
        p0 = f2_fma(wt, in2[t], p0);
        p1 = f2_fma(wt, in2[t + 1], p1);
    }
}

// the same into ring slot J
template <int R, int J>
__device__ __forceinline__ void s2_y(const f32x2* __restrict__ txp, int q, int lx,
                                     const f32x2 (&wp)[R + 1], f32x2 (&ring)[2 * R + 1][2]) {
    s2_y_pair<R>(txp, q, lx, wp, ring[J][0], ring[J][1]);
}

// z pass over the ring whose newest plane is in slot J, oldest plane first:
// r0 = (row 2q, row 2q + TY/2), r1 = (row 2q + 1, row 2q + TY/2 + 1)
template <int R, int J>
__device__ __forceinline__ void s2_z(const f32x2 (&wp)[R + 1], const f32x2 (&ring)[2 * R + 1][2],
                                     f32x2& r0, f32x2& r1) {
    constexpr int K = 2 * R + 1;
    r0 = 0ull;
    r1 = 0ull;
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const f32x2 wt = wp[t <= R ? t : 2 * R - t];
        r0 = f2_fma(wt, ring[(J + 1 + t) % K][0], r0);
        r1 = f2_fma(wt, ring[(J + 1 + t) % K][1], r1);
    }
}

// The ring-position switch: runs the statement list (variadic, may contain
// commas) with the compile-time constant J equal to `pos` (0 <= pos < 2R+1 <= 9).
#define S2_RING_CASE(R_, j, ...) \
    case j: {                    \
        constexpr int J = (j) % (2 * (R_) + 1); \
        __VA_ARGS__;             \
    } break;
#define S2_RING_SWITCH(R_, pos, ...)                                                       \
    switch (pos) {                                                                         \
        S2_RING_CASE(R_, 0, __VA_ARGS__) S2_RING_CASE(R_, 1, __VA_ARGS__)                  \
        S2_RING_CASE(R_, 2, __VA_ARGS__) S2_RING_CASE(R_, 3, __VA_ARGS__)                  \
        S2_RING_CASE(R_, 4, __VA_ARGS__) S2_RING_CASE(R_, 5, __VA_ARGS__)                  \
        S2_RING_CASE(R_, 6, __VA_ARGS__) S2_RING_CASE(R_, 7, __VA_ARGS__)                  \
        S2_RING_CASE(R_, 8, __VA_ARGS__)                                                   \
        default: break;                                                                    \
    }

}  // namespace dirk
