// dir_smooth.cu -- separable 3-D Gaussian low-pass filter (Sec. 2.5).
//
// out = G_sigma * in, applied along x, then y, then z, with replicated edges,
// on 1 or 3 components, in three forms:
//  * smooth2_kernel (single-precision fields): one component of a 32 x TY
//    tile (TY = 32 on large levels, 16 otherwise) over a z chunk, fed by a
//    ring of TMA plane copies, y and z passes on packed f32x2 row pairs;
//  * smooth_small_kernel (single precision, small levels): all planes of a
//    two-plane chunk and all three components in one TMA copy;
//  * smooth_kernel (double precision, int16 or bf16 storage): the TMA-fed
//    plane pipeline of dir_stencil.cuh on 32 x 8 tiles.
// The components run as independent blocks (three times the marching chains
// per SM).  Every input voxel is read from HBM about once per launch (plus
// the 2R-plane halo of each z chunk).
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_common.cuh"
#include "dir_launch.h"
#include "dir_smooth2.cuh"
#include "dir_split.cuh"
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


// ---------------------------------------------------------------------------
// Single-precision field smoothing, packed (building blocks and layout in
// dir_smooth2.cuh): a block of 8 TY threads smooths one component of a
// 32 x TY tile over a z chunk, fed by a 6-deep ring of TMA plane copies.
// ---------------------------------------------------------------------------
constexpr int S2STAGES = 6;
constexpr bool kSmoothTall = true;  // 32-row tiles on large levels

template <int R, int TY>
struct S2Smem {
    using G = S2Geom<R, TY>;
    static constexpr int SMEM = 128 + S2STAGES * G::SLOT_STRIDE + G::TXP_STRIDE + 64;
};

template <int R, int TY>
__global__ void __launch_bounds__(8 * TY, 16 / TY * 8)
    smooth2_kernel(const __grid_constant__ CUtensorMap tmap, const SmoothArgs a, int zchunk) {
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    using G = S2Geom<R, TY>;
    constexpr int K = G::K, H = G::H, HA = G::HA, WB = G::WB, NT = G::NTG;
    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned by pointer arithmetic on the shared array (keeps the
    // accesses below in the shared address space)
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    f32x2* txp = reinterpret_cast<f32x2*>(base + S2STAGES * G::SLOT_STRIDE);
    float* txf = reinterpret_cast<float*>(txp);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + S2STAGES * G::SLOT_STRIDE + G::TXP_STRIDE);
    const Grid3 g = a.g;
    float w[R + 1];  // symmetric taps w[0..R]
    f32x2 wp[R + 1];
#pragma unroll
    for (int t = 0; t <= R; ++t) {
        w[t] = a.taps.wf[t];
        wp[t] = f2_pack(w[t], w[t]);
    }
    const int tid = threadIdx.x;
    const int lx = tid & 31, q = tid >> 5;
    const int comp = blockIdx.z % a.ncomp;
    const int x0 = blockIdx.x * S2X, y0 = blockIdx.y * TY;
    const int z0 = (blockIdx.z / a.ncomp) * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    const int nsteps = (z1 - z0) + 2 * R;  // input planes z0-R .. z1-1+R (clamped)
    const int bx = x0 - HA, by = y0 - R;
    const bool edge = (bx < 0) || (bx + WB > g.nx) || (by < 0) || (by + H > g.ny);
    float* __restrict__ out = static_cast<float*>(a.out) + (long long)comp * g.cs;

    auto issue = [&](int step) {
        const int sl = step % S2STAGES;
        const int pc = clampi(z0 - R + step, 0, g.nz - 1);
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[sl], (uint32_t)G::SLOT);
        tma_load_4d(base + sl * G::SLOT_STRIDE, &tmap, bx, by, pc, comp, &full[sl]);
    };
    if (tid == 0) {
        for (int sl = 0; sl < S2STAGES; ++sl) mbar_init(&full[sl], 1);
        fence_mbar_init();
        fence_proxy_async();
        for (int st = 0; st < S2STAGES - 1 && st < nsteps; ++st) issue(st);
    }
    __syncthreads();

    f32x2 ring[K][2];
#pragma unroll
    for (int t = 0; t < K; ++t) ring[t][0] = ring[t][1] = 0ull;

    const int x = x0 + lx;
    const int ya = y0 + 2 * q;  // rows ya, ya + 1 (lane 0) and ya + TY/2, ya + TY/2 + 1 (lane 1)
    const int px = (int)g.px;
    const int rows_left = x < g.nx ? g.ny - ya : 0;  // 0: this thread stores nothing
    for (int step = 0; step < nsteps; ++step) {
        if (tid == 0 && step + S2STAGES - 1 < nsteps) issue(step + S2STAGES - 1);
        const int sl = step % S2STAGES;
        const uint32_t parity = (uint32_t)((step / S2STAGES) & 1);
        bool ok = true;
        if (tid == 0) ok = mbar_wait_bounded(&full[sl], parity, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && a.err) atomicOr(a.err, kErrTmaTimeout);
            return;
        }
        (void)mbar_try_wait(&full[sl], parity);
        float* slot = reinterpret_cast<float*>(base + sl * G::SLOT_STRIDE);  // [H][WB]
        if (edge) s2_edge_fix<R, TY>(slot, G::SLOT_STRIDE / 4, 1, bx, by, g, tid, NT);
        s2_xpass<R, TY>(slot, txf, tid, w);
        __syncthreads();
        const bool emit = step >= 2 * R;
        float* o = out + offs(g, x < g.nx ? x : 0, ya, emit ? z0 + step - 2 * R : 0);
        S2_RING_SWITCH(R, step % K, {
            s2_y<R, J>(txp, q, lx, wp, ring);
            if (emit) {
                f32x2 r0, r1;
                s2_z<R, J>(wp, ring, r0, r1);
                float a0, b0, a1, b1;
                f2_unpack(r0, a0, b0);
                f2_unpack(r1, a1, b1);
                if (rows_left > 0) o[0] = a0;
                if (rows_left > 1) o[px] = a1;
                if (rows_left > TY / 2) o[(TY / 2) * px] = b0;
                if (rows_left > TY / 2 + 1) o[(TY / 2 + 1) * px] = b1;
            }
        })
        // no barrier here: the next step's __syncthreads_or orders this
        // step's reads of the pair rows before the next x pass rewrites them
    }
}

// ---------------------------------------------------------------------------
// The x and y passes alone (single precision, three components), for the
// schedule that runs the z pass inside the force kernel (dir_force_tma.cu):
// out(x, y, z) = G_y * G_x * in on every plane, plane by plane.  Without a z
// pass there is no z halo, so a block's z chunk can be as short as the
// occupancy wants at no extra work, and there is no ring of filtered planes.
// Same building blocks, layout and order of operations as smooth2_kernel.
// ---------------------------------------------------------------------------
template <int R, int TY>
__global__ void __launch_bounds__(8 * TY)
    smooth_xy_kernel(const __grid_constant__ CUtensorMap tmap, const SmoothArgs a, int zchunk) {
    sxy_block<R, TY>(&tmap, a, zchunk, BlockPos::of_grid());
}

// ---------------------------------------------------------------------------
// Field smoothing for small levels: a block of 384 threads (a group of 128
// per component) owns a 32 x 16 tile and SZC = 2 output planes, fetches the
// SZC + 2R input planes of all three components in one TMA copy and runs the
// x, y and z passes over all planes at once (see the fused small-level kernel
// in dir_fused.cu; same building blocks and order of operations as the
// marching kernel above).
// ---------------------------------------------------------------------------
constexpr int SZC = 2, SST = 3 * S2T;

template <int R>
struct SSGeom {
    using G = S2Geom<R>;
    static constexpr int NP = SZC + 2 * R;
    static constexpr int PLANE = G::H * G::WB;
    static constexpr int VBOX = 3 * NP * PLANE * 4;
    static constexpr int YPL = (S2Y / 2) * S2X;
    static constexpr int OFF_TXP = (VBOX + 127) / 128 * 128;
    static constexpr int OFF_BAR = OFF_TXP + 3 * NP * G::TXP_STRIDE;
    static constexpr int SMEM = 128 + OFF_BAR + 64;
    static_assert(3 * NP * YPL * 8 <= VBOX, "y-filtered planes reuse the plane boxes");
};

template <int R>
__global__ void __launch_bounds__(SST, 1)
    smooth_small_kernel(const __grid_constant__ CUtensorMap tmap, const SmoothArgs a) {
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    using G = S2Geom<R>;
    using F = SSGeom<R>;
    constexpr int K = G::K, H = G::H, HA = G::HA, WB = G::WB, NP = F::NP;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + F::OFF_BAR);
    float* vbox = reinterpret_cast<float*>(base);  // [3][NP][H][WB]
    f32x2* ypl = reinterpret_cast<f32x2*>(base);   // [3][NP][8][32], after the x pass
    const Grid3 g = a.g;
    float w[R + 1];
    f32x2 wp[R + 1];
#pragma unroll
    for (int t = 0; t <= R; ++t) {
        w[t] = a.taps.wf[t];
        wp[t] = f2_pack(w[t], w[t]);
    }
    const int tid = threadIdx.x;
    const int grp = tid >> 7, gt = tid & 127;
    const int lx = gt & 31, q = gt >> 5;
    const int x0 = blockIdx.x * S2X, y0 = blockIdx.y * S2Y;
    const int z0 = blockIdx.z * SZC;
    const int zb = z0 - R;
    const int bx = x0 - HA, by = y0 - R;
    const bool edge = (bx < 0) || (bx + WB > g.nx) || (by < 0) || (by + H > g.ny);
    const int pa = max(0, -zb), pb = min(NP - 1, g.nz - 1 - zb);  // in-volume planes

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)F::VBOX);
        tma_load_4d(vbox, &tmap, bx, by, zb, 0, bar);
    }
    __syncthreads();
    bool ok = true;
    if (tid == 0) ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (__syncthreads_or(!ok)) {
        if (tid == 0 && a.err) atomicOr(a.err, kErrTmaTimeout);
        return;
    }
    (void)mbar_try_wait(bar, 0);
    if (edge) s2_edge_fix<R>(vbox, H * WB, 3 * NP, bx, by, g, tid, SST);
    f32x2* txp_c = reinterpret_cast<f32x2*>(base + F::OFF_TXP) + (size_t)grp * NP * (G::TXP_STRIDE / 8);
    for (int p = pa; p <= pb; ++p)
        s2_xpass<R>(vbox + (grp * NP + p) * F::PLANE,
                    reinterpret_cast<float*>(txp_c + p * (G::TXP_STRIDE / 8)), gt, w);
    __syncthreads();
    for (int p = pa; p <= pb; ++p) {
        const f32x2* tp = txp_c + p * (G::TXP_STRIDE / 8);
        f32x2 in2[K + 1];
#pragma unroll
        for (int m = 0; m < K + 1; ++m) in2[m] = tp[(2 * q + m) * S2TP + lx];
        f32x2 p0 = 0ull, p1 = 0ull;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const f32x2 wt = wp[t <= R ? t : 2 * R - t];
            p0 = f2_fma(wt, in2[t], p0);
            p1 = f2_fma(wt, in2[t + 1], p1);
        }
        f32x2* yp = ypl + (size_t)(grp * NP + p) * F::YPL;
        yp[(2 * q) * S2X + lx] = p0;
        yp[(2 * q + 1) * S2X + lx] = p1;
    }
    __syncthreads();
    float* __restrict__ out = static_cast<float*>(a.out) + (long long)grp * g.cs;
    const int x = x0 + lx, ya = y0 + 2 * q;
    const int rows_left = x < g.nx ? g.ny - ya : 0;
    const int px = (int)g.px;
#pragma unroll
    for (int j = 0; j < SZC; ++j) {
        if (z0 + j >= g.nz) break;
        f32x2 r0 = 0ull, r1 = 0ull;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int pp = clampi(j + t, pa, pb);  // plane z0 + j - R + t, clamped
            const f32x2* yp = ypl + (size_t)(grp * NP + pp) * F::YPL;
            const f32x2 wt = wp[t <= R ? t : 2 * R - t];
            r0 = f2_fma(wt, yp[(2 * q) * S2X + lx], r0);
            r1 = f2_fma(wt, yp[(2 * q + 1) * S2X + lx], r1);
        }
        float a0, b0, a1, b1;
        f2_unpack(r0, a0, b0);
        f2_unpack(r1, a1, b1);
        float* o = out + offs(g, x < g.nx ? x : 0, ya, z0 + j);
        if (rows_left > 0) o[0] = a0;
        if (rows_left > 1) o[px] = a1;
        if (rows_left > S2Y / 2) o[(S2Y / 2) * px] = b0;
        if (rows_left > S2Y / 2 + 1) o[(S2Y / 2 + 1) * px] = b1;
    }
}

static bool smooth_small_level(const Grid3& g, int num_sms) {
    const long long tiles = (long long)((g.nx + S2X - 1) / S2X) * ((g.ny + S2Y - 1) / S2Y);
    return tiles * ((g.nz + SZC - 1) / SZC) <= num_sms;
}

template <int R>
static cudaError_t launch_ss(const SmoothArgs& a, cudaStream_t s) {
    using G = S2Geom<R>;
    using F = SSGeom<R>;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorInvalidValue;
    const Grid3& g = a.g;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
    const cuuint64_t strides[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                   (cuuint64_t)g.cs * 4};
    const cuuint32_t box[4] = {(cuuint32_t)G::WB, (cuuint32_t)G::H, (cuuint32_t)F::NP, 3u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    CUtensorMap map;
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(a.in), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    const cudaError_t e = setup_kernel(setup, smooth_small_kernel<R>, F::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.nx + S2X - 1) / S2X, (g.ny + S2Y - 1) / S2Y, (g.nz + SZC - 1) / SZC);
    smooth_small_kernel<R><<<grid, dim3(SST, 1, 1), F::SMEM, s>>>(map, a);
    return cudaGetLastError();
}

template <int R, int TY>
static bool make_s2_map(CUtensorMap* map, const void* ptr, const Grid3& g, int ncomp) {
    using G = S2Geom<R, TY>;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz,
                                (cuuint64_t)ncomp};
    const cuuint64_t strides[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                   (cuuint64_t)g.cs * 4};
    const cuuint32_t box[4] = {(cuuint32_t)G::WB, (cuuint32_t)G::H, 1u, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(ptr), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// z chunk for the packed kernel: the largest number of chunks that still fits
// in one wave of resident blocks
static int s2_zchunk(const Grid3& g, int ty, int per_sm, int num_sms, int ncomp) {
    if (per_sm < 1) per_sm = 1;
    const long long bxy = (long long)((g.nx + S2X - 1) / S2X) * ((g.ny + ty - 1) / ty) * ncomp;
    long long chunks = ((long long)per_sm * num_sms) / bxy;
    if (chunks < 1) chunks = 1;
    if (chunks > g.nz) chunks = g.nz;
    const int zc = (int)((g.nz + chunks - 1) / chunks);
    return zc < 1 ? 1 : zc;
}

template <int R, int TY>
static cudaError_t launch_s2(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    using G = S2Smem<R, TY>;
    CUtensorMap map;
    if (!make_s2_map<R, TY>(&map, a.in, a.g, a.ncomp)) return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    int per_sm = 1;
    const cudaError_t e = setup_kernel(setup, smooth2_kernel<R, TY>, G::SMEM, 8 * TY, &per_sm);
    if (e != cudaSuccess) return e;
    int zc = a.zchunk > 0 ? a.zchunk : s2_zchunk(a.g, TY, per_sm, num_sms, a.ncomp);
    if (zc > a.g.nz) zc = a.g.nz;
    const int chunks = (a.g.nz + zc - 1) / zc;
    const dim3 grid((a.g.nx + S2X - 1) / S2X, (a.g.ny + TY - 1) / TY, chunks * a.ncomp);
    smooth2_kernel<R, TY><<<grid, dim3(8 * TY, 1, 1), G::SMEM, s>>>(map, a, zc);
    return cudaGetLastError();
}

// tile height: 32 rows where the level is large enough that fewer, taller
// tiles still fill the GPU (less y halo per output), else 16
template <int R>
static cudaError_t launch_s2t(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    const long long tiles32 = (long long)((a.g.nx + S2X - 1) / S2X) * ((a.g.ny + 31) / 32) * a.ncomp;
    if (kSmoothTall && tiles32 * a.g.nz >= 8LL * num_sms) return launch_s2<R, 32>(a, num_sms, s);
    return launch_s2<R, S2Y>(a, num_sms, s);
}

template <int R, int TY>
static cudaError_t launch_sxy(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    using G = SXYSmem<R, TY>;
    CUtensorMap map;
    if (!make_s2_map<R, TY>(&map, a.in, a.g, a.ncomp)) return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    int per_sm = 1;
    const cudaError_t e = setup_kernel(setup, smooth_xy_kernel<R, TY>, G::SMEM, 8 * TY, &per_sm);
    if (e != cudaSuccess) return e;
    // No z halo, so short chunks cost nothing extra: the longest of 4, 2, 1
    // planes that still gives a wave of resident blocks (the autotuner's choice
    // on each level of the 256x256x100 pyramid)
    int zc = a.zchunk;
    if (zc <= 0) {
        const long long bxy =
            (long long)((a.g.nx + S2X - 1) / S2X) * ((a.g.ny + TY - 1) / TY) * a.ncomp;
        const long long slots = (long long)(per_sm < 1 ? 1 : per_sm) * num_sms;
        zc = 1;
        for (int c = 4; c > 1; c /= 2)
            if (bxy * ((a.g.nz + c - 1) / c) >= slots) {
                zc = c;
                break;
            }
    }
    if (zc > a.g.nz) zc = a.g.nz;
    const int chunks = (a.g.nz + zc - 1) / zc;
    const dim3 grid((a.g.nx + S2X - 1) / S2X, (a.g.ny + TY - 1) / TY, chunks * a.ncomp);
    return launch_ex(smooth_xy_kernel<R, TY>, grid, dim3(8 * TY, 1, 1), G::SMEM, s, a.pdl, map, a, zc);
}

template <typename Real, int R, typename TIN, typename TOUT>
static cudaError_t launch_rt(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    using G = StencilGeom<Real, R, 1, 8, TIN>;
    CUtensorMap map;
    if (!make_plane_map<Real, R, 1, TIN>(&map, a.in, a.g, a.ncomp)) return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    int per_sm = 1;
    const cudaError_t e =
        setup_kernel(setup, smooth_kernel<Real, R, TIN, TOUT>, G::BASE_SMEM, G::YT, &per_sm);
    if (e != cudaSuccess) return e;
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

bool smooth_xy_supported(const SmoothArgs& a) {
    return a.ncomp == 3 && a.in_type == kStoreF32 && a.out_type == kStoreF32 && a.taps.R >= 1 &&
           a.taps.R <= 4;
}

cudaError_t launch_smooth_xy(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    if (!smooth_xy_supported(a)) return cudaErrorInvalidValue;
    const long long tiles32 = (long long)((a.g.nx + S2X - 1) / S2X) * ((a.g.ny + 31) / 32) * a.ncomp;
    const bool tall = tiles32 * a.g.nz >= 8LL * num_sms;
    switch (a.taps.R) {
        case 1: return tall ? launch_sxy<1, 32>(a, num_sms, s) : launch_sxy<1, S2Y>(a, num_sms, s);
        case 2: return tall ? launch_sxy<2, 32>(a, num_sms, s) : launch_sxy<2, S2Y>(a, num_sms, s);
        case 3: return tall ? launch_sxy<3, 32>(a, num_sms, s) : launch_sxy<3, S2Y>(a, num_sms, s);
        case 4: return tall ? launch_sxy<4, 32>(a, num_sms, s) : launch_sxy<4, S2Y>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_smooth(bool fp64, const SmoothArgs& a, int num_sms, cudaStream_t s,
                          bool plain) {
    if (a.ncomp != 1 && a.ncomp != 3) return cudaErrorInvalidValue;
    if (fp64) {
        if (a.in_type != kStoreF64 || a.out_type != kStoreF64) return cudaErrorInvalidValue;
        return launch_types<double, double, double>(a, num_sms, s);
    }
    if (a.in_type == kStoreF32 && a.out_type == kStoreF32) {
        if (plain) return launch_types<float, float, float>(a, num_sms, s);
        if (a.ncomp == 3 && a.zchunk == 0 && smooth_small_level(a.g, num_sms)) {
            switch (a.taps.R) {  // small levels: all planes of a chunk at once
                case 1: return launch_ss<1>(a, s);
                case 2: return launch_ss<2>(a, s);
                case 3: return launch_ss<3>(a, s);
                default: break;
            }
        }
        switch (a.taps.R) {  // the packed kernel for the usual radii
            case 1: return launch_s2t<1>(a, num_sms, s);
            case 2: return launch_s2t<2>(a, num_sms, s);
            case 3: return launch_s2t<3>(a, num_sms, s);
            case 4: return launch_s2t<4>(a, num_sms, s);
            default: return launch_types<float, float, float>(a, num_sms, s);
        }
    }
    if (a.in_type == kStoreI16 && a.out_type == kStoreF32)
        return launch_types<float, int16_t, float>(a, num_sms, s);
    if (a.in_type == kStoreBF16 && a.out_type == kStoreBF16)
        return launch_types<float, bf16, bf16>(a, num_sms, s);
    return cudaErrorInvalidValue;
}

}  // namespace dirk
