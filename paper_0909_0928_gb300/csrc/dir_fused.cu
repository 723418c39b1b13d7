// dir_fused.cu -- one demons iteration in one pass, for the force laws that
// need no gradient of the warped image (Eq. 1 passive, Eq. 2 evolved passive).
//
// Iteration k keeps v_k = u_k + du_k in memory instead of u_k: the kernel reads
// v_{k-1}, smooths it on the fly into u_k = G_sigma * v_{k-1} (Sec. 2.1: the
// total field is smoothed), then warps M by u_k, applies the force and writes
// v_k, with the reductions of Sec. 2.4 on the way.  The first iteration of a
// level (u_0 given) uses the plain force kernel and the last v is smoothed
// once more by the smoothing kernel, so the arithmetic and its order are those
// of the two-kernel schedule while each iteration moves about 32 bytes per
// voxel instead of 56.
//
// Layout: the TMA plane pipeline of dir_stencil.cuh smooths the three field
// components of a 32 x 8 column tile plane by plane; the smoothed plane goes
// through shared memory to the 256 force threads (one voxel each), which
// gather M through L1/L2 and keep a rolling z window of S (and M for Eq. 2).
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_common.cuh"
#include "dir_force_kernel.cuh"
#include "dir_force_law.cuh"
#include "dir_launch.h"
#include "dir_smooth2.cuh"
#include "dir_stencil.cuh"

namespace dirk {

constexpr int FUSED_NT = STX * STY;  // 256: one force voxel per thread and plane

template <typename Real, int R>
struct FusedGeom {
    using G = StencilGeom<Real, R, 3>;
    static constexpr int UTILE_BYTES = 3 * STY * STX * (int)sizeof(Real);
    static constexpr int SMEM = G::BASE_SMEM + UTILE_BYTES;
};

template <typename Real, int R, int V>
__global__ void __launch_bounds__(FUSED_NT, R <= 4 ? 2 : 1)
    fused_kernel(const __grid_constant__ CUtensorMap tmap, const FusedArgs a, int zchunk) {
    static_assert(V == 0 || V == 1, "fused iteration needs no warped-image gradient");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    using G = StencilGeom<Real, R, 3>;
    constexpr int K = G::K;
    extern __shared__ unsigned char smem_raw[];
    const Grid3 g = a.g;
    const Real* __restrict__ S = static_cast<const Real*>(a.S);
    const Real* __restrict__ M = static_cast<const Real*>(a.M);
    Real* __restrict__ vout = static_cast<Real*>(a.v);
    Real w[K];
#pragma unroll
    for (int t = 0; t < K; ++t) w[t] = tap<Real>(a.taps, t);

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * STX, y0 = blockIdx.y * STY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    // smoothing role (first G::YT threads): column, component, row group
    const bool smoother = tid < G::YT;
    const int lx = tid % STX;
    const int c_own = (tid / STX) % 3;
    const int q_own = (tid / STX) / 3;
    // force role (all threads): one voxel of the tile
    const int fx = tid % STX, fy = tid / STX;
    const int x = x0 + fx, y = y0 + fy;
    const bool valid = (x < g.nx) && (y < g.ny);
    const int xc = min(x, g.nx - 1), yc = min(y, g.ny - 1);
    const int xm = max(xc - 1, 0), xp = min(xc + 1, g.nx - 1);
    const int ym = max(yc - 1, 0), yp = min(yc + 1, g.ny - 1);

    PlanePipe<Real, R, 3> pipe;
    pipe.setup(smem_raw, g, x0, y0, z0, z1);
    Real* utile = reinterpret_cast<Real*>(pipe.extra());  // [3][STY][STX]
    pipe.start(&tmap, g, tid);

    Real ring[K][YW];
#pragma unroll
    for (int t = 0; t < K; ++t)
#pragma unroll
        for (int r = 0; r < YW; ++r) ring[t][r] = Real(0);

    // rolling z windows of S (and M for Eq. 2) at this thread's force voxel
    Real s_m1 = __ldg(S + offs(g, xc, yc, max(z0 - 1, 0)));
    Real s_0 = __ldg(S + offs(g, xc, yc, z0));
    Real m_m1 = 0, m_0 = 0;
    if (V == 1) {
        m_m1 = __ldg(M + offs(g, xc, yc, max(z0 - 1, 0)));
        m_0 = __ldg(M + offs(g, xc, yc, z0));
    }
    Real sd2 = 0, sdu = 0, su = 0;  // per-thread partial sums
    CorrSums<Real> corr_s;          // with a.corr: the correlation sums

    for (int step = 0; step < pipe.nsteps; ++step) {
        if (!pipe.template xpass<FUSED_NT>(&tmap, g, step, tid, w, a.err)) {
            return;
        }
        const bool out_plane = step >= 2 * R;
        if (smoother) {
            pipe.ypass(c_own, q_own, lx, w, ring);
            if (out_plane) {
#pragma unroll
                for (int r = 0; r < YW; ++r)
                    utile[(c_own * STY + q_own * YW + r) * STX + lx] = zpass<Real, R>(w, ring, r);
            }
        }
        __syncthreads();
        if (out_plane) {
            const int zo = z0 + step - 2 * R;
            const int zn = min(zo + 1, g.nz - 1);
            const Real s_p1 = __ldg(S + offs(g, xc, yc, zn));
            Real m_p1 = 0;
            if (V == 1) m_p1 = __ldg(M + offs(g, xc, yc, zn));
            if (valid) {
                const int o = offs(g, x, y, zo);
                const Real ux = utile[(0 * STY + fy) * STX + fx];
                const Real uy = utile[(1 * STY + fy) * STX + fx];
                const Real uz = utile[(2 * STY + fy) * STX + fx];
                const Real d = trilinear(M, g, x, ux, y, uy, zo, uz, s_0);  // W - S
                if (a.corr) corr_s.add(s_0, d);
                const int ro = offs(g, 0, y, zo);
                const Real gsx = Real(0.5) * (__ldg(S + ro + xp) - __ldg(S + ro + xm));
                const Real gsy =
                    Real(0.5) * (__ldg(S + offs(g, x, yp, zo)) - __ldg(S + offs(g, x, ym, zo)));
                const Real gsz = Real(0.5) * (s_p1 - s_m1);
                Real bm = 0;
                if (V == 1) {
                    const Real mx = Real(0.5) * (__ldg(M + ro + xp) - __ldg(M + ro + xm));
                    const Real my = Real(0.5) *
                                    (__ldg(M + offs(g, x, yp, zo)) - __ldg(M + offs(g, x, ym, zo)));
                    const Real mz = Real(0.5) * (m_p1 - m_m1);
                    bm = r_sqrt(mx * mx + my * my + mz * mz);
                }
                Real dx, dy, dz;
                demons_force<Real, V>(d, gsx, gsy, gsz, Real(0), Real(0), Real(0), bm, Real(0), dx,
                                      dy, dz);
                dx = -dx;
                dy = -dy;
                dz = -dz;
                sd2 += d * d;
                sdu += r_norm_fast(dx * dx + dy * dy + dz * dz);
                su += r_norm_fast(ux * ux + uy * uy + uz * uz);
                vout[o] = ux + dx;
                vout[o + (int)g.cs] = uy + dy;
                vout[o + 2 * (int)g.cs] = uz + dz;
            }
            s_m1 = s_0;
            s_0 = s_p1;
            if (V == 1) {
                m_m1 = m_0;
                m_0 = m_p1;
            }
        }
    }
    block_reduce3_atomic<FUSED_NT, Real>(sd2, sdu, su, a.red);
    if (a.corr) block_reduce4_atomic<FUSED_NT, Real>(corr_s, a.corr);
}

template <typename Real, int R, int V>
static cudaError_t launch_rv(const FusedArgs& a, int num_sms, cudaStream_t s) {
    using F = FusedGeom<Real, R>;
    CUtensorMap map;
    if (!make_plane_map<Real, R, 3>(&map, a.vin, a.g, 3)) return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    int per_sm = 1;
    const cudaError_t e = setup_kernel(setup, fused_kernel<Real, R, V>, F::SMEM, FUSED_NT, &per_sm);
    if (e != cudaSuccess) return e;
    const int zc = stencil_zchunk(a.g, per_sm, num_sms);
    const dim3 grid((a.g.nx + STX - 1) / STX, (a.g.ny + STY - 1) / STY, (a.g.nz + zc - 1) / zc);
    fused_kernel<Real, R, V><<<grid, dim3(FUSED_NT, 1, 1), F::SMEM, s>>>(map, a, zc);
    return cudaGetLastError();
}

template <typename Real, int R>
static cudaError_t launch_r(int variant, const FusedArgs& a, int num_sms, cudaStream_t s) {
    return variant == 1 ? launch_rv<Real, R, 1>(a, num_sms, s) : launch_rv<Real, R, 0>(a, num_sms, s);
}

template <typename Real>
static cudaError_t launch_t(int variant, const FusedArgs& a, int num_sms, cudaStream_t s) {
    switch (a.taps.R) {
        case 1: return launch_r<Real, 1>(variant, a, num_sms, s);
        case 2: return launch_r<Real, 2>(variant, a, num_sms, s);
        case 3: return launch_r<Real, 3>(variant, a, num_sms, s);
        case 4: return launch_r<Real, 4>(variant, a, num_sms, s);
        case 5: return launch_r<Real, 5>(variant, a, num_sms, s);
        case 6: return launch_r<Real, 6>(variant, a, num_sms, s);
        case 7: return launch_r<Real, 7>(variant, a, num_sms, s);
        case 8: return launch_r<Real, 8>(variant, a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}


// ---------------------------------------------------------------------------
// Single-precision fused iteration on the packed smoothing of dir_smooth2.cuh.
// A block of 384 threads owns a 32 x 16 column tile and a z chunk: three
// groups of 128 threads smooth the three components of v_{k-1} plane by plane
// (one TMA copy brings the plane box of all three), the smoothed plane u_k
// goes through shared memory, and 256 threads then do the force work for its
// 512 voxels, two each (rows r and r + 8).  S arrives by TMA too, one plane
// box (tile + 1-voxel halo) per step into a ring that holds the planes zo - 1,
// zo, zo + 1 of the output plane zo, so the static gradient and the reference
// S(x) of the warped difference come from shared memory; M is gathered
// through L1/L2.  The arithmetic of every voxel is that of the smoothing and
// force kernels (same building blocks, same order).
// ---------------------------------------------------------------------------
constexpr int F2T = 3 * S2T;            // 384 threads
constexpr int F2ST = 4;                 // stages of the v plane ring
constexpr int F2SST = F2ST + 3;         // S ring: 3 planes read, F2ST - 1 in flight, 1 spare
constexpr int F2SX = 4;                 // S box x halo (16-byte aligned start)
constexpr int F2SW = S2X + 2 * F2SX;    // S box width: x0 - 4 .. x0 + 35
constexpr int F2SH = S2Y + 2;           // S box rows: y0 - 1 .. y0 + 16

template <int R>
struct F2Geom {
    using G = S2Geom<R>;
    static constexpr int VBOX = 3 * G::SLOT;  // the plane box of all three components
    static constexpr int VSTRIDE = (VBOX + 127) / 128 * 128;
    static constexpr int SBOX = F2SH * F2SW * 4;
    static constexpr int SSTRIDE = (SBOX + 127) / 128 * 128;
    static constexpr int UTILE = 3 * S2Y * S2X * 4;
    static constexpr int OFF_S = F2ST * VSTRIDE;
    static constexpr int OFF_TXP = OFF_S + F2SST * SSTRIDE;
    static constexpr int OFF_U = OFF_TXP + 3 * G::TXP_STRIDE;
    static constexpr int OFF_BAR = OFF_U + UTILE;
    static constexpr int SMEM = 128 + OFF_BAR + 64;
};

template <int R, int V>
__global__ void __launch_bounds__(F2T, 2)
    fused2_kernel(const __grid_constant__ CUtensorMap vmap, const __grid_constant__ CUtensorMap smap,
                  const FusedArgs a, int zchunk) {
    static_assert(V == 0 || V == 1, "fused iteration needs no warped-image gradient");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    using G = S2Geom<R>;
    using F = F2Geom<R>;
    constexpr int K = G::K, H = G::H, HA = G::HA, WB = G::WB;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + F::OFF_BAR);
    float* utile = reinterpret_cast<float*>(base + F::OFF_U);  // [3][S2Y][S2X]
    const Grid3 g = a.g;
    const float* __restrict__ M = static_cast<const float*>(a.M);
    float* __restrict__ vout = static_cast<float*>(a.v);
    float w[R + 1];
    f32x2 wp[R + 1];
#pragma unroll
    for (int t = 0; t <= R; ++t) {
        w[t] = a.taps.wf[t];
        wp[t] = f2_pack(w[t], w[t]);
    }
    const int tid = threadIdx.x;
    const int grp = tid >> 7, gt = tid & 127;  // smoothing: component group, thread in it
    const int lx = gt & 31, q = gt >> 5;
    f32x2* txp = reinterpret_cast<f32x2*>(base + F::OFF_TXP + grp * G::TXP_STRIDE);
    float* txf = reinterpret_cast<float*>(txp);
    const int x0 = blockIdx.x * S2X, y0 = blockIdx.y * S2Y;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    const int nsteps = (z1 - z0) + 2 * R;
    const int bx = x0 - HA, by = y0 - R;
    const int sbx = x0 - F2SX, sby = y0 - 1;
    const bool edge = (bx < 0) || (bx + WB > g.nx) || (by < 0) || (by + H > g.ny);

    // step s loads the v planes z0 - R + s and the S plane z0 - 2R + 1 + s
    // (the plane above the output plane of that step), both clamped
    auto issue = [&](int step) {
        const int sl = step % F2ST;
        const int pv = clampi(z0 - R + step, 0, g.nz - 1);
        const int ps = clampi(z0 - 2 * R + 1 + step, 0, g.nz - 1);
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[sl], (uint32_t)(F::VBOX + F::SBOX));
        tma_load_4d(base + sl * F::VSTRIDE, &vmap, bx, by, pv, 0, &full[sl]);
        tma_load_4d(base + F::OFF_S + (step % F2SST) * F::SSTRIDE, &smap, sbx, sby, ps, 0,
                    &full[sl]);
    };
    if (tid == 0) {
        for (int sl = 0; sl < F2ST; ++sl) mbar_init(&full[sl], 1);
        fence_mbar_init();
        fence_proxy_async();
        for (int st = 0; st < F2ST - 1 && st < nsteps; ++st) issue(st);
    }
    __syncthreads();

    f32x2 ring[K][2];
#pragma unroll
    for (int t = 0; t < K; ++t) ring[t][0] = ring[t][1] = 0ull;

    // force role: threads 0..255, column fx, rows fr and fr + 8 of the tile
    const bool forcer = tid < 2 * S2T;
    const int fx = tid & 31, fr = (tid >> 5) & 7;
    const int x = x0 + fx;
    const int xc = min(x, g.nx - 1);
    const int sxm = max(xc - 1, 0) - sbx, sxc = xc - sbx, sxp = min(xc + 1, g.nx - 1) - sbx;
    const Interp ip(g);
    const int cs = (int)g.cs;
    float sd2 = 0.0f, sdu = 0.0f, su = 0.0f;
    CorrSums<float> corr_s;  // with a.corr: the correlation sums

    for (int step = 0; step < nsteps; ++step) {
        if (tid == 0 && step + F2ST - 1 < nsteps) issue(step + F2ST - 1);
        const int sl = step % F2ST;
        const uint32_t parity = (uint32_t)((step / F2ST) & 1);
        bool ok = true;
        if (tid == 0) ok = mbar_wait_bounded(&full[sl], parity, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && a.err) atomicOr(a.err, kErrTmaTimeout);
            return;
        }
        (void)mbar_try_wait(&full[sl], parity);
        float* vslots = reinterpret_cast<float*>(base + sl * F::VSTRIDE);  // [3][H][WB]
        if (edge) s2_edge_fix<R>(vslots, H * WB, 3, bx, by, g, tid, F2T);
        s2_xpass<R>(vslots + grp * H * WB, txf, gt, w);
        __syncthreads();
        const bool emit = step >= 2 * R;
        S2_RING_SWITCH(R, step % K, {
            s2_y<R, J>(txp, q, lx, wp, ring);
            if (emit) {
                f32x2 r0, r1;
                s2_z<R, J>(wp, ring, r0, r1);
                float a0, b0, a1, b1;
                f2_unpack(r0, a0, b0);
                f2_unpack(r1, a1, b1);
                float* ut = utile + grp * (S2Y * S2X) + lx;
                ut[(2 * q) * S2X] = a0;
                ut[(2 * q + 1) * S2X] = a1;
                ut[(2 * q + S2Y / 2) * S2X] = b0;
                ut[(2 * q + S2Y / 2 + 1) * S2X] = b1;
            }
        })
        if (!emit) continue;  // uniform
        __syncthreads();
        if (forcer) {
            const int zo = z0 + step - 2 * R;
            // S planes zo - 1, zo, zo + 1 (clamped) from the ring
            const float* Sm = reinterpret_cast<const float*>(
                base + F::OFF_S + ((step + F2SST - 2) % F2SST) * F::SSTRIDE);
            const float* Sc = reinterpret_cast<const float*>(
                base + F::OFF_S + ((step + F2SST - 1) % F2SST) * F::SSTRIDE);
            const float* Sp =
                reinterpret_cast<const float*>(base + F::OFF_S + (step % F2SST) * F::SSTRIDE);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = fr + h * (S2Y / 2);
                const int y = y0 + row;
                if (x < g.nx && y < g.ny) {
                    const int syc = y - sby, sym = max(y - 1, 0) - sby, syp = min(y + 1, g.ny - 1) - sby;
                    const float ux = utile[(0 * S2Y + row) * S2X + fx];
                    const float uy = utile[(1 * S2Y + row) * S2X + fx];
                    const float uz = utile[(2 * S2Y + row) * S2X + fx];
                    const float s0 = Sc[syc * F2SW + sxc];
                    const float gsx = 0.5f * (Sc[syc * F2SW + sxp] - Sc[syc * F2SW + sxm]);
                    const float gsy = 0.5f * (Sc[syp * F2SW + sxc] - Sc[sym * F2SW + sxc]);
                    const float gsz = 0.5f * (Sp[syc * F2SW + sxc] - Sm[syc * F2SW + sxc]);
                    const float d = interp_rel(M, ip, x, ux, y, uy, zo, uz, s0);  // W - S
                    if (a.corr) corr_s.add(s0, d);
                    float bm = 0.0f;
                    if (V == 1) {
                        const int o = offs(g, x, y, zo);
                        const int xm = max(x - 1, 0), xp = min(x + 1, g.nx - 1);
                        const int ro = o - x;
                        const float mx = 0.5f * (__ldg(M + ro + xp) - __ldg(M + ro + xm));
                        const float my = 0.5f * (__ldg(M + offs(g, x, min(y + 1, g.ny - 1), zo)) -
                                                 __ldg(M + offs(g, x, max(y - 1, 0), zo)));
                        const float mz = 0.5f * (__ldg(M + offs(g, x, y, min(zo + 1, g.nz - 1))) -
                                                 __ldg(M + offs(g, x, y, max(zo - 1, 0))));
                        bm = r_sqrt(mx * mx + my * my + mz * mz);
                    }
                    float dx, dy, dz;
                    demons_force<float, V>(d, gsx, gsy, gsz, 0.0f, 0.0f, 0.0f, bm, 0.0f, dx, dy, dz);
                    dx = -dx;
                    dy = -dy;
                    dz = -dz;
                    sd2 += d * d;
                    sdu += r_norm_fast(dx * dx + dy * dy + dz * dz);
                    su += r_norm_fast(ux * ux + uy * uy + uz * uz);
                    const int o = offs(g, x, y, zo);
                    vout[o] = ux + dx;
                    vout[o + cs] = uy + dy;
                    vout[o + 2 * cs] = uz + dz;
                }
            }
        }
        // the next step's __syncthreads_or orders these reads of the u tile and
        // of the S ring before they are rewritten
    }
    block_reduce3_atomic<F2T, float>(sd2, sdu, su, a.red);
    if (a.corr) block_reduce4_atomic<F2T, float>(corr_s, a.corr);
}

template <int R>
static bool make_f2_maps(CUtensorMap* vmap, CUtensorMap* smap, const FusedArgs& a) {
    using G = S2Geom<R>;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const Grid3& g = a.g;
    const cuuint64_t vdims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
    const cuuint64_t sdims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 1};
    const cuuint64_t strides[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                   (cuuint64_t)g.cs * 4};
    const cuuint32_t vbox[4] = {(cuuint32_t)G::WB, (cuuint32_t)G::H, 1u, 3u};
    const cuuint32_t sbox[4] = {(cuuint32_t)F2SW, (cuuint32_t)F2SH, 1u, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    auto ok = [&](CUtensorMap* m, const void* p, const cuuint64_t* d, const cuuint32_t* b) {
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(p), d, strides, b, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
               CUDA_SUCCESS;
    };
    return ok(vmap, a.vin, vdims, vbox) && ok(smap, a.S, sdims, sbox);
}

template <int R, int V>
static cudaError_t launch_f2(const FusedArgs& a, int num_sms, cudaStream_t s) {
    using F = F2Geom<R>;
    CUtensorMap vmap, smap;
    if (!make_f2_maps<R>(&vmap, &smap, a)) return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    int per_sm = 1;
    const cudaError_t e = setup_kernel(setup, fused2_kernel<R, V>, F::SMEM, F2T, &per_sm);
    if (e != cudaSuccess) return e;
    const int tiles = ((a.g.nx + S2X - 1) / S2X) * ((a.g.ny + S2Y - 1) / S2Y);
    long long chunks = ((long long)(per_sm < 1 ? 1 : per_sm) * num_sms) / tiles;
    if (chunks < 1) chunks = 1;
    if (chunks > a.g.nz) chunks = a.g.nz;
    const int zc = (int)((a.g.nz + chunks - 1) / chunks);
    const dim3 grid((a.g.nx + S2X - 1) / S2X, (a.g.ny + S2Y - 1) / S2Y, (a.g.nz + zc - 1) / zc);
    fused2_kernel<R, V><<<grid, dim3(F2T, 1, 1), F::SMEM, s>>>(vmap, smap, a, zc);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Fused iteration for small levels (where the marching kernel would get z
// chunks of one or two planes and spend each iteration waiting on a chain of
// plane steps): a block of 384 threads owns a 32 x 16 tile and FZC = 2 output
// planes, fetches the FZC + 2R input planes of all three components in ONE
// TMA copy (plus the S planes zo - 1 .. zo + FZC), and runs every pass over all
// planes at once: x pass of all planes, y pass into per-plane pair rows, z pass
// with the clamped plane indices, then the force work.  One copy latency and
// four barriers per iteration instead of 2R + FZC sequential steps.  Same
// building blocks and order of operations as the marching kernels.
// ---------------------------------------------------------------------------
constexpr int FZC = 2;

template <int R>
struct FSGeom {
    using G = S2Geom<R>;
    static constexpr int NP = FZC + 2 * R;                          // input planes
    static constexpr int PLANE = G::H * G::WB;                      // floats per plane box
    static constexpr int VBOX = 3 * NP * PLANE * 4;                 // [3][NP][H][WB]
    static constexpr int SNP = FZC + 2;                             // S planes
    static constexpr int SBOX = SNP * F2SH * F2SW * 4;              // [SNP][F2SH][F2SW]
    static constexpr int YPL = (S2Y / 2) * S2X;                     // f32x2 per y-filtered plane
    static constexpr int OFF_S = (VBOX + 127) / 128 * 128;
    static constexpr int OFF_TXP = OFF_S + (SBOX + 127) / 128 * 128;
    static constexpr int OFF_U = OFF_TXP + 3 * NP * G::TXP_STRIDE;
    static constexpr int UT = FZC * 3 * S2Y * S2X * 4;              // [FZC][3][S2Y][S2X]
    static constexpr int OFF_BAR = OFF_U + UT;
    static constexpr int SMEM = 128 + OFF_BAR + 64;
    static_assert(3 * NP * YPL * 8 <= VBOX, "y-filtered planes reuse the plane boxes");
};

template <int R, int V>
__global__ void __launch_bounds__(F2T, 1)
    fused_small_kernel(const __grid_constant__ CUtensorMap vmap,
                       const __grid_constant__ CUtensorMap smap, const FusedArgs a) {
    static_assert(V == 0 || V == 1, "fused iteration needs no warped-image gradient");
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    using G = S2Geom<R>;
    using F = FSGeom<R>;
    constexpr int K = G::K, H = G::H, HA = G::HA, WB = G::WB, NP = F::NP;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + F::OFF_BAR);
    float* vbox = reinterpret_cast<float*>(base);                      // [3][NP][H][WB]
    f32x2* ypl = reinterpret_cast<f32x2*>(base);                       // [3][NP][8][32], after x
    const float* sbox = reinterpret_cast<const float*>(base + F::OFF_S);  // [SNP][F2SH][F2SW]
    float* utile = reinterpret_cast<float*>(base + F::OFF_U);          // [FZC][3][S2Y][S2X]
    const Grid3 g = a.g;
    const float* __restrict__ M = static_cast<const float*>(a.M);
    float* __restrict__ vout = static_cast<float*>(a.v);
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
    const int z0 = blockIdx.z * FZC;
    const int zb = z0 - R;       // z of box plane 0 (v)
    const int zs = z0 - 1;       // z of box plane 0 (S)
    const int bx = x0 - HA, by = y0 - R;
    const int sbx = x0 - F2SX, sby = y0 - 1;
    const bool edge = (bx < 0) || (bx + WB > g.nx) || (by < 0) || (by + H > g.ny);
    // input planes inside the volume (the others are zero-filled by the copy
    // and never read: every plane index below is clamped into [pa, pb])
    const int pa = max(0, -zb), pb = min(NP - 1, g.nz - 1 - zb);

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, (uint32_t)(F::VBOX + F::SBOX));
        tma_load_4d(vbox, &vmap, bx, by, zb, 0, bar);
        tma_load_4d(base + F::OFF_S, &smap, sbx, sby, zs, 0, bar);
    }
    __syncthreads();
    bool ok = true;
    if (tid == 0) ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (__syncthreads_or(!ok)) {
        if (tid == 0 && a.err) atomicOr(a.err, kErrTmaTimeout);
        return;
    }
    (void)mbar_try_wait(bar, 0);
    if (edge) s2_edge_fix<R>(vbox, H * WB, 3 * NP, bx, by, g, tid, F2T);
    // x pass of every in-volume plane of this group's component
    f32x2* txp_c = reinterpret_cast<f32x2*>(base + F::OFF_TXP) + (size_t)grp * NP * (G::TXP_STRIDE / 8);
    for (int p = pa; p <= pb; ++p)
        s2_xpass<R>(vbox + (grp * NP + p) * F::PLANE,
                    reinterpret_cast<float*>(txp_c + p * (G::TXP_STRIDE / 8)), gt, w);
    __syncthreads();
    // y pass of every in-volume plane into the pair-row planes (the plane
    // boxes are dead now); pairs (row 2q + j, row 2q + j + 8), j = 0, 1
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
    // z pass of the output planes, oldest plane first, clamped plane indices
#pragma unroll
    for (int j = 0; j < FZC; ++j) {
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
        float* ut = utile + ((j * 3 + grp) * S2Y) * S2X + lx;
        ut[(2 * q) * S2X] = a0;
        ut[(2 * q + 1) * S2X] = a1;
        ut[(2 * q + S2Y / 2) * S2X] = b0;
        ut[(2 * q + S2Y / 2 + 1) * S2X] = b1;
    }
    __syncthreads();
    // force work: FZC planes x 512 voxels over the 384 threads
    const Interp ip(g);
    const int cs = (int)g.cs;
    const int spa = max(0, -zs), spb = min(F::SNP - 1, g.nz - 1 - zs);  // in-volume S planes
    float sd2 = 0.0f, sdu = 0.0f, su = 0.0f;
    CorrSums<float> corr_s;  // with a.corr: the correlation sums
    for (int k = tid; k < FZC * S2Y * S2X; k += F2T) {
        const int j = k / (S2Y * S2X), row = (k / S2X) % S2Y, fx = k % S2X;
        const int x = x0 + fx, y = y0 + row, zo = z0 + j;
        if (x >= g.nx || y >= g.ny || zo >= g.nz) continue;
        const int sxc = x - sbx, sxm = max(x - 1, 0) - sbx, sxp = min(x + 1, g.nx - 1) - sbx;
        const int syc = y - sby, sym = max(y - 1, 0) - sby, syp = min(y + 1, g.ny - 1) - sby;
        const float* Sc = sbox + clampi(j + 1, spa, spb) * (F2SH * F2SW);
        const float* Sm = sbox + clampi(j, spa, spb) * (F2SH * F2SW);
        const float* Sp = sbox + clampi(j + 2, spa, spb) * (F2SH * F2SW);
        const float* ut = utile + (j * 3 * S2Y + row) * S2X + fx;
        const float ux = ut[0], uy = ut[S2Y * S2X], uz = ut[2 * S2Y * S2X];
        const float s0 = Sc[syc * F2SW + sxc];
        const float gsx = 0.5f * (Sc[syc * F2SW + sxp] - Sc[syc * F2SW + sxm]);
        const float gsy = 0.5f * (Sc[syp * F2SW + sxc] - Sc[sym * F2SW + sxc]);
        const float gsz = 0.5f * (Sp[syc * F2SW + sxc] - Sm[syc * F2SW + sxc]);
        const float d = interp_rel(M, ip, x, ux, y, uy, zo, uz, s0);  // W - S
        if (a.corr) corr_s.add(s0, d);
        float bm = 0.0f;
        if (V == 1) {
            const int o = offs(g, x, y, zo);
            const int ro = o - x;
            const float mx = 0.5f * (__ldg(M + ro + min(x + 1, g.nx - 1)) - __ldg(M + ro + max(x - 1, 0)));
            const float my = 0.5f * (__ldg(M + offs(g, x, min(y + 1, g.ny - 1), zo)) -
                                     __ldg(M + offs(g, x, max(y - 1, 0), zo)));
            const float mz = 0.5f * (__ldg(M + offs(g, x, y, min(zo + 1, g.nz - 1))) -
                                     __ldg(M + offs(g, x, y, max(zo - 1, 0))));
            bm = r_sqrt(mx * mx + my * my + mz * mz);
        }
        float dx, dy, dz;
        demons_force<float, V>(d, gsx, gsy, gsz, 0.0f, 0.0f, 0.0f, bm, 0.0f, dx, dy, dz);
        dx = -dx;
        dy = -dy;
        dz = -dz;
        sd2 += d * d;
        sdu += r_norm_fast(dx * dx + dy * dy + dz * dz);
        su += r_norm_fast(ux * ux + uy * uy + uz * uz);
        const int o = offs(g, x, y, zo);
        vout[o] = ux + dx;
        vout[o + cs] = uy + dy;
        vout[o + 2 * cs] = uz + dz;
    }
    block_reduce3_atomic<F2T, float>(sd2, sdu, su, a.red);
    if (a.corr) block_reduce4_atomic<F2T, float>(corr_s, a.corr);
}

// one block per SM with FZC-plane chunks covers the level
static bool small_level(const Grid3& g, int num_sms) {
    const long long tiles = (long long)((g.nx + S2X - 1) / S2X) * ((g.ny + S2Y - 1) / S2Y);
    return tiles * ((g.nz + FZC - 1) / FZC) <= num_sms;
}

template <int R, int V>
static cudaError_t launch_fs(const FusedArgs& a, cudaStream_t s) {
    using G = S2Geom<R>;
    using F = FSGeom<R>;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorInvalidValue;
    const Grid3& g = a.g;
    const cuuint64_t vdims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 3};
    const cuuint64_t sdims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 1};
    const cuuint64_t strides[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                   (cuuint64_t)g.cs * 4};
    const cuuint32_t vbox[4] = {(cuuint32_t)G::WB, (cuuint32_t)G::H, (cuuint32_t)F::NP, 3u};
    const cuuint32_t sbox[4] = {(cuuint32_t)F2SW, (cuuint32_t)F2SH, (cuuint32_t)F::SNP, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    CUtensorMap vmap, smap;
    auto enc4 = [&](CUtensorMap* m, const void* p, const cuuint64_t* d, const cuuint32_t* b) {
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(p), d, strides, b, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
               CUDA_SUCCESS;
    };
    if (!enc4(&vmap, a.vin, vdims, vbox) || !enc4(&smap, a.S, sdims, sbox))
        return cudaErrorInvalidValue;
    static KernelSetup setup;  // per instantiation
    const cudaError_t e = setup_kernel(setup, fused_small_kernel<R, V>, F::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.nx + S2X - 1) / S2X, (g.ny + S2Y - 1) / S2Y, (g.nz + FZC - 1) / FZC);
    fused_small_kernel<R, V><<<grid, dim3(F2T, 1, 1), F::SMEM, s>>>(vmap, smap, a);
    return cudaGetLastError();
}

template <int R>
static cudaError_t launch_f2r(int variant, const FusedArgs& a, int num_sms, cudaStream_t s) {
    if (R <= 3 && small_level(a.g, num_sms))
        return variant == 1 ? launch_fs<R <= 3 ? R : 3, 1>(a, s) : launch_fs<R <= 3 ? R : 3, 0>(a, s);
    return variant == 1 ? launch_f2<R, 1>(a, num_sms, s) : launch_f2<R, 0>(a, num_sms, s);
}

bool fused_supported(int variant) { return variant == 0 || variant == 1; }

bool fused_small_level(const Grid3& g, int num_sms) { return small_level(g, num_sms); }

cudaError_t launch_fused(int variant, bool fp64, const FusedArgs& a, int num_sms, cudaStream_t s) {
    if (!fused_supported(variant)) return cudaErrorInvalidValue;
    if (fp64) return launch_t<double>(variant, a, num_sms, s);
    switch (a.taps.R) {  // the packed kernel for the usual radii
        case 1: return launch_f2r<1>(variant, a, num_sms, s);
        case 2: return launch_f2r<2>(variant, a, num_sms, s);
        case 3: return launch_f2r<3>(variant, a, num_sms, s);
        case 4: return launch_f2r<4>(variant, a, num_sms, s);
        default: return launch_t<float>(variant, a, num_sms, s);
    }
}

}  // namespace dirk
