// dir_smooth.cu -- separable 3-D Gaussian low-pass filter (Sec. 2.5).
//
// out = G_sigma * in, applied along x, then y, then z, with replicated edges,
// on 1 or 3 components.  The paper stages data in shared memory so that the
// strided y and z passes stay coalesced; here a block owns a 32 x 8 column tile
// and marches through a chunk of z planes:
//   * one thread issues TMA tensor copies (cp.async.bulk.tensor) of each input
//     plane's tile plus halo, all components at once, into a 4-slot ring of
//     shared memory, several planes ahead, each slot completing on its own
//     mbarrier;
//   * edge tiles overwrite the zero-filled out-of-volume cells with the nearest
//     edge voxel (replicate boundary) in shared memory;
//   * x pass: each task filters 4 adjacent outputs of one row from three
//     128-bit shared loads; y pass: each thread filters 4 rows of one column of
//     one component; z pass: a rolling window of 2R+1 y-filtered planes in the
//     same thread's registers.
// Every input voxel is read from HBM about once per launch (plus the 2R-plane
// halo of each z chunk), and the filter costs about 10 instructions per tap
// row of 4 outputs instead of one shared load per tap.
#include <cuda.h>
#include <cuda_runtime.h>

#include "dir_common.cuh"
#include "dir_launch.h"

namespace dirk {

constexpr int STX = 32, STY = 8, STAGES = 4, YW = 4;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

template <typename Real>
struct Vec16;  // 16-byte vector of Real
template <>
struct Vec16<float> {
    using T = float4;
    static constexpr int N = 4;
};
template <>
struct Vec16<double> {
    using T = double2;
    static constexpr int N = 2;
};

__device__ __forceinline__ void unpack(const float4& t, float* d) {
    d[0] = t.x;
    d[1] = t.y;
    d[2] = t.z;
    d[3] = t.w;
}
__device__ __forceinline__ void unpack(const double2& t, double* d) {
    d[0] = t.x;
    d[1] = t.y;
}
__device__ __forceinline__ float4 pack4(const float* s) { return make_float4(s[0], s[1], s[2], s[3]); }
__device__ __forceinline__ double2 pack2(const double* s) { return make_double2(s[0], s[1]); }
__device__ __forceinline__ void store4(float* dst, const float* s) {
    *reinterpret_cast<float4*>(dst) = pack4(s);
}
__device__ __forceinline__ void store4(double* dst, const double* s) {
    reinterpret_cast<double2*>(dst)[0] = pack2(s);
    reinterpret_cast<double2*>(dst)[1] = pack2(s + 2);
}

template <typename Real, int R, int NC>
struct SmoothGeom {
    static constexpr int HA = (R + 3) / 4 * 4;   // x halo rounded up: TMA x start 16-byte aligned
    static constexpr int WB = STX + 2 * HA;      // box width
    static constexpr int H = STY + 2 * R;        // box height
    static constexpr int K = 2 * R + 1;
    static constexpr int NT = STX * NC * (STY / YW);  // threads: one per (x, component, row group)
    static constexpr int XL = 4 + 2 * R;              // inputs of one 4-output x task
    static constexpr int XLV = (HA - R + XL + 3) / 4 * 4;  // loaded span, whole 16-byte vectors
    static constexpr int SLOT_ELEMS = NC * H * WB;
    static constexpr int SLOT_BYTES = SLOT_ELEMS * (int)sizeof(Real);
    static constexpr int SLOT_STRIDE = (SLOT_BYTES + 127) / 128 * 128;
    static constexpr int TXP_BYTES = NC * H * STX * (int)sizeof(Real);
    static constexpr int SMEM = 128 /*align slack*/ + STAGES * SLOT_STRIDE + TXP_BYTES + 64;
};

template <typename Real, int R, int NC>
__global__ void __launch_bounds__(SmoothGeom<Real, R, NC>::NT)
    smooth_kernel(const __grid_constant__ CUtensorMap tmap, const SmoothArgs a, int zchunk) {
    if (a.stop_iter != nullptr && *a.stop_iter < a.iter) return;
    using G = SmoothGeom<Real, R, NC>;
    using V = typename Vec16<Real>::T;
    constexpr int HA = G::HA, WB = G::WB, H = G::H, K = G::K, NT = G::NT;
    constexpr int VN = Vec16<Real>::N;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    Real* txp = reinterpret_cast<Real*>(base + STAGES * G::SLOT_STRIDE);          // [NC][H][STX]
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * G::SLOT_STRIDE + G::TXP_BYTES);

    const Grid3 g = a.g;
    Real* __restrict__ out = static_cast<Real*>(a.out);
    Real w[K];
#pragma unroll
    for (int t = 0; t < K; ++t) w[t] = (Real)a.taps.w[t];

    const int tid = threadIdx.x;
    // y/z role: column x, component c, rows y0 + 4*q .. +3
    const int lx = tid % STX;
    const int grp = tid / STX;
    const int c_own = grp % NC;
    const int q_own = grp / NC;
    const int x0 = blockIdx.x * STX, y0 = blockIdx.y * STY;
    const int x = x0 + lx;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    const int nsteps = (z1 - z0) + 2 * R;  // input planes z0-R .. z1-1+R (clamped)
    const int bx = x0 - HA, by = y0 - R;   // box origin in the volume
    const bool edge = (bx < 0) || (bx + WB > g.nx) || (by < 0) || (by + H > g.ny);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
        fence_proxy_async();
    }
    __syncthreads();
    auto issue = [&](int step) {
        const int s = step % STAGES;
        const int pc = clampi(z0 - R + step, 0, g.nz - 1);
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[s], (uint32_t)G::SLOT_BYTES);
        tma_load_4d(base + s * G::SLOT_STRIDE, &tmap, bx, by, pc, 0, &full[s]);
    };
    if (tid == 0) {
        for (int st = 0; st < STAGES - 1 && st < nsteps; ++st) issue(st);
    }

    Real ring[K][YW];
#pragma unroll
    for (int t = 0; t < K; ++t)
#pragma unroll
        for (int r = 0; r < YW; ++r) ring[t][r] = Real(0);

    for (int step = 0; step < nsteps; ++step) {
        // refill the slot freed by the previous step (all threads are past its reads)
        if (tid == 0 && step + STAGES - 1 < nsteps) issue(step + STAGES - 1);
        const int s = step % STAGES;
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((step / STAGES) & 1), kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && a.err) atomicOr(a.err, kErrTmaTimeout);
            return;
        }
        Real* slot = reinterpret_cast<Real*>(base + s * G::SLOT_STRIDE);  // [NC][H][WB]
        if (edge) {
            // replicate boundary: columns first (within every row), then rows
            for (int q = tid; q < NC * H * WB; q += NT) {
                const int hx = q % WB;
                const int gx = bx + hx;
                if (gx < 0 || gx >= g.nx) {
                    const int src = clampi(gx, 0, g.nx - 1) - bx;  // in-volume column
                    slot[q] = slot[q - hx + src];
                }
            }
            __syncthreads();
            for (int q = tid; q < NC * H * WB; q += NT) {
                const int hx = q % WB;
                const int r = q / WB;
                const int hy = r % H;
                const int gy = by + hy;
                if (gy < 0 || gy >= g.ny) {
                    const int src = clampi(gy, 0, g.ny - 1) - by;
                    slot[q] = slot[(r - hy + src) * WB + hx];
                }
            }
            __syncthreads();
        }
        // x pass: task = (component, row, group of 4 outputs)
        for (int tk = tid; tk < NC * H * (STX / 4); tk += NT) {
            const int gq = tk % (STX / 4);
            const int row = tk / (STX / 4);  // c * H + r
            const Real* src = slot + row * WB + 4 * gq;  // 16-byte aligned
            Real in[G::XLV];
#pragma unroll
            for (int v = 0; v < G::XLV / VN; ++v) unpack(reinterpret_cast<const V*>(src)[v], in + v * VN);
            Real o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                Real acc = Real(0);
#pragma unroll
                for (int t = 0; t < K; ++t) acc += w[t] * in[HA - R + j + t];
                o[j] = acc;
            }
            store4(txp + row * STX + 4 * gq, o);
        }
        __syncthreads();
        // y pass: 4 rows of one column of one component, into the register ring
        {
            const Real* col = txp + (c_own * H + q_own * YW) * STX + lx;
            Real in[YW + 2 * R];
#pragma unroll
            for (int k = 0; k < YW + 2 * R; ++k) in[k] = col[k * STX];
#pragma unroll
            for (int t = 0; t < K - 1; ++t)
#pragma unroll
                for (int r = 0; r < YW; ++r) ring[t][r] = ring[t + 1][r];
#pragma unroll
            for (int r = 0; r < YW; ++r) {
                Real acc = Real(0);
#pragma unroll
                for (int t = 0; t < K; ++t) acc += w[t] * in[r + t];
                ring[K - 1][r] = acc;
            }
        }
        // z pass for plane z0 + step - 2R
        if (step >= 2 * R && x < g.nx) {
            const int zo = z0 + step - 2 * R;
#pragma unroll
            for (int r = 0; r < YW; ++r) {
                const int y = y0 + q_own * YW + r;
                if (y < g.ny) {
                    Real acc = Real(0);
#pragma unroll
                    for (int t = 0; t < K; ++t) acc += w[t] * ring[t][r];
                    out[offs(g, x, y, zo) + c_own * g.cs] = acc;
                }
            }
        }
        // no barrier here: the next step's __syncthreads_or orders these reads of
        // txp before its x pass rewrites them
    }
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

template <typename Real, int R, int NC>
static cudaError_t launch_rn(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    using G = SmoothGeom<Real, R, NC>;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // 4-D view: (x, y, z, component), strides in bytes
    const cuuint64_t dims[4] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny, (cuuint64_t)a.g.nz,
                                (cuuint64_t)NC};
    const cuuint64_t strides[3] = {(cuuint64_t)a.g.px * sizeof(Real),
                                   (cuuint64_t)a.g.plane * sizeof(Real),
                                   (cuuint64_t)a.g.cs * sizeof(Real)};
    const cuuint32_t box[4] = {(cuuint32_t)G::WB, (cuuint32_t)G::H, 1u, (cuuint32_t)NC};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    CUtensorMap map;
    const CUresult r = enc(&map, sizeof(Real) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                           4, const_cast<void*>(a.in), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(smooth_kernel<Real, R, NC>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   G::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    // z chunk: about one wave of resident blocks; small volumes use short
    // chunks (down to 1 plane) so that enough blocks run
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smooth_kernel<Real, R, NC>, G::NT,
                                                  G::SMEM);
    if (per_sm < 1) per_sm = 1;
    const long long bxy = (long long)((a.g.nx + STX - 1) / STX) * ((a.g.ny + STY - 1) / STY);
    const long long target = (long long)per_sm * num_sms;
    long long chunks = (target + bxy - 1) / bxy;
    if (chunks < 1) chunks = 1;
    int zc = (int)((a.g.nz + chunks - 1) / chunks);
    if (zc < 1) zc = 1;
    const dim3 grid((a.g.nx + STX - 1) / STX, (a.g.ny + STY - 1) / STY, (a.g.nz + zc - 1) / zc);
    smooth_kernel<Real, R, NC><<<grid, dim3(G::NT, 1, 1), G::SMEM, s>>>(map, a, zc);
    return cudaGetLastError();
}

template <typename Real, int R>
static cudaError_t launch_r(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    return a.ncomp == 3 ? launch_rn<Real, R, 3>(a, num_sms, s) : launch_rn<Real, R, 1>(a, num_sms, s);
}

template <typename Real>
static cudaError_t launch_t(const SmoothArgs& a, int num_sms, cudaStream_t s) {
    switch (a.taps.R) {
        case 1: return launch_r<Real, 1>(a, num_sms, s);
        case 2: return launch_r<Real, 2>(a, num_sms, s);
        case 3: return launch_r<Real, 3>(a, num_sms, s);
        case 4: return launch_r<Real, 4>(a, num_sms, s);
        case 5: return launch_r<Real, 5>(a, num_sms, s);
        case 6: return launch_r<Real, 6>(a, num_sms, s);
        case 7: return launch_r<Real, 7>(a, num_sms, s);
        case 8: return launch_r<Real, 8>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_smooth(bool fp64, const SmoothArgs& a, int num_sms, cudaStream_t s) {
    if (a.ncomp != 1 && a.ncomp != 3) return cudaErrorInvalidValue;
    return fp64 ? launch_t<double>(a, num_sms, s) : launch_t<float>(a, num_sms, s);
}

}  // namespace dirk
