// dir_stencil.cuh -- the separable Gaussian's building blocks (Sec. 2.5 low-pass
// filter), shared by the smoothing kernel and the fused iteration kernel.
//
// A block owns a 32 x 8 (x, y) column tile and marches through a chunk of z
// planes.  Each input plane's tile plus halo arrives by TMA
// (cp.async.bulk.tensor, all components in one copy) into a 4-slot ring of
// shared memory several planes ahead; out-of-volume halo cells (zero-filled by
// the copy) are overwritten with the nearest edge voxel (replicate boundary);
// the x pass filters 4 adjacent outputs per task from 128-bit shared loads;
// the y pass filters 4 rows of one column of one component per thread into a
// rolling register window of 2R+1 planes, from which the z pass is taken.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <type_traits>

#include "dir_common.cuh"
#include "dir_launch.h"

namespace dirk {

constexpr int STX = 32, STY = 8, YW = 4;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

// Vector loads of the staged rows: 16 bytes for 4- and 8-byte elements, 8
// bytes for 2-byte elements (their task offsets are only 8-byte aligned).
template <typename T>
struct VecLd;
template <>
struct VecLd<float> {
    using V = float4;
    static constexpr int N = 4;
};
template <>
struct VecLd<double> {
    using V = double2;
    static constexpr int N = 2;
};
template <>
struct VecLd<int16_t> {
    using V = uint2;
    static constexpr int N = 4;
};
template <>
struct VecLd<bf16> {
    using V = uint2;
    static constexpr int N = 4;
};

template <typename Real>
__device__ __forceinline__ void unpack(const float4& t, Real* d) {
    d[0] = t.x;
    d[1] = t.y;
    d[2] = t.z;
    d[3] = t.w;
}
template <typename Real>
__device__ __forceinline__ void unpack(const double2& t, Real* d) {
    d[0] = t.x;
    d[1] = t.y;
}
template <typename T, typename Real>
__device__ __forceinline__ void unpack16(const uint2& t, Real* d) {
    const uint32_t w[2] = {t.x, t.y};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned short h = (unsigned short)(w[k >> 1] >> (16 * (k & 1)));
        if constexpr (sizeof(T) == 2 && std::is_same<T, int16_t>::value) {
            d[k] = (Real)(short)h;
        } else {
            d[k] = (Real)__bfloat162float(__ushort_as_bfloat16(h));
        }
    }
}
__device__ __forceinline__ void store4(float* dst, const float* s) {
    *reinterpret_cast<float4*>(dst) = make_float4(s[0], s[1], s[2], s[3]);
}
__device__ __forceinline__ void store4(double* dst, const double* s) {
    reinterpret_cast<double2*>(dst)[0] = make_double2(s[0], s[1]);
    reinterpret_cast<double2*>(dst)[1] = make_double2(s[2], s[3]);
}

template <typename Real, int R, int NC, int STAGES_ = 4, typename TIN = Real>
struct StencilGeom {
    static constexpr int STAGES = STAGES_;
    static constexpr int ALIGN = 16 / (int)sizeof(TIN);      // elements per 16 bytes
    static constexpr int HA = (R + ALIGN - 1) / ALIGN * ALIGN;  // x halo: TMA x start 16-byte aligned
    static constexpr int WB = STX + 2 * HA;      // box width
    static constexpr int H = STY + 2 * R;        // box height
    static constexpr int K = 2 * R + 1;
    static constexpr int YT = STX * NC * (STY / YW);  // y/z tasks: (x, component, row group)
    static constexpr int XL = 4 + 2 * R;              // inputs of one 4-output x task
    static constexpr int VN = VecLd<TIN>::N;
    static constexpr int XLV = (HA - R + XL + VN - 1) / VN * VN;  // loaded span, whole vectors
    static constexpr int SLOT_ELEMS = NC * H * WB;
    static constexpr int SLOT_BYTES = SLOT_ELEMS * (int)sizeof(TIN);
    static constexpr int SLOT_STRIDE = (SLOT_BYTES + 127) / 128 * 128;
    static constexpr int TXP_BYTES = NC * H * STX * (int)sizeof(Real);
    static constexpr int TXP_STRIDE = (TXP_BYTES + 127) / 128 * 128;
    // dynamic shared memory: align slack, slots, x-pass rows, barriers, extra
    static constexpr int BASE_SMEM = 128 + STAGES * SLOT_STRIDE + TXP_STRIDE + 64;
};

// Per-block state of the TMA plane pipeline.
template <typename Real, int R, int NC, int STAGES_ = 4, typename TIN = Real>
struct PlanePipe {
    using G = StencilGeom<Real, R, NC, STAGES_, TIN>;
    static constexpr int STAGES = STAGES_;
    unsigned char* base;
    Real* txp;
    uint64_t* full;
    int z0, nsteps, bx, by;
    bool edge;

    int comp0;  // first component of the copies (tensor-map coordinate 3)

    __device__ void setup(unsigned char* smem_raw, const Grid3& g, int x0, int y0, int zstart,
                          int zend, int c0 = 0) {
        comp0 = c0;
        // 128-byte aligned by pointer arithmetic on the shared array, so that
        // the accesses stay in the shared address space
        base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
        txp = reinterpret_cast<Real*>(base + STAGES * G::SLOT_STRIDE);
        full = reinterpret_cast<uint64_t*>(base + STAGES * G::SLOT_STRIDE + G::TXP_STRIDE);
        z0 = zstart;
        nsteps = (zend - zstart) + 2 * R;  // input planes z0-R .. z1-1+R (clamped)
        bx = x0 - G::HA;
        by = y0 - R;
        edge = (bx < 0) || (bx + G::WB > g.nx) || (by < 0) || (by + G::H > g.ny);
    }
    __device__ unsigned char* extra() const {
        return base + STAGES * G::SLOT_STRIDE + G::TXP_STRIDE + 64;
    }
    __device__ void issue(const CUtensorMap* map, const Grid3& g, int step) {
        const int s = step % STAGES;
        const int pc = clampi(z0 - R + step, 0, g.nz - 1);
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[s], (uint32_t)G::SLOT_BYTES);
        tma_load_4d(base + s * G::SLOT_STRIDE, map, bx, by, pc, comp0, &full[s]);
    }
    // thread 0: init barriers and prefetch; everyone: barrier
    __device__ void start(const CUtensorMap* map, const Grid3& g, int tid) {
        if (tid == 0) {
            for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
            fence_mbar_init();
            fence_proxy_async();
            for (int st = 0; st < STAGES - 1 && st < nsteps; ++st) issue(map, g, st);
        }
        __syncthreads();
    }
    // Step `step`: refill, wait for the slot (bounded), fix edges, x pass.
    // Returns false (for every thread) if the copy never arrived.
    template <int NT>
    __device__ bool xpass(const CUtensorMap* map, const Grid3& g, int step, int tid,
                          const Real* w, int* err) {
        if (tid == 0 && step + STAGES - 1 < nsteps) issue(map, g, step + STAGES - 1);
        const int s = step % STAGES;
        const uint32_t parity = (uint32_t)((step / STAGES) & 1);
        // one thread spins (bounded); after the barrier every thread observes
        // the completed phase once, which makes the copied bytes visible to it
        bool ok = true;
        if (tid == 0) ok = mbar_wait_bounded(&full[s], parity, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && err) atomicOr(err, kErrTmaTimeout);
            return false;
        }
        (void)mbar_try_wait(&full[s], parity);
        constexpr int HA = G::HA, WB = G::WB, H = G::H, K = G::K;
        using V = typename VecLd<TIN>::V;
        constexpr int VN = VecLd<TIN>::N;
        TIN* slot = reinterpret_cast<TIN*>(base + s * G::SLOT_STRIDE);  // [NC][H][WB]
        if (edge) {
            // replicate boundary: out-of-volume columns first (a thread per
            // row), then out-of-volume rows (a thread per column, rows already
            // column-fixed)
            const int lo = max(0, -bx);         // first in-volume column of the box
            const int hi = min(WB, g.nx - bx);  // one past the last
            for (int row = tid; row < NC * H; row += NT) {
                TIN* r = slot + row * WB;
                const TIN left = r[lo], right = r[hi - 1];
                for (int hx = 0; hx < lo; ++hx) r[hx] = left;
                for (int hx = hi; hx < WB; ++hx) r[hx] = right;
            }
            __syncthreads();
            const int rlo = max(0, -by);
            const int rhi = min(H, g.ny - by);
            for (int col = tid; col < NC * WB; col += NT) {
                TIN* cbase = slot + (col / WB) * H * WB + (col % WB);
                const TIN top = cbase[rlo * WB], bot = cbase[(rhi - 1) * WB];
                for (int hy = 0; hy < rlo; ++hy) cbase[hy * WB] = top;
                for (int hy = rhi; hy < H; ++hy) cbase[hy * WB] = bot;
            }
            __syncthreads();
        }
        for (int tk = tid; tk < NC * H * (STX / 4); tk += NT) {
            const int gq = tk % (STX / 4);
            const int row = tk / (STX / 4);  // c * H + r
            const TIN* src = slot + row * WB + 4 * gq;  // vector aligned
            Real in[G::XLV];
#pragma unroll
            for (int v = 0; v < G::XLV / VN; ++v) {
                if constexpr (sizeof(TIN) == 2)
                    unpack16<TIN, Real>(reinterpret_cast<const V*>(src)[v], in + v * VN);
                else
                    unpack<Real>(reinterpret_cast<const V*>(src)[v], in + v * VN);
            }
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
        return true;
    }
    // y pass of rows q*YW .. q*YW+YW-1 of column lx, component c, into the ring
    __device__ void ypass(int c, int q, int lx, const Real* w, Real (&ring)[G::K][YW]) const {
        constexpr int H = G::H, K = G::K;
        const Real* col = txp + (c * H + q * YW) * STX + lx;
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
};

template <typename Real, int R>
__device__ __forceinline__ Real zpass(const Real* w, const Real (&ring)[2 * R + 1][YW], int r) {
    Real acc = Real(0);
#pragma unroll
    for (int t = 0; t < 2 * R + 1; ++t) acc += w[t] * ring[t][r];
    return acc;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
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

// One-time set-up of a kernel on each device: the opt-in to more than 48 KB of
// dynamic shared memory (cudaFuncSetAttribute acts on the function for the
// current device only) and, if asked, its resident blocks per SM.  One
// KernelSetup per kernel instantiation; safe to call from several host
// threads and devices.
struct KernelSetup {
    static constexpr int kMaxDevices = 64;
    std::atomic<unsigned long long> done{0};  // bit d: set up on device d
    int per_sm[kMaxDevices] = {};
};

inline std::mutex& kernel_setup_mutex() {
    static std::mutex m;
    return m;
}

template <typename Fn>
inline cudaError_t setup_kernel(KernelSetup& st, Fn* fn, int smem, int threads = 0,
                                int* per_sm_out = nullptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= KernelSetup::kMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long bit = 1ull << dev;
    if (!(st.done.load(std::memory_order_acquire) & bit)) {
        std::lock_guard<std::mutex> lock(kernel_setup_mutex());
        if (!(st.done.load(std::memory_order_relaxed) & bit)) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            int n = 1;
            if (threads > 0) {
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem);
                if (e != cudaSuccess) return e;
            }
            st.per_sm[dev] = n < 1 ? 1 : n;
            st.done.fetch_or(bit, std::memory_order_release);
        }
    }
    if (per_sm_out) *per_sm_out = st.per_sm[dev];
    return cudaSuccess;
}

// Tensor map of a pitched (x, y, z, component) array of ncomp components with
// the plane box of StencilGeom<Real, R, NC> (NC components per copy).
// Returns false if the driver refuses it.
// Launch a kernel; with pdl, as a programmatic dependent launch (it may start
// while the kernel before it in the stream still runs; see pdl_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex(void (*fn)(KArgs...), dim3 grid, dim3 block, int smem,
                             cudaStream_t s, bool pdl, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, fn, static_cast<Args&&>(args)...);
}

template <typename T>
inline CUtensorMapDataType tma_type();
template <>
inline CUtensorMapDataType tma_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <>
inline CUtensorMapDataType tma_type<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
template <>
inline CUtensorMapDataType tma_type<int16_t>() { return CU_TENSOR_MAP_DATA_TYPE_UINT16; }  // bit copy
template <>
inline CUtensorMapDataType tma_type<bf16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }

template <typename Real, int R, int NC, typename TIN = Real>
inline bool make_plane_map(CUtensorMap* map, const void* ptr, const Grid3& g, int ncomp) {
    using G = StencilGeom<Real, R, NC, 4, TIN>;  // the box does not depend on the stage count
    using Real_ = TIN;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz,
                                (cuuint64_t)ncomp};
    const cuuint64_t strides[3] = {(cuuint64_t)g.px * sizeof(Real_),
                                   (cuuint64_t)g.plane * sizeof(Real_),
                                   (cuuint64_t)g.cs * sizeof(Real_)};
    const cuuint32_t box[4] = {(cuuint32_t)G::WB, (cuuint32_t)G::H, 1u, (cuuint32_t)NC};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    return enc(map, tma_type<TIN>(),
               4, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// z chunk: as many chunks as fit in one wave of resident blocks (a partial
// second wave would leave most SMs idle while it runs); short chunks (down to
// one plane) for small volumes so that enough blocks run
inline int stencil_zchunk(const Grid3& g, int blocks_per_sm, int num_sms, int copies = 1) {
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    const long long bxy =
        (long long)((g.nx + STX - 1) / STX) * ((g.ny + STY - 1) / STY) * copies;
    const long long wave = (long long)blocks_per_sm * num_sms;
    long long chunks = wave / bxy;
    if (chunks < 1) chunks = 1;
    if (chunks > g.nz) chunks = g.nz;
    const int zc = (int)((g.nz + chunks - 1) / chunks);
    return zc < 1 ? 1 : zc;
}

}  // namespace dirk
