// dir_engine.cu -- registration engine and C ABI of libdir.so (see include/dir.h).
//
// The engine owns every device buffer of a context and issues the whole
// registration as one stream-ordered sequence:
//   pyramid build (Gaussian + decimation, Sec. 2.3)
//   for each level, coarsest first:
//     field init (zero / init_field) or up-sampling of the coarser field (Sec. 2.3)
//     per iteration: fused force kernel (u -> v), Gaussian smoothing (v -> u),
//                    optional relative-norm stop test (Sec. 2.4)
//   inverse-consistent output field (Eq. 6) when that variant runs.
// With use_graph the sequence is captured once into a CUDA graph and replayed
// by later registrations, so the hundreds of small coarse-level launches cost
// one graph launch.  A device-side stop flag per level lets the captured graph
// skip the remaining iterations of a level without a host round trip.
// Images and fields live on the device as float (DIR_F32) or double (DIR_F64).
// Single precision runs the TMA-tiled production kernels, or with
// plain_kernels the plain-load kernels; double precision runs the plain-load
// kernels in double.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "dir.h"
#include "dir_common.cuh"
#include "dir_launch.h"

using dirk::Grid3;

namespace {

constexpr int kIcInvertSteps = 20;
constexpr int kStopUnset = 0x7f7f7f7f;  // memset byte 0x7f

thread_local std::string g_create_error;

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

Grid3 make_grid(int nx, int ny, int nz) {
    Grid3 g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.px = (int)round_up(nx, 32);
    g.plane = (long long)g.px * ny;
    g.cs = round_up(g.plane * nz, 64);
    return g;
}

bool make_taps(double sigma, dirk::Taps* t) {
    if (!(sigma > 0.0) || !isfinite(sigma)) return false;
    const int R = (int)ceil(3.0 * sigma);
    if (R < 1 || R > dirk::kMaxRadius) return false;
    double w[2 * dirk::kMaxRadius + 1];
    double sum = 0.0;
    for (int k = -R; k <= R; ++k) {
        w[k + R] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        sum += w[k + R];
    }
    t->R = R;
    for (int k = 0; k < 17; ++k) {
        t->w[k] = 0.0;
        t->wf[k] = 0.0f;
    }
    for (int k = 0; k < 2 * R + 1; ++k) t->w[k] = w[k] / sum;
    // Single-precision taps: rounding each tap alone leaves their sum off 1 by
    // a few 1e-8, and every smoothing pass would scale the field by that sum
    // (3 passes x hundreds of iterations).  Keep the taps symmetric, then move
    // mirrored pairs (outermost first, finest steps) and finally the centre
    // tap by one float step at a time while that brings the exact sum closer
    // to 1.
    for (int k = 0; k < 2 * R + 1; ++k) t->wf[k] = (float)t->w[k];
    auto err = [&]() {
        double s = 0.0;
        for (int k = 0; k < 2 * R + 1; ++k) s += (double)t->wf[k];
        return s - 1.0;
    };
    for (int pass = 0; pass < 4; ++pass) {
        for (int k = 0; k <= R; ++k) {
            const bool centre = (k == R);
            for (int step = 0; step < 64; ++step) {
                const double e0 = err();
                if (e0 == 0.0) break;
                const float cur = t->wf[k];
                const float nxt = nextafterf(cur, e0 > 0.0 ? 0.0f : 1.0f);
                const double delta = ((double)nxt - (double)cur) * (centre ? 1.0 : 2.0);
                if (fabs(e0 + delta) >= fabs(e0)) break;
                t->wf[k] = nxt;
                t->wf[2 * R - k] = nxt;
            }
        }
    }
    return true;
}

}  // namespace

struct LevelBuf {
    Grid3 g;
    char* S;
    char* M;
};

struct dir_ctx {
    int dims[3];
    float spacing[3];
    int variant;
    dir_params p;
    bool fp64;
    size_t esz;          // arithmetic type (float or double) = coarse image storage
    int real_type;       // kStoreF32 or kStoreF64
    int img0_type;       // storage of the finest-level images (kStoreI16 for int16 HU input)
    size_t iesz0;        // its element size
    int field_type;      // storage of the fields (kStoreF32, kStoreBF16, kStoreF64)
    size_t fesz;         // its element size
    int input_dtype;     // dir_dtype of the images the caller passes (DIR_F32 or DIR_I16)

    int img_type(int l) const { return l == 0 ? img0_type : real_type; }
    size_t img_esz(int l) const { return l == 0 ? iesz0 : esz; }
    cudaStream_t stream;
    int device;
    int num_sms;
    int levels;
    LevelBuf lv[DIR_MAX_LEVELS];
    char* img_pool = nullptr;
    char* A = nullptr;
    char* B = nullptr;
    char* C = nullptr;     // Eqs. 3-6 split with the difference image: u and D of a level
    size_t C_bytes = 0;
    double* red = nullptr;
    double* corr = nullptr;   // 4 sums per iteration of the correlation coefficient, or null
    double* lhist = nullptr;
    int* ctl = nullptr;
    int* derr = nullptr;
    int total_iters = 0;
    int level_first[DIR_MAX_LEVELS];
    int fused_level[DIR_MAX_LEVELS];
    int tune_depth[DIR_MAX_LEVELS] = {0};    // force brick depth per level, 0 = heuristic
    int tune_zchunk[DIR_MAX_LEVELS] = {0};   // smoothing z chunk per level (of the x/y kernel
                                             // on split levels), 0 = the launcher's choice
    char* final_field = nullptr;
    bool have_field = false;
    bool pending = false;
    char* stage_img = nullptr;      // pitched, element type of the context
    float* stage_f32 = nullptr;     // dense float, 3*N
    double* stage_f64 = nullptr;    // dense double, 3*N
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> tev;  // 3 per timed iteration: before force, between, after smooth
    int n_timed = 0;
    int launches = 0;
    dirk::Taps taps, taps1;
    std::vector<double> red_host;
    std::vector<double> corr_host;
    std::vector<int> ctl_host;
    int iters_run[DIR_MAX_LEVELS];
    std::string err;

    size_t nvox() const { return (size_t)dims[0] * dims[1] * dims[2]; }
};

static void set_err(dir_ctx* c, const char* what, cudaError_t e) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
}

#define CK(ctx, call)                       \
    do {                                    \
        cudaError_t e_ = (call);            \
        if (e_ != cudaSuccess) {            \
            set_err((ctx), #call, e_);      \
            return DIR_ECUDA;               \
        }                                   \
    } while (0)

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// context's stream): freeing a finished context does not synchronise the
// device, so other contexts keep running (the serving loop relies on it).
static int ensure(dir_ctx* c, void** p, size_t bytes) {
    if (*p) return DIR_OK;
    if (cudaMallocAsync(p, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        c->err = "device allocation failed";
        return DIR_ENOMEM;
    }
    return DIR_OK;
}

// Dense volume(s) (host or device) of element size src_esz (4 = float,
// 2 = int16) -> pitched volume(s) of storage type dst_type.  Same element type:
// a 2-D copy (exact); float -> bf16 / double: through the import kernel.
static int import_dense(dir_ctx* c, const void* src, int on_device, int src_esz, char* dst,
                        int dst_type, const Grid3& g, int ncomp, cudaStream_t s) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t dst_esz = dst_type == dirk::kStoreF64 ? 8 : (dst_type == dirk::kStoreF32 ? 4 : 2);
    const bool same = (src_esz == 4 && dst_type == dirk::kStoreF32) ||
                      (src_esz == 2 && dst_type == dirk::kStoreI16);
    if (same) {
        const size_t w = (size_t)g.nx * src_esz;
        for (int comp = 0; comp < ncomp; ++comp)
            CK(c, cudaMemcpy2DAsync(dst + comp * g.cs * dst_esz, (size_t)g.px * dst_esz,
                                    static_cast<const char*>(src) + comp * n * src_esz, w, w,
                                    (size_t)g.ny * g.nz,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    s));
        return DIR_OK;
    }
    if (src_esz != 4) return DIR_EUNSUPPORTED;
    const float* dsrc = static_cast<const float*>(src);
    if (!on_device) {
        const int rc = ensure(c, (void**)&c->stage_f32, 3 * n * sizeof(float));
        if (rc != DIR_OK) return rc;
        CK(c, cudaMemcpyAsync(c->stage_f32, src, ncomp * n * sizeof(float), cudaMemcpyHostToDevice,
                              s));
        dsrc = c->stage_f32;
    }
    CK(c, dirk::launch_import(dst_type == dirk::kStoreF64, dst_type, dsrc, dst, g, ncomp, s));
    return DIR_OK;
}

static int upload_pair(dir_ctx* c, const void* S, const void* M, int on_device, cudaStream_t s) {
    const int se = c->input_dtype == DIR_I16 ? 2 : 4;
    int rc = import_dense(c, S, on_device, se, c->lv[0].S, c->img0_type, c->lv[0].g, 1, s);
    if (rc == DIR_OK)
        rc = import_dense(c, M, on_device, se, c->lv[0].M, c->img0_type, c->lv[0].g, 1, s);
    return rc;
}

static int record(dir_ctx* c, cudaEvent_t e, cudaStream_t s, bool capturing) {
    CK(c, capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                    : cudaEventRecord(e, s));
    return DIR_OK;
}

// Issues the whole registration on stream s (captured or direct).
// Programmatic dependent launch of a level's iteration kernels, above 2^18
// voxels: a kernel's blocks set up and copy the static images while the one
// before drains its last wave (they start only once all its blocks have).
// Measured per level on the 256x256x100 pyramid: 128x128x50 passive 17.96 ->
// 16.7 us per iteration, 256x256x100 94.15 -> 93.48 us (Eq. 2: 103.8 ->
// 102.0), but the 64x64x25 level slower (7.19 -> 7.28 us; Eq. 6 18.1 -> 19.7).
// Not with a stop test (the kernels read the stop flag before they wait), nor
// with timing events between the kernels.  Split schedule only: the same
// launches made the force + smoothing kernels slower (Eq. 3: 13.20 -> 13.35 ms
// per registration, Eq. 6: 17.07 -> 17.27; split passive 8.20 -> 8.04).
static bool level_pdl(const dir_ctx* c, const Grid3& g, bool timed) {
    return c->p.pdl && c->p.stop_mode == 0 && !timed && !c->fp64 && !c->p.plain_kernels &&
           (long long)g.nx * g.ny * g.nz > (1LL << 18);
}

// The split kernels: FP32 field, float or int16 images, radius 3
static bool level_split_ok(const dir_ctx* c, int l) {
    return !c->fp64 && !c->p.plain_kernels && c->field_type == dirk::kStoreF32 &&
           (c->img_type(l) == dirk::kStoreF32 || c->img_type(l) == dirk::kStoreI16) &&
           c->taps.R == 3;
}

// Schedule 3, Eqs. 3-6 only: the split iteration with the difference image
// formed once per voxel (x/y kernel, z + D kernel, stencil force kernel), on
// every level with fuse = 2 or 4.  Measured per iteration on the 256x256x100
// pyramid against the one-pass z + force kernel (schedule 2) and, on the
// finest level, the force + smoothing kernels (schedule 0), active: 125.4 us
// against 169.7 and 148.6 on the finest level, 21.7 against 27.8 on
// 128x128x50, 10.2 against 10.5 on 64x64x25; Eq. 6: 170.8 against 229.1 and
// 207.8, 36.6 against 45.4, 16.8 against 17.8.  It needs the u + D scratch
// (dir_ctx::C), allocated for the levels that run it; without one
// (dir_register_noalloc) a level runs what the rules below give.
static bool level_wants_d(const dir_ctx* c, int l) {
    if (c->variant < 2 || !level_split_ok(c, l)) return false;
    return c->p.fuse == 2 || c->p.fuse == 4;
}

// The z + D kernel runs at most 4 deep: at 8 its 64 registers and 43 KB of
// shared memory leave four blocks per SM and its gathers' latency shows (ncu,
// 256x256x100, Eq. 3: 53.9 us against 50.9 us at 4), while the stencil force
// kernel gains from 8 (38.3 us against 42.3 us)
constexpr int kZdMaxDepth = 4;

static size_t level_d_bytes(const dir_ctx* c, int l) {
    return (size_t)dirk::force_d_planes(c->variant) * (size_t)c->lv[l].g.cs * sizeof(float);
}

// Iteration schedule of pyramid level l: 0 force + smoothing kernels, 1 fused
// iteration (the Gaussian of v_{k-1} folded into the force pass), 2 split
// Gaussian (its x and y passes as their own kernel, its z pass inside the
// force kernel), 3 split with the difference image (above).  All four give the
// same field bit for bit.  fuse = 2 (the default) takes the split schedule
// where it applies for Eqs. 1-2 on every level and for Eqs. 3-6 on the small
// levels (there in form 3), otherwise the fused one on the small levels:
// measured per level on the 256x256x100 pyramid.
static int level_schedule(const dir_ctx* c, int l) {
    if (c->fp64 || c->p.plain_kernels) return 0;
    const Grid3& g = c->lv[l].g;
    const bool split_ok = level_split_ok(c, l);
    if (level_wants_d(c, l) && c->C && c->C_bytes >= level_d_bytes(c, l)) return 3;
    const bool eqs12 = c->variant == 0 || c->variant == 1;
    const bool fused_ok = c->p.stop_mode == 0 && dirk::fused_supported(c->variant) &&
                          c->field_type == c->real_type && c->img_type(l) == c->real_type;
    switch (c->p.fuse) {
        case 1: return fused_ok ? 1 : 0;
        case 2: {
            // (Eqs. 3-6 here only without the scratch of schedule 3.)  They
            // need u on the brick's one-voxel halo too, so their split kernel
            // runs the z pass on 34 x 10 columns of a deeper box: it pays on
            // levels of at most 2^21 voxels (the marching smoothing's z halo
            // costs more there) and not above (256x256x100, active: 137 us
            // against 98 + 54 - 37 us per finest iteration)
            const bool small = (long long)g.nx * g.ny * g.nz <= (1LL << 21);
            if (split_ok && (eqs12 || small)) return 2;
            return fused_ok && dirk::fused_small_level(g, c->num_sms) ? 1 : 0;
        }
        case 3:
        case 4: return split_ok ? 2 : 0;
        default: return 0;
    }
}

// The start of every registration: the reduction rows, stop flags and error
// word cleared, and the pyramid (Sec. 2.3: level l+1 = unit-sigma Gaussian of
// level l at even indices).
static int enqueue_prologue(dir_ctx* c, cudaStream_t s) {
    c->launches = 0;
    const int L = c->levels;
    const bool f64 = c->fp64;
    const bool plain = c->p.plain_kernels != 0;
    CK(c, cudaMemsetAsync(c->red, 0, sizeof(double) * 3 * (size_t)(c->total_iters > 0 ? c->total_iters : 1), s));
    if (c->corr)
        CK(c, cudaMemsetAsync(c->corr, 0,
                              sizeof(double) * 4 * (size_t)(c->total_iters > 0 ? c->total_iters : 1),
                              s));
    CK(c, cudaMemsetAsync(c->ctl, 0x7f, sizeof(int) * (size_t)L, s));
    CK(c, cudaMemsetAsync(c->derr, 0, sizeof(int), s));
    for (int l = 1; l < L; ++l) {
        const Grid3& gf = c->lv[l - 1].g;
        const Grid3& gc = c->lv[l].g;
        for (int img = 0; img < 2; ++img) {
            dirk::SmoothArgs sa;
            sa.in = img ? c->lv[l - 1].M : c->lv[l - 1].S;
            sa.out = c->B;
            sa.g = gf;
            sa.ncomp = 1;
            sa.taps = c->taps1;
            sa.stop_iter = nullptr;
            sa.iter = 0;
            sa.err = c->derr;
            sa.in_type = c->img_type(l - 1);
            sa.out_type = c->real_type;
            sa.zchunk = 0;
            CK(c, dirk::launch_smooth(f64, sa, c->num_sms, s, plain));
            CK(c, dirk::launch_decimate(f64, c->B, gf, img ? c->lv[l].M : c->lv[l].S, gc, s));
            c->launches += 2;
        }
    }
    return DIR_OK;
}

// The field at the start of level lc (coarsest first): the initial field or
// zero on the coarsest level, else the upsampled field of the level before;
// cur holds it afterwards, oth is free.
static int enqueue_level_start(dir_ctx* c, int lc, char*& cur, char*& oth, cudaStream_t s) {
    const int l = c->levels - 1 - lc;
    const Grid3& g = c->lv[l].g;
    if (lc == 0) {
        if (c->p.init_field) {
            const int rc = import_dense(c, c->p.init_field, 1, 4, cur, c->field_type, g, 3, s);
            if (rc != DIR_OK) return rc;
            if (c->field_type != dirk::kStoreF32) c->launches += 1;
        } else {
            CK(c, cudaMemsetAsync(cur, 0, c->fesz * 3 * (size_t)g.cs, s));
        }
    } else {
        CK(c, dirk::launch_upsample(c->fp64, c->field_type, cur, c->lv[l + 1].g, oth, g, s));
        c->launches += 1;
        char* t = cur;
        cur = oth;
        oth = t;
    }
    return DIR_OK;
}

// Force and smoothing arguments of level lc (buffers, rows and iteration set
// by the caller)
static dirk::ForceArgs level_force_args(const dir_ctx* c, int lc) {
    const int l = c->levels - 1 - lc;
    const Grid3& g = c->lv[l].g;
    dirk::ForceArgs fa;
    fa.S = c->lv[l].S;
    fa.M = c->lv[l].M;
    fa.g = g;
    fa.alpha2 = c->p.alpha * c->p.alpha;
    fa.stop_iter = c->ctl + lc;
    fa.depth = c->tune_depth[l] ? c->tune_depth[l] : dirk::force_brick_depth(g, c->num_sms);
    // L2 prefetch of the bricks of the block one block per SM ahead (a
    // quarter of a wave of four blocks per SM; measured on 256x256x100
    // against 2, 3, 4, 6 and 8 blocks per SM ahead and none)
    fa.pf_stride = c->num_sms;
    fa.err = c->derr;
    fa.img_type = c->img_type(l);
    fa.field_type = c->field_type;
    return fa;
}

static dirk::SmoothArgs level_smooth_args(const dir_ctx* c, int lc) {
    const int l = c->levels - 1 - lc;
    dirk::SmoothArgs sa;
    sa.g = c->lv[l].g;
    sa.ncomp = 3;
    sa.taps = c->taps;
    sa.stop_iter = c->ctl + lc;
    sa.err = c->derr;
    sa.in_type = c->field_type;
    sa.out_type = c->field_type;
    sa.zchunk = c->tune_zchunk[l];
    return sa;
}

// The end of every registration: the static-grid field of Eq. 6 for the
// inverse-consistent law, and where the result lives.
static int enqueue_epilogue(dir_ctx* c, char* cur, char* oth, cudaStream_t s) {
    if (c->variant == DIR_INVERSE_CONSISTENT) {
        CK(c, dirk::launch_ic_invert(c->fp64, c->field_type, cur, oth, c->lv[0].g, kIcInvertSteps, s));
        c->launches += 1;
        c->final_field = oth;
    } else {
        c->final_field = cur;
    }
    return DIR_OK;
}

static int enqueue_registration(dir_ctx* c, cudaStream_t s, bool capturing) {
    const int L = c->levels;
    const bool f64 = c->fp64;
    const bool plain = c->p.plain_kernels != 0;
    {
        const int rc = enqueue_prologue(c, s);
        if (rc != DIR_OK) return rc;
    }
    char* cur = c->A;
    char* oth = c->B;
    int row = 0;
    c->n_timed = 0;
    for (int lc = 0; lc < L; ++lc) {
        const int l = L - 1 - lc;
        const Grid3& g = c->lv[l].g;
        {
            const int rc = enqueue_level_start(c, lc, cur, oth, s);
            if (rc != DIR_OK) return rc;
        }
        c->level_first[lc] = row;
        dirk::ForceArgs fa = level_force_args(c, lc);
        dirk::SmoothArgs sa = level_smooth_args(c, lc);
        const bool timed = c->p.timing && l == 0;
        const int n = c->p.iters[lc];
        const int sched = level_schedule(c, l);
        if (sched == 1 && n > 0) {
            // iteration 0 from u, iterations 1..n-1 from the previous v with the
            // smoothing folded in, then one smoothing of the last v
            char* vbuf = oth;
            char* spare = cur;
            for (int it = 0; it < n; ++it, ++row) {
                cudaEvent_t* e = timed ? &c->tev[3 * (size_t)c->n_timed] : nullptr;
                if (timed && record(c, e[0], s, capturing) != DIR_OK) return DIR_ECUDA;
                if (it == 0) {
                    fa.u = cur;
                    fa.v = vbuf;
                    fa.red = c->red + 3 * (size_t)row;
                    fa.corr = c->corr ? c->corr + 4 * (size_t)row : nullptr;
                    fa.iter = it;
                    CK(c, dirk::launch_force(c->variant, f64, fa, s, plain));
                } else {
                    dirk::FusedArgs ua;
                    ua.S = c->lv[l].S;
                    ua.M = c->lv[l].M;
                    ua.vin = vbuf;
                    ua.v = spare;
                    ua.g = g;
                    ua.taps = c->taps;
                    ua.red = c->red + 3 * (size_t)row;
                    ua.stop_iter = c->ctl + lc;
                    ua.iter = it;
                    ua.err = c->derr;
                    ua.corr = c->corr ? c->corr + 4 * (size_t)row : nullptr;
                    CK(c, dirk::launch_fused(c->variant, f64, ua, c->num_sms, s));
                    char* t = vbuf;
                    vbuf = spare;
                    spare = t;
                }
                c->launches += 1;
                if (timed) {
                    if (record(c, e[1], s, capturing) != DIR_OK) return DIR_ECUDA;
                    if (it < n - 1 && record(c, e[2], s, capturing) != DIR_OK) return DIR_ECUDA;
                }
                if (it == n - 1) {
                    sa.in = vbuf;
                    sa.out = spare;
                    sa.iter = it;
                    CK(c, dirk::launch_smooth(f64, sa, c->num_sms, s, plain));
                    c->launches += 1;
                    if (timed && record(c, e[2], s, capturing) != DIR_OK) return DIR_ECUDA;
                    cur = spare;
                    oth = vbuf;
                }
                if (timed) c->n_timed += 1;
            }
            c->fused_level[lc] = 1;
            continue;
        }
        if ((sched == 2 || sched == 3) && n > 0) {
            // iteration 0 from u; iteration k > 0: t = G_y G_x v (xy kernel), then
            // v = u - dr(u) with u = G_z t (force kernel; schedule 3: the z + D
            // kernel writes u and D to the scratch, the stencil force kernel
            // reads them); then u = G v of the last iteration run
            char* vbuf = oth;
            char* tbuf = cur;
            dirk::SmoothArgs xa = sa;
            xa.in = vbuf;
            xa.out = tbuf;
            xa.zchunk = c->tune_zchunk[l];  // 0: the launcher's own chunking
            // brick depths: of the z + force kernel (tuned or its own rule), and
            // of the plain force pass of iteration 0
            const int zs_depth = c->tune_depth[l] ? c->tune_depth[l]
                                 : sched == 3 ? dirk::force_d_depth(g, c->num_sms)
                                              : dirk::force_zs_depth(c->variant, g, c->num_sms);
            const int first_depth = dirk::force_brick_depth(g, c->num_sms);
            const bool pdl = level_pdl(c, g, timed);
            for (int it = 0; it < n; ++it, ++row) {
                cudaEvent_t* e = timed ? &c->tev[3 * (size_t)c->n_timed] : nullptr;
                if (timed && record(c, e[0], s, capturing) != DIR_OK) return DIR_ECUDA;
                fa.red = c->red + 3 * (size_t)row;
                fa.corr = c->corr ? c->corr + 4 * (size_t)row : nullptr;
                fa.iter = it;
                fa.v = vbuf;
                if (it == 0) {
                    fa.u = cur;
                    fa.depth = first_depth;
                    CK(c, dirk::launch_force(c->variant, f64, fa, s, plain));
                    c->launches += 1;
                    if (timed && record(c, e[1], s, capturing) != DIR_OK) return DIR_ECUDA;
                } else {
                    xa.iter = it;
                    xa.pdl = pdl;
                    CK(c, dirk::launch_smooth_xy(xa, c->num_sms, s));
                    if (timed && record(c, e[1], s, capturing) != DIR_OK) return DIR_ECUDA;
                    fa.depth = zs_depth;
                    fa.pdl = pdl;
                    if (sched == 3) {
                        dirk::ForceArgs za = fa, ta = fa;
                        char* dpl = c->C + 3 * (size_t)g.cs * sizeof(float);
                        za.depth = std::min(zs_depth, kZdMaxDepth);
                        za.u = tbuf;
                        za.v = c->C;
                        za.dbuf = ta.dbuf = dpl;
                        za.dbuf2 = ta.dbuf2 =
                            c->variant == DIR_INVERSE_CONSISTENT ? dpl + (size_t)g.cs * sizeof(float)
                                                                 : nullptr;
                        ta.u = c->C;
                        CK(c, dirk::launch_force_d(c->variant, za, ta, c->taps, s));
                        c->launches += 3;
                    } else {
                        fa.u = tbuf;
                        CK(c, dirk::launch_force_zs(c->variant, fa, c->taps, s));
                        c->launches += 2;
                    }
                }
                if (timed && record(c, e[2], s, capturing) != DIR_OK) return DIR_ECUDA;
                if (c->p.stop_mode >= 1) {
                    CK(c, dirk::launch_stop_test(c->red, c->p.stop_mode == 2 ? c->corr : nullptr,
                                                 (double)g.nx * g.ny * g.nz, c->lhist, row,
                                                 c->level_first[lc], c->p.stop_window, c->p.eps,
                                                 c->ctl + lc, it, s));
                    c->launches += 1;
                }
                if (timed) c->n_timed += 1;
            }
            sa.in = vbuf;
            sa.out = tbuf;
            sa.iter = 0;
            sa.stop_iter = nullptr;  // always: v of the last iteration run
            CK(c, dirk::launch_smooth(f64, sa, c->num_sms, s, plain));
            c->launches += 1;
            cur = tbuf;
            oth = vbuf;
            c->fused_level[lc] = sched;
            continue;
        }
        c->fused_level[lc] = 0;
        for (int it = 0; it < n; ++it, ++row) {
            cudaEvent_t* e = timed ? &c->tev[3 * (size_t)c->n_timed] : nullptr;
            if (timed && record(c, e[0], s, capturing) != DIR_OK) return DIR_ECUDA;
            fa.u = cur;
            fa.v = oth;
            fa.red = c->red + 3 * (size_t)row;
            fa.corr = c->corr ? c->corr + 4 * (size_t)row : nullptr;
            fa.iter = it;
            CK(c, dirk::launch_force(c->variant, f64, fa, s, plain));
            c->launches += 1;
            if (c->p.stop_mode >= 1) {
                // Sec. 2.4 on the relative norm, or (stop_mode 2) on the correlation
                CK(c, dirk::launch_stop_test(c->red, c->p.stop_mode == 2 ? c->corr : nullptr,
                                             (double)g.nx * g.ny * g.nz, c->lhist, row,
                                             c->level_first[lc], c->p.stop_window, c->p.eps,
                                             c->ctl + lc, it, s));
                c->launches += 1;
            }
            if (timed && record(c, e[1], s, capturing) != DIR_OK) return DIR_ECUDA;
            sa.in = oth;
            sa.out = cur;
            sa.iter = it;
            CK(c, dirk::launch_smooth(f64, sa, c->num_sms, s, plain));
            c->launches += 1;
            if (timed) {
                if (record(c, e[2], s, capturing) != DIR_OK) return DIR_ECUDA;
                c->n_timed += 1;
            }
        }
    }
    return enqueue_epilogue(c, cur, oth, s);
}

static int capture_graph(dir_ctx* c) {
    CK(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_registration(c, c->cap, true);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
    if (rc != DIR_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) {
        set_err(c, "cudaStreamEndCapture", e);
        return DIR_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        set_err(c, "cudaGraphInstantiate", ei);
        c->exec = nullptr;
        return DIR_ECUDA;
    }
    return DIR_OK;
}

static void release(dir_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    for (cudaEvent_t e : c->tev)
        if (e) cudaEventDestroy(e);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->cap) cudaStreamDestroy(c->cap);
    void* bufs[] = {c->img_pool, c->A, c->B, c->C, c->red, c->corr, c->lhist, c->ctl, c->derr,
                    c->stage_img, c->stage_f32, c->stage_f64};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, c->stream);
    delete c;
}

static int validate_params(const dir_params* p) {
    if (p->levels < 1 || p->levels > DIR_MAX_LEVELS) return DIR_EINVAL;
    for (int l = 0; l < p->levels; ++l)
        if (p->iters[l] < 0 || p->iters[l] > 1000000) return DIR_EINVAL;
    dirk::Taps t;
    if (!make_taps(p->sigma, &t)) return DIR_EINVAL;
    if (!isfinite(p->alpha)) return DIR_EINVAL;
    if (p->stop_mode < 0 || p->stop_mode > 2) return DIR_EINVAL;
    if (p->stop_mode >= 1 && (p->stop_window < 1 || !(p->eps >= 0.0))) return DIR_EINVAL;
    if (p->correlation != 0 && p->correlation != 1) return DIR_EINVAL;
    if (p->pdl != 0 && p->pdl != 1) return DIR_EINVAL;
    if (p->precision != DIR_F32 && p->precision != DIR_F64) return DIR_EUNSUPPORTED;
    if (p->field_dtype != DIR_F32 && p->field_dtype != DIR_BF16) return DIR_EUNSUPPORTED;
    if (p->field_dtype == DIR_BF16 && p->precision != DIR_F32) return DIR_EUNSUPPORTED;
    if (p->init_field && p->levels != 1) return DIR_EINVAL;
    if (p->fuse < 0 || p->fuse > 4) return DIR_EINVAL;
    if (p->plain_kernels != 0 && p->plain_kernels != 1) return DIR_EINVAL;
    return DIR_OK;
}

// Storage of images and fields from the requested dtypes (validated already).
static void setup_storage(dir_ctx* c, dir_dtype image_dtype) {
    c->fp64 = (c->p.precision == DIR_F64);
    c->esz = c->fp64 ? sizeof(double) : sizeof(float);
    c->real_type = c->fp64 ? dirk::kStoreF64 : dirk::kStoreF32;
    c->input_dtype = image_dtype;
    c->img0_type = image_dtype == DIR_I16 ? dirk::kStoreI16 : c->real_type;
    c->iesz0 = image_dtype == DIR_I16 ? 2 : c->esz;
    c->field_type = c->fp64 ? dirk::kStoreF64
                            : (c->p.field_dtype == DIR_BF16 ? dirk::kStoreBF16 : dirk::kStoreF32);
    c->fesz = c->field_type == dirk::kStoreF64 ? 8 : (c->field_type == dirk::kStoreF32 ? 4 : 2);
}

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

extern "C" {

int dir_params_default(dir_params* p) {
    if (!p) return DIR_EINVAL;
    memset(p, 0, sizeof *p);
    p->levels = 3;
    p->iters[0] = 200;
    p->iters[1] = 100;
    p->iters[2] = 50;
    p->sigma = 1.0;
    p->alpha = 0.4;
    p->stop_mode = 0;
    p->eps = 1e-4;
    p->stop_window = 10;
    p->field_dtype = DIR_F32;
    p->init_field = nullptr;
    p->use_graph = 1;
    p->timing = 0;
    p->precision = DIR_F32;
    p->fuse = 2;
    p->plain_kernels = 0;
    p->correlation = 0;
    p->pdl = 1;
    return DIR_OK;
}

int dir_create(dir_ctx** out, const void* static_img, const void* moving_img, const int dims[3],
               const float spacing_mm[3], dir_dtype image_dtype, int inputs_on_device,
               dir_variant variant, const dir_params* params, void* cuda_stream) {
    g_create_error.clear();
    if (!out) return DIR_EINVAL;
    *out = nullptr;
    if (!static_img || !moving_img || !dims || !spacing_mm) {
        g_create_error = "NULL argument";
        return DIR_EINVAL;
    }
    long long nvox = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || dims[a] > DIR_MAX_DIM || !(spacing_mm[a] > 0.0f) ||
            !isfinite(spacing_mm[a])) {
            g_create_error = "bad dims or spacing";
            return DIR_EINVAL;
        }
        nvox *= dims[a];
    }
    if (nvox > DIR_MAX_VOXELS) {
        g_create_error = "volume too large";
        return DIR_EINVAL;
    }
    if ((int)variant < 0 || (int)variant > 5) {
        g_create_error = "bad variant";
        return DIR_EINVAL;
    }
    if (image_dtype != DIR_F32 && image_dtype != DIR_I16) {
        g_create_error = "image dtype not supported by this build";
        return DIR_EUNSUPPORTED;
    }
    dir_params p;
    if (params)
        p = *params;
    else
        dir_params_default(&p);
    const int prc = validate_params(&p);
    if (prc != DIR_OK) {
        g_create_error = "bad params";
        return prc;
    }
    if (image_dtype == DIR_I16 && p.precision != DIR_F32) {
        g_create_error = "int16 images need single-precision arithmetic";
        return DIR_EUNSUPPORTED;
    }

    dir_ctx* c = new (std::nothrow) dir_ctx();
    if (!c) return DIR_ENOMEM;
    for (int a = 0; a < 3; ++a) {
        c->dims[a] = dims[a];
        c->spacing[a] = spacing_mm[a];
    }
    c->variant = (int)variant;
    c->p = p;
    setup_storage(c, image_dtype);
    c->stream = (cudaStream_t)cuda_stream;
    c->levels = p.levels;
    make_taps(p.sigma, &c->taps);
    make_taps(1.0, &c->taps1);

    auto fail = [&](int code) {
        if (g_create_error.empty()) g_create_error = c->err;
        release(c);
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        set_err(c, "cudaGetDevice", e);
        return fail(DIR_ECUDA);
    }

    // level grids and one pool for all pyramid images
    int nx = dims[0], ny = dims[1], nz = dims[2];
    size_t pool = 0;  // bytes
    size_t img_off[DIR_MAX_LEVELS][2];
    for (int l = 0; l < c->levels; ++l) {
        c->lv[l].g = make_grid(nx, ny, nz);
        for (int k = 0; k < 2; ++k) {
            img_off[l][k] = pool;
            pool = align256(pool + (size_t)c->lv[l].g.cs * c->img_esz(l));
        }
        nx = (nx + 1) / 2;
        ny = (ny + 1) / 2;
        nz = (nz + 1) / 2;
    }
    const size_t field = 3 * (size_t)c->lv[0].g.cs;
    if (field >= (size_t)0x7fffffff) {  // kernels index fields with 32-bit offsets
        g_create_error = "volume too large for 32-bit field offsets";
        return fail(DIR_EINVAL);
    }
    c->total_iters = 0;
    for (int l = 0; l < c->levels; ++l) c->total_iters += p.iters[l];
    const size_t nred = (size_t)(c->total_iters > 0 ? c->total_iters : 1);
    cudaStream_t st = c->stream;
    if (cudaMallocAsync(&c->img_pool, pool, st) != cudaSuccess ||
        cudaMallocAsync(&c->A, field * c->fesz, st) != cudaSuccess ||
        cudaMallocAsync(&c->B, field * c->fesz, st) != cudaSuccess ||
        cudaMallocAsync(&c->red, 3 * nred * sizeof(double), st) != cudaSuccess ||
        ((p.correlation || p.stop_mode == 2) &&
         cudaMallocAsync(&c->corr, 4 * nred * sizeof(double), st) != cudaSuccess) ||
        cudaMallocAsync(&c->lhist, nred * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync(&c->ctl, DIR_MAX_LEVELS * sizeof(int), st) != cudaSuccess ||
        cudaMallocAsync(&c->derr, sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "device allocation failed";
        return fail(DIR_ENOMEM);
    }
    for (int l = 0; l < c->levels; ++l) {
        c->lv[l].S = c->img_pool + img_off[l][0];
        c->lv[l].M = c->img_pool + img_off[l][1];
    }
    // the u + D scratch of schedule 3, for the largest level that runs it
    for (int l = 0; l < c->levels; ++l)
        if (p.iters[c->levels - 1 - l] > 0 && level_wants_d(c, l))
            c->C_bytes = std::max(c->C_bytes, level_d_bytes(c, l));
    if (c->C_bytes > 0 && cudaMallocAsync(&c->C, c->C_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "device allocation failed";
        return fail(DIR_ENOMEM);
    }
    e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e != cudaSuccess) {
        set_err(c, "stream/event creation", e);
        return fail(DIR_ECUDA);
    }
    if (p.timing) {
        const int n = p.iters[c->levels - 1];
        c->tev.resize(3 * (size_t)n, nullptr);
        for (auto& ev : c->tev) {
            e = cudaEventCreate(&ev);
            if (e != cudaSuccess) {
                set_err(c, "cudaEventCreate", e);
                return fail(DIR_ECUDA);
            }
        }
    }
    e = cudaMemsetAsync(c->img_pool, 0, pool, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) {
        set_err(c, "cudaMemsetAsync", e);
        return fail(DIR_ECUDA);
    }
    const int rc = upload_pair(c, static_img, moving_img, inputs_on_device, c->stream);
    if (rc != DIR_OK) return fail(rc);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        set_err(c, "cudaStreamSynchronize", e);
        return fail(DIR_ECUDA);
    }
    *out = c;
    return DIR_OK;
}

int dir_load(dir_ctx* c, const void* S, const void* M, dir_dtype dt, int on_device) {
    if (!c || !S || !M) return DIR_EINVAL;
    if (dt != c->input_dtype) return DIR_EUNSUPPORTED;
    if (c->pending) return DIR_ESTATE;
    const int rc = upload_pair(c, S, M, on_device, c->stream);
    if (rc != DIR_OK) return rc;
    c->have_field = false;
    CK(c, cudaStreamSynchronize(c->stream));
    return DIR_OK;
}

int dir_register_async(dir_ctx* c) {
    if (!c) return DIR_EINVAL;
    if (c->pending) return DIR_ESTATE;
    if (c->p.use_graph && !c->exec) {
        const int rc = capture_graph(c);
        if (rc != DIR_OK) return rc;
    }
    CK(c, cudaEventRecord(c->ev0, c->stream));
    if (c->p.use_graph) {
        CK(c, cudaGraphLaunch(c->exec, c->stream));
    } else {
        const int rc = enqueue_registration(c, c->stream, false);
        if (rc != DIR_OK) return rc;
    }
    CK(c, cudaEventRecord(c->ev1, c->stream));
    c->pending = true;
    c->have_field = false;
    return DIR_OK;
}

int dir_sync(dir_ctx* c, dir_stats* st) {
    if (!c) return DIR_EINVAL;
    if (!c->pending) return DIR_ESTATE;
    c->pending = false;
    const size_t nred = (size_t)(c->total_iters > 0 ? c->total_iters : 1);
    c->red_host.resize(3 * nred);
    c->ctl_host.resize(DIR_MAX_LEVELS + 1);
    CK(c, cudaMemcpyAsync(c->red_host.data(), c->red, 3 * nred * sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream));
    if (c->corr) {
        c->corr_host.resize(4 * nred);
        CK(c, cudaMemcpyAsync(c->corr_host.data(), c->corr, 4 * nred * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
    }
    CK(c, cudaMemcpyAsync(c->ctl_host.data(), c->ctl, c->levels * sizeof(int),
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(c->ctl_host.data() + DIR_MAX_LEVELS, c->derr, sizeof(int),
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (c->ctl_host[DIR_MAX_LEVELS] != 0) {
        c->err = "a device-side wait for a tensor copy timed out";
        return DIR_ETIMEOUT;
    }
    c->have_field = true;
    long long vu = 0;
    for (int lc = 0; lc < c->levels; ++lc) {
        const int stop = c->ctl_host[lc];
        int run = c->p.iters[lc];
        if (stop != kStopUnset && stop + 1 < run) run = stop + 1;
        c->iters_run[lc] = run;
        const Grid3& g = c->lv[c->levels - 1 - lc].g;
        vu += (long long)g.nx * g.ny * g.nz * run;
    }
    if (st) {
        memset(st, 0, sizeof *st);
        st->levels = c->levels;
        for (int lc = 0; lc < c->levels; ++lc) st->iters_run[lc] = c->iters_run[lc];
        const int fin = c->levels - 1;
        const Grid3& g0 = c->lv[0].g;
        const double n0 = (double)g0.nx * g0.ny * g0.nz;
        if (c->iters_run[fin] > 0) {
            const int r0 = c->level_first[fin];
            const int r1 = r0 + c->iters_run[fin] - 1;
            st->mse_first = c->red_host[3 * r0] / n0;
            st->mse_final = c->red_host[3 * r1] / n0;
            const double B = c->red_host[3 * r1 + 2];
            st->relnorm_final = B > 0.0 ? c->red_host[3 * r1 + 1] / B : 0.0;
        }
        float ms = 0.0f;
        CK(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        st->ms_total = ms;
        st->voxel_updates = vu;
        st->kernel_launches = c->launches;
        st->schedule_finest = c->fused_level[fin];
        if (c->p.timing) {
            const int runs = c->iters_run[fin];
            const bool fused = c->fused_level[fin] == 1;
            const bool split = c->fused_level[fin] >= 2;
            for (int i = 0; i < c->n_timed && i < runs; ++i) {
                float a = 0.f, b = 0.f;
                CK(c, cudaEventElapsedTime(&a, c->tev[3 * i], c->tev[3 * i + 1]));
                CK(c, cudaEventElapsedTime(&b, c->tev[3 * i + 1], c->tev[3 * i + 2]));
                if (split) {  // iterations > 0: the xy smoothing, then the z + force kernel
                    if (i > 0) {
                        st->ms_smooth_finest += a;
                        st->n_smooth_finest += 1;
                        st->ms_force_finest += b;
                        st->n_force_finest += 1;
                    }
                    continue;
                }
                if (fused && i > 0) {
                    st->ms_fused_finest += a;
                    st->n_fused_finest += 1;
                } else {
                    st->ms_force_finest += a;
                    st->n_force_finest += 1;
                }
                if (!fused || i == runs - 1) {
                    st->ms_smooth_finest += b;
                    st->n_smooth_finest += 1;
                }
            }
        }
    }
    return DIR_OK;
}

int dir_register(dir_ctx* c, dir_stats* st) {
    const int rc = dir_register_async(c);
    if (rc != DIR_OK) return rc;
    return dir_sync(c, st);
}

int dir_get_history(dir_ctx* c, double* out, int max_iters) {
    if (!c || (!out && max_iters > 0) || max_iters < 0) return DIR_EINVAL;
    if (!c->have_field) return DIR_ESTATE;
    int w = 0;
    for (int lc = 0; lc < c->levels; ++lc) {
        const Grid3& g = c->lv[c->levels - 1 - lc].g;
        const double n = (double)g.nx * g.ny * g.nz;
        for (int it = 0; it < c->iters_run[lc] && w < max_iters; ++it, ++w) {
            const double* r = &c->red_host[3 * (size_t)(c->level_first[lc] + it)];
            out[3 * w + 0] = r[0] / n;
            out[3 * w + 1] = r[1];
            out[3 * w + 2] = r[2];
        }
    }
    return w;
}

int dir_get_correlation(dir_ctx* c, double* out, int max_iters) {
    if (!c || (!out && max_iters > 0) || max_iters < 0) return DIR_EINVAL;
    if (!c->corr) return DIR_EUNSUPPORTED;  // not asked for at dir_create
    if (!c->have_field) return DIR_ESTATE;
    int w = 0;
    for (int lc = 0; lc < c->levels; ++lc) {
        const Grid3& g = c->lv[c->levels - 1 - lc].g;
        const double n = (double)g.nx * g.ny * g.nz;
        for (int it = 0; it < c->iters_run[lc] && w < max_iters; ++it, ++w) {
            const size_t row = (size_t)(c->level_first[lc] + it);
            out[w] = dirk::correlation_from_sums(c->red_host[3 * row], &c->corr_host[4 * row], n);
        }
    }
    return w;
}

static int get_field(dir_ctx* c, void* out, int in_mm, int out_on_device, bool out_fp64) {
    if (!c || !out) return DIR_EINVAL;
    if (!c->have_field || !c->final_field) return DIR_ESTATE;
    const Grid3& g = c->lv[0].g;
    const size_t n = c->nvox();
    const size_t osz = out_fp64 ? sizeof(double) : sizeof(float);
    void* dst = out;
    if (!out_on_device) {
        void** stage = out_fp64 ? (void**)&c->stage_f64 : (void**)&c->stage_f32;
        const int rc = ensure(c, stage, 3 * n * osz);
        if (rc != DIR_OK) return rc;
        dst = *stage;
    }
    const double sx = in_mm ? c->spacing[0] : 1.0;
    const double sy = in_mm ? c->spacing[1] : 1.0;
    const double sz = in_mm ? c->spacing[2] : 1.0;
    CK(c, dirk::launch_export_field(c->fp64, c->field_type, c->final_field, g, sx, sy, sz, dst,
                                    out_fp64,
                                    c->stream));
    if (!out_on_device)
        CK(c, cudaMemcpyAsync(out, dst, 3 * n * osz, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return DIR_OK;
}

int dir_get_field(dir_ctx* c, float* out, int in_mm, int out_on_device) {
    return get_field(c, out, in_mm, out_on_device, false);
}

int dir_get_field_f64(dir_ctx* c, double* out, int in_mm, int out_on_device) {
    return get_field(c, out, in_mm, out_on_device, true);
}

int dir_warp(dir_ctx* c, const void* img_in, void* img_out, dir_dtype dt, int on_device) {
    if (!c || !img_in || !img_out) return DIR_EINVAL;
    if (dt != DIR_F32) return DIR_EUNSUPPORTED;
    if (!c->have_field || !c->final_field) return DIR_ESTATE;
    const Grid3& g = c->lv[0].g;
    const size_t n = c->nvox();
    int rc = ensure(c, (void**)&c->stage_img, (size_t)g.cs * c->esz);
    if (rc != DIR_OK) return rc;
    rc = import_dense(c, img_in, on_device, 4, c->stage_img, c->real_type, g, 1, c->stream);
    if (rc != DIR_OK) return rc;
    float* dst = (float*)img_out;
    if (!on_device) {
        rc = ensure(c, (void**)&c->stage_f32, 3 * n * sizeof(float));
        if (rc != DIR_OK) return rc;
        dst = c->stage_f32;
    }
    CK(c, dirk::launch_warp(c->fp64, c->field_type, c->stage_img, c->final_field, g, dst,
                            c->stream));
    if (!on_device)
        CK(c, cudaMemcpyAsync(img_out, dst, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return DIR_OK;
}

void dir_destroy(dir_ctx* c) { release(c); }

const char* dir_status_string(int s) {
    switch (s) {
        case DIR_OK: return "ok";
        case DIR_EINVAL: return "invalid argument";
        case DIR_ENOMEM: return "out of memory";
        case DIR_ECUDA: return "CUDA error";
        case DIR_ESTATE: return "call out of order";
        case DIR_EUNSUPPORTED: return "not supported by this build";
        case DIR_ETIMEOUT: return "device-side wait timed out";
        default: return "unknown status";
    }
}

const char* dir_last_error(const dir_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

const char* dir_version(void) { return "gb300-demons 0.2 (sm_103a)"; }

int dir_check_wait_timeout(void* stream_ptr, double limit_ms) {
    if (!(limit_ms >= 1.0 && limit_ms <= 2000.0)) return DIR_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream_ptr);
    int* word = nullptr;
    int flagged = 0;
    if (cudaMallocAsync(reinterpret_cast<void**>(&word), sizeof(int), s) != cudaSuccess)
        return DIR_ECUDA;
    bool ok = cudaMemsetAsync(word, 0, sizeof(int), s) == cudaSuccess &&
              dirk::launch_wait_probe(word, (unsigned long long)(limit_ms * 1.0e6), s) ==
                  cudaSuccess &&
              cudaMemcpyAsync(&flagged, word, sizeof(int), cudaMemcpyDeviceToHost, s) ==
                  cudaSuccess;
    ok = cudaFreeAsync(word, s) == cudaSuccess && ok;
    ok = cudaStreamSynchronize(s) == cudaSuccess && ok;
    if (!ok) return DIR_ECUDA;
    return (flagged & dirk::kErrTmaTimeout) ? DIR_ETIMEOUT : DIR_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Batched registrations and launch-shape autotuning.
//
// dir_batch_create captures the registrations of many contexts into one CUDA
// graph: the contexts are spread over K branches (longest job first onto the
// least loaded branch), the branches run concurrently on the GPU, and one
// graph launch replays the whole batch.  Small volumes and coarse pyramid
// levels, each of which leaves most SMs idle, then fill the GPU together.
//
// dir_autotune times, per pyramid level of a context, the force kernel's brick
// depth (1, 2, 4, 8 voxels per thread along z) and the smoothing kernel's z
// chunk (planes per block), keeps the fastest of each and drops the context's
// captured graph so that the next registration uses them.
// ------------------------------------------------------------------------
struct dir_batch {
    std::vector<dir_ctx*> ctxs;
    cudaStream_t stream = nullptr;       // the caller's stream: where the graph runs
    cudaStream_t origin = nullptr;       // capture helpers
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaGraphExec_t exec = nullptr;
    int branches = 1;
    bool grouped = false;  // grouped launches per iteration (else per-context branches)
};

static double ctx_work(const dir_ctx* c) {
    double w = 0.0;
    for (int lc = 0; lc < c->levels; ++lc) {
        const Grid3& g = c->lv[c->levels - 1 - lc].g;
        w += (double)g.nx * g.ny * g.nz * c->p.iters[lc];
    }
    return c->variant == DIR_INVERSE_CONSISTENT ? 1.4 * w : w;
}

static void batch_release(dir_batch* b) {
    if (!b) return;
    if (b->stream || b->origin) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaStream_t s : b->br) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

#define BK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) {                      \
            set_err(nullptr, #call, e_);              \
            batch_release(b);                         \
            return DIR_ECUDA;                         \
        }                                             \
    } while (0)

// The grouped form's requirements (see dir_batch_create in dir.h)
static bool batch_groupable(dir_ctx* const* ctxs, int n) {
    const dir_ctx* c0 = ctxs[0];
    for (int i = 0; i < n; ++i) {
        const dir_ctx* c = ctxs[i];
        if (c->fp64 || c->p.plain_kernels || c->field_type != dirk::kStoreF32 ||
            c->p.stop_mode != 0 || (c->p.fuse != 2 && c->p.fuse != 3) || c->taps.R != 3 ||
            c->levels != c0->levels || c->taps.wf[0] != c0->taps.wf[0])
            return false;
        for (int lc = 0; lc < c->levels; ++lc)
            if (c->p.iters[lc] != c0->p.iters[lc]) return false;
        for (int l = 0; l < c->levels; ++l)
            if (c->img_type(l) != dirk::kStoreF32 && c->img_type(l) != dirk::kStoreI16) return false;
    }
    return true;
}

// Records one chunk of the grouped form on stream s (under capture): jobs of
// one force law and image storage, at most kGroupMax, moving in lockstep.  Per
// level: each job's field start and first force pass, then every later
// iteration as one grouped x/y and one grouped z + force launch over all the
// jobs, then each job's last smoothing.
static int enqueue_grouped_chunk(dir_ctx* const* ctxs, const std::vector<int>& jobs,
                                 cudaStream_t s) {
    const int n = (int)jobs.size();
    const int L = ctxs[jobs[0]]->levels;
    std::vector<char*> cur(n), oth(n);
    std::vector<int> row(n, 0);
    for (int q = 0; q < n; ++q) {
        dir_ctx* c = ctxs[jobs[q]];
        const int rc = enqueue_prologue(c, s);
        if (rc != DIR_OK) return rc;
        cur[q] = c->A;
        oth[q] = c->B;
        c->n_timed = 0;
    }
    dir_ctx* c0 = ctxs[jobs[0]];
    for (int lc = 0; lc < L; ++lc) {
        const int l = L - 1 - lc;
        const int iters = c0->p.iters[lc];
        std::vector<Grid3> grids(n);
        for (int q = 0; q < n; ++q) {
            dir_ctx* c = ctxs[jobs[q]];
            const int rc = enqueue_level_start(c, lc, cur[q], oth[q], s);
            if (rc != DIR_OK) return rc;
            c->level_first[lc] = row[q];
            c->fused_level[lc] = 0;
            grids[q] = c->lv[l].g;
        }
        if (iters == 0) continue;
        // Eqs. 3-6 where every job has its u + D scratch: the split after the
        // difference image, as each job's own registration would run it
        bool dform = c0->variant >= 2;
        for (int q = 0; q < n; ++q) {
            const dir_ctx* c = ctxs[jobs[q]];
            dform = dform && c->C && c->C_bytes >= level_d_bytes(c, l);
        }
        for (int q = 0; q < n; ++q) ctxs[jobs[q]]->fused_level[lc] = dform ? 3 : 2;
        // iteration 0 from the level's starting field, per job
        for (int q = 0; q < n; ++q) {
            dir_ctx* c = ctxs[jobs[q]];
            dirk::ForceArgs fa = level_force_args(c, lc);
            fa.u = cur[q];
            fa.v = oth[q];
            fa.red = c->red + 3 * (size_t)row[q];
            fa.corr = c->corr ? c->corr + 4 * (size_t)row[q] : nullptr;
            fa.iter = 0;
            fa.depth = dirk::force_brick_depth(c->lv[l].g, c->num_sms);
            CK(c, dirk::launch_force(c->variant, false, fa, s, false));
            c->launches += 1;
        }
        int ty = 0, zc = 0, depth = 0;
        dirk::group_shapes(c0->variant, grids.data(), n, c0->num_sms, &ty, &zc, &depth);
        dirk::XYGroup X;
        dirk::ZSGroup Z;
        dirk::ZDGroup ZD;
        dirk::STGroup ST;
        X.ty = ty;
        X.zchunk = zc;
        Z.variant = ZD.variant = ST.variant = c0->variant;
        Z.depth = ZD.depth = ST.depth = depth;
        Z.taps = ZD.taps = c0->taps;
        for (int q = 0; q < n; ++q) {
            dir_ctx* c = ctxs[jobs[q]];
            dirk::SmoothArgs sa = level_smooth_args(c, lc);
            sa.in = oth[q];
            sa.out = cur[q];
            sa.stop_iter = nullptr;
            sa.iter = 0;
            dirk::ForceArgs fa = level_force_args(c, lc);
            fa.u = cur[q];
            fa.v = oth[q];
            fa.stop_iter = nullptr;
            fa.depth = depth;
            bool added = dirk::xy_group_add(X, sa);
            if (dform) {
                dirk::ForceArgs za = fa, ta = fa;
                char* dpl = c->C + 3 * (size_t)grids[q].cs * sizeof(float);
                za.v = c->C;
                ta.u = c->C;
                za.dbuf = ta.dbuf = dpl;
                za.dbuf2 = ta.dbuf2 = c->variant == DIR_INVERSE_CONSISTENT
                                          ? dpl + (size_t)grids[q].cs * sizeof(float)
                                          : nullptr;
                added = added && dirk::d_group_add(ZD, ST, za, ta);
            } else {
                added = added && dirk::zs_group_add(Z, fa);
            }
            if (!added) {
                c->err = "grouped batch: a tensor map could not be made";
                return DIR_EINVAL;
            }
        }
        const int img = c0->img_type(l);
        long long chunk_vox = 0;  // the level of the whole chunk, for the rule of level_pdl
        for (int q = 0; q < n; ++q) chunk_vox += (long long)grids[q].nx * grids[q].ny * grids[q].nz;
        const bool pdl = c0->p.pdl && chunk_vox > (1LL << 18);
        for (int it = 1; it < iters; ++it) {
            for (int q = 0; q < n; ++q) {
                dir_ctx* c = ctxs[jobs[q]];
                const size_t r = (size_t)(row[q] + it);
                dirk::ForceArgs& fa = dform ? ST.a[q] : Z.a[q];
                fa.red = c->red + 3 * r;
                fa.corr = c->corr ? c->corr + 4 * r : nullptr;
                fa.iter = it;
                ZD.a[q].iter = it;
                X.a[q].iter = it;
                c->launches += dform ? 3 : 2;
            }
            CK(c0, dirk::launch_smooth_xy_grouped(X, s, pdl));
            if (dform)
                CK(c0, dirk::launch_force_d_grouped(img, ZD, ST, s, pdl));
            else
                CK(c0, dirk::launch_force_zs_grouped(c0->variant, img, Z, s, pdl));
        }
        // u = G v of the last iteration, per job
        for (int q = 0; q < n; ++q) {
            dir_ctx* c = ctxs[jobs[q]];
            dirk::SmoothArgs sa = level_smooth_args(c, lc);
            sa.in = oth[q];
            sa.out = cur[q];
            sa.stop_iter = nullptr;
            sa.iter = 0;
            CK(c, dirk::launch_smooth(false, sa, c->num_sms, s, false));
            c->launches += 1;
            row[q] += iters;
        }
    }
    for (int q = 0; q < n; ++q) {
        const int rc = enqueue_epilogue(ctxs[jobs[q]], cur[q], oth[q], s);
        if (rc != DIR_OK) return rc;
    }
    return DIR_OK;
}

// Chunks of the grouped form: contexts of one force law and level-0 image
// storage, split into near-equal chunks of at most kGroupMax
static std::vector<std::vector<int>> grouped_chunks(dir_ctx* const* ctxs, int n) {
    std::vector<std::vector<int>> out;
    std::vector<bool> done(n, false);
    for (int i = 0; i < n; ++i) {
        if (done[i]) continue;
        std::vector<int> m;
        for (int k = i; k < n; ++k)
            if (!done[k] && ctxs[k]->variant == ctxs[i]->variant &&
                ctxs[k]->img_type(0) == ctxs[i]->img_type(0)) {
                m.push_back(k);
                done[k] = true;
            }
        const int parts = ((int)m.size() + dirk::kGroupMax - 1) / dirk::kGroupMax;
        for (int p = 0; p < parts; ++p) {
            std::vector<int> chunk;
            for (int q = p; q < (int)m.size(); q += parts) chunk.push_back(m[q]);
            out.push_back(chunk);
        }
    }
    return out;
}

extern "C" int dir_batch_create(dir_batch** out, dir_ctx* const* ctxs, int n, int branches,
                                int flags, void* cuda_stream) {
    g_create_error.clear();
    if (!out) return DIR_EINVAL;
    *out = nullptr;
    if (!ctxs || n < 1 || branches < 1) return DIR_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || ctxs[i]->pending || ctxs[i]->p.timing) {
            g_create_error = "dir_batch_create: NULL, busy or timed context";
            return DIR_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) {
                g_create_error = "dir_batch_create: a context appears twice";
                return DIR_EINVAL;
            }
    }
    dir_batch* b = new (std::nothrow) dir_batch();
    if (!b) return DIR_ENOMEM;
    b->ctxs.assign(ctxs, ctxs + n);
    b->stream = (cudaStream_t)cuda_stream;
    // grouped form: one branch per chunk; branch form: `branches` (at most n)
    b->grouped = !(flags & DIR_BATCH_BRANCHES) && batch_groupable(ctxs, n);
    std::vector<std::vector<int>> chunks;
    if (b->grouped) chunks = grouped_chunks(ctxs, n);
    b->branches = b->grouped ? (int)chunks.size() : (branches < n ? branches : n);
    BK(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
    BK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    BK(cudaEventCreate(&b->t0));
    BK(cudaEventCreate(&b->t1));
    b->br.resize(b->branches, nullptr);
    b->join.resize(b->branches, nullptr);
    for (int k = 0; k < b->branches; ++k) {
        BK(cudaStreamCreateWithFlags(&b->br[k], cudaStreamNonBlocking));
        BK(cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming));
    }
    // longest job first onto the least loaded branch
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && ctx_work(ctxs[order[j]]) > ctx_work(ctxs[order[j - 1]]); --j) {
            const int t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
        }
    std::vector<double> load(b->branches, 0.0);
    std::vector<int> branch_of(n, 0);
    for (int i : order) {
        int best = 0;
        for (int k = 1; k < b->branches; ++k)
            if (load[k] < load[best]) best = k;
        branch_of[i] = best;
        load[best] += ctx_work(ctxs[i]);
    }
    BK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    int rc = DIR_OK;
    cudaError_t ce = cudaSuccess;
    if (b->grouped) {
        // each chunk on its own branch (chunks never share data), in lockstep
        // within the chunk
        ce = cudaEventRecord(b->fork, b->origin);
        for (int k = 0; k < b->branches && ce == cudaSuccess; ++k)
            ce = cudaStreamWaitEvent(b->br[k], b->fork, 0);
        for (size_t k = 0; k < chunks.size() && ce == cudaSuccess && rc == DIR_OK; ++k) {
            rc = enqueue_grouped_chunk(ctxs, chunks[k], b->br[k]);
            if (rc != DIR_OK)
                for (int i : chunks[k])
                    if (!ctxs[i]->err.empty()) g_create_error = ctxs[i]->err;
        }
        for (int k = 0; k < b->branches && ce == cudaSuccess; ++k) {
            ce = cudaEventRecord(b->join[k], b->br[k]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->origin, b->join[k], 0);
        }
    } else {
        ce = cudaEventRecord(b->fork, b->origin);
        for (int k = 0; k < b->branches && ce == cudaSuccess; ++k)
            ce = cudaStreamWaitEvent(b->br[k], b->fork, 0);
        for (int i : order) {
            if (ce != cudaSuccess || rc != DIR_OK) break;
            rc = enqueue_registration(ctxs[i], b->br[branch_of[i]], true);
            if (rc != DIR_OK) g_create_error = ctxs[i]->err;
        }
        for (int k = 0; k < b->branches && ce == cudaSuccess; ++k) {
            ce = cudaEventRecord(b->join[k], b->br[k]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->origin, b->join[k], 0);
        }
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->origin, &graph);
    if (rc != DIR_OK || ce != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (rc == DIR_OK) set_err(nullptr, "batch capture", ce != cudaSuccess ? ce : ee);
        batch_release(b);
        return rc != DIR_OK ? rc : DIR_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        b->exec = nullptr;
        set_err(nullptr, "cudaGraphInstantiate", ei);
        batch_release(b);
        return DIR_ECUDA;
    }
    *out = b;
    return DIR_OK;
}

extern "C" int dir_batch_run(dir_batch* b, float* ms_out) {
    if (!b) return DIR_EINVAL;
    for (dir_ctx* c : b->ctxs)
        if (c->pending) return DIR_ESTATE;
    cudaError_t e = cudaEventRecord(b->t0, b->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->t1, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        set_err(nullptr, "dir_batch_run", e);
        return DIR_ECUDA;
    }
    // per-context results: iterations run, reductions, field ready
    for (dir_ctx* c : b->ctxs) {
        c->pending = true;
        const int rc = dir_sync(c, nullptr);
        if (rc != DIR_OK) return rc;
    }
    if (ms_out) {
        e = cudaEventElapsedTime(ms_out, b->t0, b->t1);
        if (e != cudaSuccess) return DIR_ECUDA;
    }
    return DIR_OK;
}

extern "C" int dir_batch_grouped(const dir_batch* b) { return b ? (b->grouped ? 1 : 0) : -1; }

extern "C" void dir_batch_destroy(dir_batch* b) { batch_release(b); }

extern "C" int dir_autotune(dir_ctx* c, int reps, int* shapes_out) {
    if (!c || reps < 1) return DIR_EINVAL;
    if (c->pending) return DIR_ESTATE;
    if (!c->have_field) return DIR_ESTATE;  // needs the pyramid of a finished registration
    const Grid3& g0 = c->lv[0].g;
    const size_t fbytes = align256(3 * (size_t)g0.cs * c->fesz);
    char* scratch = nullptr;  // u, v and the reduction sums of the trial launches
    if (cudaMallocAsync((void**)&scratch, 2 * fbytes + 256, c->stream) != cudaSuccess) {
        cudaGetLastError();
        c->err = "autotune: allocation failed";
        return DIR_ENOMEM;
    }
    void* u = scratch;
    void* v = scratch + fbytes;
    double* red = reinterpret_cast<double*>(scratch + 2 * fbytes);
    cudaEvent_t ea = nullptr, eb = nullptr;
    int rc = DIR_OK;
    auto timed = [&](auto&& launch, float* ms) -> int {
        CK(c, launch());  // warm up (also sets kernel attributes)
        CK(c, cudaEventRecord(ea, c->stream));
        for (int r = 0; r < reps; ++r) CK(c, launch());
        CK(c, cudaEventRecord(eb, c->stream));
        CK(c, cudaEventSynchronize(eb));
        CK(c, cudaEventElapsedTime(ms, ea, eb));
        return DIR_OK;
    };
    if (cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess) rc = DIR_ECUDA;
    if (rc == DIR_OK && cudaMemsetAsync(scratch, 0, 2 * fbytes + 256, c->stream) != cudaSuccess)
        rc = DIR_ECUDA;
    for (int l = 0; l < c->levels && rc == DIR_OK; ++l) {
        const Grid3& g = c->lv[l].g;
        dirk::ForceArgs fa;
        fa.S = c->lv[l].S;
        fa.M = c->lv[l].M;
        fa.u = u;
        fa.v = v;
        fa.g = g;
        fa.alpha2 = c->p.alpha * c->p.alpha;
        fa.red = red;
        fa.stop_iter = nullptr;
        fa.iter = 0;
        fa.img_type = c->img_type(l);
        fa.field_type = c->field_type;
        fa.err = c->derr;
        fa.pf_stride = c->num_sms;  // as in the registration
        const int sched = level_schedule(c, l);  // time the kernels the level runs
        const bool split = sched >= 2;
        float best = 1e30f;
        int best_d = 0;
        const int depths[5] = {1, 2, 4, 8, 6};  // 6: the split force kernel only
        // schedule 3: the z + D and stencil force kernels, u and D in the scratch
        dirk::ForceArgs za = fa, ta = fa;
        if (sched == 3) {
            char* dpl = c->C + 3 * (size_t)g.cs * sizeof(float);
            za.v = c->C;
            ta.u = c->C;
            za.dbuf = ta.dbuf = dpl;
            za.dbuf2 = ta.dbuf2 = c->variant == DIR_INVERSE_CONSISTENT
                                      ? dpl + (size_t)g.cs * sizeof(float)
                                      : nullptr;
        }
        for (int di = 0; di < (sched == 2 ? 5 : 4) && rc == DIR_OK; ++di) {
            const int d = depths[di];
            fa.depth = ta.depth = d;
            za.depth = std::min(d, kZdMaxDepth);
            float ms = 0.0f;
            rc = timed([&]() {
                if (sched == 3) return dirk::launch_force_d(c->variant, za, ta, c->taps, c->stream);
                if (split) return dirk::launch_force_zs(c->variant, fa, c->taps, c->stream);
                return dirk::launch_force(c->variant, c->fp64, fa, c->stream, c->p.plain_kernels != 0);
            }, &ms);
            if (rc == DIR_OK && ms < best) {
                best = ms;
                best_d = d;
            }
        }
        dirk::SmoothArgs sa;
        sa.in = v;
        sa.out = u;
        sa.g = g;
        sa.ncomp = 3;
        sa.taps = c->taps;
        sa.stop_iter = nullptr;
        sa.iter = 0;
        sa.err = c->derr;
        sa.in_type = c->field_type;
        sa.out_type = c->field_type;
        best = 1e30f;
        int best_z = 0;
        int cand[16], nc = 0;
        cand[nc++] = 0;  // one wave (the default)
        for (int z = 1; z < g.nz && nc < 15; z *= 2) cand[nc++] = z;
        cand[nc++] = g.nz;
        for (int k = 0; k < nc && rc == DIR_OK; ++k) {
            sa.zchunk = cand[k];
            float ms = 0.0f;
            rc = timed([&]() {
                if (split) return dirk::launch_smooth_xy(sa, c->num_sms, c->stream);
                return dirk::launch_smooth(c->fp64, sa, c->num_sms, c->stream, c->p.plain_kernels != 0);
            }, &ms);
            if (rc == DIR_OK && ms < best) {
                best = ms;
                best_z = cand[k];
            }
        }
        c->tune_depth[l] = best_d;
        c->tune_zchunk[l] = best_z;
        if (shapes_out) {
            shapes_out[2 * l] = best_d;
            shapes_out[2 * l + 1] = best_z;
        }
    }
    if (ea) cudaEventDestroy(ea);
    if (eb) cudaEventDestroy(eb);
    cudaFreeAsync(scratch, c->stream);
    cudaStreamSynchronize(c->stream);
    if (c->exec) {  // recapture with the new shapes at the next registration
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    return rc;
}

// ------------------------------------------------------------------------
// Registration without device allocation (see dir_register_noalloc in dir.h).
//
// All scratch -- pyramid images, the two field buffers, reduction rows, stop
// flags -- lives in one file-scope device array.  Its device address is looked
// up once per device with cudaGetSymbolAddress (the array's name in host code
// is only a host-side stand-in) and cached.  Every call shares the array, so
// calls whose GPU work overlaps (different streams, or another host thread)
// race on it.
// ------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t kNoallocScratchBytes = 48ull << 20;  // 48 MiB
constexpr int kNoallocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

}  // namespace

extern "C" int dir_register_noalloc(const float* static_img, const float* moving_img,
                                    const int dims[3], dir_variant variant,
                                    const dir_params* params, float* field_out, void* cuda_stream,
                                    dir_stats* stats_out) {
    g_create_error.clear();
    if (!static_img || !moving_img || !dims || !field_out) return DIR_EINVAL;
    if ((int)variant < 0 || (int)variant > 5) return DIR_EINVAL;
    long long nvox = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || dims[a] > DIR_MAX_DIM) return DIR_EINVAL;
        nvox *= dims[a];
    }
    dir_params p;
    if (params)
        p = *params;
    else
        dir_params_default(&p);
    const int prc = validate_params(&p);
    if (prc != DIR_OK) return prc;
    if (p.timing) return DIR_EINVAL;  // event timing is not offered here

    // the context lives on the stack and points into the static scratch
    dir_ctx c;
    for (int a = 0; a < 3; ++a) {
        c.dims[a] = dims[a];
        c.spacing[a] = 1.0f;
    }
    c.variant = (int)variant;
    c.p = p;
    c.p.use_graph = 0;
    setup_storage(&c, DIR_F32);
    c.stream = (cudaStream_t)cuda_stream;
    c.levels = p.levels;
    make_taps(p.sigma, &c.taps);
    make_taps(1.0, &c.taps1);

    // scratch layout, each piece 256-byte aligned
    int nx = dims[0], ny = dims[1], nz = dims[2];
    size_t at = 0;
    size_t lvl_off[DIR_MAX_LEVELS][2];
    for (int l = 0; l < c.levels; ++l) {
        c.lv[l].g = make_grid(nx, ny, nz);
        lvl_off[l][0] = at;
        at = align256(at + (size_t)c.lv[l].g.cs * c.img_esz(l));
        lvl_off[l][1] = at;
        at = align256(at + (size_t)c.lv[l].g.cs * c.img_esz(l));
        nx = (nx + 1) / 2;
        ny = (ny + 1) / 2;
        nz = (nz + 1) / 2;
    }
    const size_t field = 3 * (size_t)c.lv[0].g.cs;
    if (field >= (size_t)0x7fffffff) return DIR_EINVAL;
    c.total_iters = 0;
    for (int l = 0; l < c.levels; ++l) c.total_iters += p.iters[l];
    const size_t nred = (size_t)(c.total_iters > 0 ? c.total_iters : 1);
    const size_t offA = at;
    at = align256(at + field * c.fesz);
    const size_t offB = at;
    at = align256(at + field * c.fesz);
    const size_t offRed = at;
    at = align256(at + 3 * nred * sizeof(double));
    const bool want_corr = p.correlation || p.stop_mode == 2;
    const size_t offCorr = at;
    if (want_corr) at = align256(at + 4 * nred * sizeof(double));
    const size_t offL = at;
    at = align256(at + nred * sizeof(double));
    const size_t offCtl = at;
    at = align256(at + DIR_MAX_LEVELS * sizeof(int));
    const size_t offErr = at;
    at = align256(at + sizeof(int));
    if (at > kNoallocScratchBytes) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "dir_register_noalloc: this volume and schedule need %.1f MiB of scratch, "
                 "the static limit is %.0f MiB",
                 at / 1048576.0, kNoallocScratchBytes / 1048576.0);
        g_create_error = buf;
        return DIR_EINVAL;
    }

    // device address of the static scratch, once per device, that device current
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        g_create_error = "dir_register_noalloc: no usable current device";
        return DIR_ECUDA;
    }
    char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                set_err(nullptr, "cudaGetSymbolAddress", e);
                return DIR_ECUDA;
            }
            g_noalloc_ptr[dev] = ptr;
        }
        base = static_cast<char*>(g_noalloc_ptr[dev]);
    }
    c.device = dev;
    e = cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        set_err(nullptr, "cudaDeviceGetAttribute", e);
        return DIR_ECUDA;
    }
    for (int l = 0; l < c.levels; ++l) {
        c.lv[l].S = base + lvl_off[l][0];
        c.lv[l].M = base + lvl_off[l][1];
    }
    c.A = base + offA;
    c.B = base + offB;
    c.red = reinterpret_cast<double*>(base + offRed);
    c.corr = want_corr ? reinterpret_cast<double*>(base + offCorr) : nullptr;
    c.lhist = reinterpret_cast<double*>(base + offL);
    c.ctl = reinterpret_cast<int*>(base + offCtl);
    c.derr = reinterpret_cast<int*>(base + offErr);

    int rc = upload_pair(&c, static_img, moving_img, 1, c.stream);
    if (rc == DIR_OK) rc = enqueue_registration(&c, c.stream, false);
    if (rc == DIR_OK && dirk::launch_export_field(c.fp64, c.field_type, c.final_field, c.lv[0].g,
                                                  1.0, 1.0, 1.0, field_out, false,
                                                  c.stream) != cudaSuccess)
        rc = DIR_ECUDA;
    int ctl[DIR_MAX_LEVELS + 1] = {0};
    if (rc == DIR_OK &&
        (cudaMemcpyAsync(ctl, c.ctl, c.levels * sizeof(int), cudaMemcpyDeviceToHost, c.stream) !=
             cudaSuccess ||
         cudaMemcpyAsync(ctl + DIR_MAX_LEVELS, c.derr, sizeof(int), cudaMemcpyDeviceToHost,
                         c.stream) != cudaSuccess ||
         cudaStreamSynchronize(c.stream) != cudaSuccess))
        rc = DIR_ECUDA;
    if (rc != DIR_OK) {
        // work queued before the failure may still be writing the shared
        // scratch: wait for it (its status is already reported by rc) so that
        // the next serialised call does not race with it
        cudaStreamSynchronize(c.stream);
        cudaGetLastError();
        if (!c.err.empty()) g_create_error = c.err;
        return rc;
    }
    if (ctl[DIR_MAX_LEVELS] != 0) return DIR_ETIMEOUT;
    if (stats_out) {
        memset(stats_out, 0, sizeof *stats_out);
        stats_out->levels = c.levels;
        long long vu = 0;
        for (int lc = 0; lc < c.levels; ++lc) {
            int run = p.iters[lc];
            if (ctl[lc] != kStopUnset && ctl[lc] + 1 < run) run = ctl[lc] + 1;
            stats_out->iters_run[lc] = run;
            const Grid3& g = c.lv[c.levels - 1 - lc].g;
            vu += (long long)g.nx * g.ny * g.nz * run;
        }
        stats_out->voxel_updates = vu;
        stats_out->kernel_launches = c.launches + 1;
    }
    return DIR_OK;
}
