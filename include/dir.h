/*
 * dir.h -- C ABI of the GB300 demons deformable image registration library
 * (libdir.so).
 *
 * The library registers a moving volume M to a static volume S with the
 * demons algorithm and its variants as defined in Gu et al., "Implementation
 * and evaluation of various demons deformable image registration algorithms on
 * GPU": every iteration warps M by the current displacement field with
 * trilinear interpolation (Sec. 2.5), computes a per-voxel demons force
 * (Eqs. 1-6), adds the update, smooths the total field with a Gaussian
 * (Sec. 2.1, Sec. 2.5) and reduces the mean squared difference and the field
 * norms used by the relative-norm stop test (Sec. 2.4), inside a coarse-to-fine
 * pyramid with factor-2 down-sampling and field up-sampling (Sec. 2.3).
 *
 * Conventions
 *   Volumes are dense, x-contiguous: voxel (i, j, k) is element
 *   i + nx * (j + ny * k) (Sec. 2.5: x as rows, y as columns, z as frames).
 *   A displacement field is three planar float arrays (x, y, z components),
 *   each nx*ny*nz elements, back to back (3*N floats), in voxel units unless a
 *   call says mm.  The field u is defined on the static grid: the warped image
 *   is W(x) = M(x + u(x)), so the static point x corresponds to the moving
 *   point x + u(x) (the convention used to apply the field to landmarks,
 *   Sec. 3.2).  All boundaries replicate the edge voxel.
 *
 * Threading and streams
 *   A context is not thread-safe: one host thread at a time.  Every call that
 *   takes work enqueues it on the CUDA stream given to dir_create (NULL = the
 *   legacy default stream) and, unless it says otherwise, waits for it before
 *   returning.  Device pointers passed in must belong to the current device.
 *
 * Errors
 *   Every int-returning call returns DIR_OK (0) or a negative DIR_E* code and
 *   never throws.  dir_last_error(ctx) describes the last failure on ctx.
 *   After a failed dir_create, *out is NULL.
 */
#ifndef DIR_H
#define DIR_H

#ifdef __cplusplus
extern "C" {
#endif

#define DIR_OK 0
#define DIR_EINVAL (-1)   /* bad argument: NULL pointer, dims, spacing, variant, params */
#define DIR_ENOMEM (-2)   /* device or host allocation failed */
#define DIR_ECUDA (-3)    /* a CUDA call failed; see dir_last_error */
#define DIR_ESTATE (-4)   /* call out of order (e.g. field requested before register) */
#define DIR_EUNSUPPORTED (-5) /* valid request that this build does not implement */
#define DIR_ETIMEOUT (-6)  /* a bounded device-side wait gave up (data copy never landed);
                              the context's results are invalid */

#define DIR_MAX_LEVELS 8
#define DIR_MAX_DIM 4096              /* per axis */
#define DIR_MAX_VOXELS (1LL << 29)    /* nx*ny*nz */

typedef struct dir_ctx dir_ctx;

/* The six force laws (Table 2 numbering minus one). */
typedef enum {
    DIR_PASSIVE = 0,            /* Eq. (1): static-image gradient, computed once per level */
    DIR_EVOLVED_PASSIVE = 1,    /* Eq. (2): also |grad M| of the un-warped moving image */
    DIR_ACTIVE = 2,             /* Eq. (3): gradient of the warped moving image, every iteration */
    DIR_DOUBLE = 3,             /* Eq. (4): passive term plus active term */
    DIR_ADJUSTED_DOUBLE = 4,    /* Eq. (5): Eq. (4) with alpha^2 d^2 in both denominators */
    DIR_INVERSE_CONSISTENT = 5  /* Eq. (6): both images deformed toward a mid-space */
} dir_variant;

/* Element types.  DIR_F16 keeps its number for compatibility of the enum but
   is accepted by no call of this build (DIR_EUNSUPPORTED): images are exact as
   int16 HU, gradients are recomputed in registers and never stored, and a
   half-precision field would sit between DIR_F32 and DIR_BF16 without a use
   the paper's workloads need. */
typedef enum { DIR_F32 = 0, DIR_I16 = 1, DIR_F16 = 2, DIR_BF16 = 3, DIR_F64 = 4 } dir_dtype;

typedef struct {
    int levels;                  /* pyramid depth, 1..DIR_MAX_LEVELS (default 3; the paper uses 2, Sec. 2.3) */
    int iters[DIR_MAX_LEVELS];   /* iterations per level, COARSEST level first (default 200, 100, 50) */
    double sigma;                /* Gaussian sigma in voxels (default 1.0, Sec. 2.5 "unit standard deviation");
                                    the filter radius is ceil(3 sigma), at most 8 */
    double alpha;                /* Eq. (5) normalisation factor (default 0.4) */
    int stop_mode;               /* 0: run iters exactly; 1: also stop a level when
                                    |l(n) - l(n - stop_window)| <= eps (Sec. 2.4), l(n) the
                                    relative norm; 2: the same test on the correlation
                                    coefficient of the warped image with S (the similarity
                                    criterion Sec. 2.4 sets against the relative norm; implies
                                    correlation = 1) */
    double eps;                  /* default 1e-4 (Sec. 2.4) */
    int stop_window;             /* default 10 (Sec. 2.4) */
    dir_dtype field_dtype;       /* storage of the displacement field on the device: DIR_F32
                                    (default) or DIR_BF16 (half the field bytes, arithmetic
                                    still FP32; only with precision DIR_F32) */
    const float* init_field;     /* NULL, or a DEVICE pointer to a level-0 field (3*N floats,
                                    voxels) to start from; only with levels == 1 (DIR_EINVAL
                                    otherwise): the paper starts the coarsest level from
                                    zero (Sec. 2.3) and defines no restriction of a fine
                                    field to the coarse grids, so a starting field is taken
                                    only where it needs none */
    int use_graph;               /* 1 (default): capture the whole registration in a CUDA graph
                                    on the first dir_register and replay it afterwards */
    int timing;                  /* 1: time every force and smoothing launch at the finest level
                                    with CUDA events (reported in dir_stats); default 0 */
    dir_dtype precision;         /* arithmetic and storage of images and fields on the device:
                                    DIR_F32 (default, the production path) or DIR_F64 (double
                                    precision for verification against an FP64 reference; it
                                    runs the plain-load kernels of plain_kernels = 1 in double,
                                    not the TMA-tiled single-precision kernels) */
    int fuse;                    /* iteration schedule (the same field bit for bit in every one).
                                    0: a force kernel, then a smoothing kernel.  1: fused -- the
                                    Gaussian of iteration k folded into the force pass of
                                    iteration k+1 (Eqs. (1)-(2), FP32 images and field, no stop
                                    test), every level.  3: split -- the Gaussian's x and y passes
                                    as their own kernel plane by plane, its z pass inside the
                                    force kernel down each thread's z column (all six laws, FP32
                                    field, float or int16 images, sigma with radius 3, any
                                    stop_mode), every level.  4: as 3, but Eqs. (3)-(6) split
                                    once more after the difference image: a z-pass kernel
                                    writes u and D = W - S once per voxel (Eq. 6: both warped
                                    differences) to a scratch of 4 (Eq. 6: 5) floats per voxel
                                    of the level, and a stencil kernel forms the force from
                                    them, instead of interpolating W on every brick's halo.
                                    2 (default): as 4 where it applies.  dir_register_noalloc
                                    has no scratch for the form of 4: there 2 is split for Eqs.
                                    (1)-(2) on every level and for Eqs. (3)-(6) on levels of at
                                    most 2^21 voxels, else fused on the small levels that one
                                    block per SM covers in two-plane chunks (e.g. 64 x 64 x 25),
                                    else 0, and 4 is 3 */
    int plain_kernels;           /* 0 (default): the production kernels (TMA-fed bricks and
                                    plane rings, packed smoothing, fused small levels).  1: the
                                    plain-load kernels with the same per-voxel arithmetic and
                                    no tiling -- one thread per voxel column reading global
                                    memory, 32 x 8 smoothing tiles, never fused -- in single
                                    precision: a reference for the tiling, halo and ring code
                                    of the production kernels.  Slower; not for production. */
    int correlation;             /* 1: record, every iteration, the correlation coefficient of
                                    the warped moving image with S before the update (Eq. 6:
                                    of the two warped images) with reductions fused into the
                                    force pass (Secs. 2.4, 3.3; dir_get_correlation); 0
                                    (default): not recorded */
    int pdl;                     /* 1 (default): on levels above 2^18 voxels without a stop test,
                                    launch the iteration kernels as programmatic dependent
                                    launches (each starts its setup while the one before
                                    drains); 0: plain launches.  The same field either way */
} dir_params;

typedef struct {
    int levels;
    int iters_run[DIR_MAX_LEVELS];  /* per level, coarsest first */
    double mse_first;               /* mean (W - S)^2 before the first iteration of the finest level */
    double mse_final;               /* the same before the last iteration run */
    double relnorm_final;           /* l(n) = sum|du| / sum|u| of the last iteration run (0 if undefined) */
    float ms_total;                 /* device time of the registration (CUDA events), ms */
    float ms_force_finest;          /* with params.timing: summed force-kernel time at level 0, ms
                                       (the plain force pass: every iteration, or only the first
                                       of a level when the smoothing is fused) */
    float ms_smooth_finest;         /* with params.timing: summed smoothing-kernel time at level 0, ms */
    int n_force_finest;             /* number of launches behind ms_force_finest */
    int n_smooth_finest;
    long long voxel_updates;        /* sum over levels of voxels * iterations run */
    int kernel_launches;            /* kernels launched by the registration (incl. early exits) */
    float ms_fused_finest;          /* with params.timing: summed fused-iteration time at level 0, ms */
    int n_fused_finest;             /* number of launches behind ms_fused_finest */
    int schedule_finest;            /* iteration schedule of level 0: 0 force + smoothing kernels,
                                       1 fused iteration, 2 split Gaussian (fuse = 3), 3 split
                                       with the difference image (fuse = 4); with a split
                                       schedule ms_smooth_finest times the x/y kernel and
                                       ms_force_finest the z + force kernel (3: the z + D and
                                       the stencil force kernels together) */
} dir_stats;

/* Fills *p with the defaults listed above.  Returns DIR_EINVAL if p is NULL. */
int dir_params_default(dir_params* p);

/*
 * Creates a registration context for one static/moving pair: the problem
 * statement of Sec. 2 (register the moving image M to the static image S; the
 * result is a per-voxel displacement field on the static grid, applied to
 * moving-image points as in Sec. 3.2).  Uploads the pair once; the pyramid
 * (Sec. 2.3) is built on the device by dir_register.
 *   static_img, moving_img  dense volumes of image_dtype: DIR_F32, or DIR_I16 (integer
 *                           HU, kept as int16 at the finest level, exact; needs
 *                           precision DIR_F32), host memory, or device memory if
 *                           inputs_on_device != 0.  They are copied; the caller keeps
 *                           ownership.
 *   dims                    {nx, ny, nz}, each 1..DIR_MAX_DIM, nx*ny*nz <= DIR_MAX_VOXELS
 *   spacing_mm              voxel size, each > 0 (used only for mm output)
 *   variant                 one of dir_variant
 *   params                  NULL for defaults
 *   cuda_stream             a cudaStream_t, or NULL for the legacy default stream
 * The context owns all device memory it allocates (sized for the finest level,
 * about 9 floats per voxel plus the pyramid).  Returns DIR_OK and sets *out, or
 * an error and sets *out = NULL.
 */
int dir_create(dir_ctx** out, const void* static_img, const void* moving_img, const int dims[3],
               const float spacing_mm[3], dir_dtype image_dtype, int inputs_on_device,
               dir_variant variant, const dir_params* params, void* cuda_stream);

/*
 * Replaces the image pair of ctx with new volumes of the same dims and dtype
 * (same ownership rules as dir_create), keeping every device buffer and the
 * captured registration graph: a resident context serves the next pair of the
 * same size (the problem statement of Sec. 2 for a new pair).  The field restarts from zero (or
 * init_field) at the next dir_register.
 */
int dir_load(dir_ctx* ctx, const void* static_img, const void* moving_img, dir_dtype image_dtype,
             int on_device);

/*
 * Runs the whole registration: pyramid build (Sec. 2.3), then for each level
 * (coarsest first) the field up-sampling (Sec. 2.3) and the iterations (warp,
 * Sec. 2.5; force and update, Eqs. 1-6; Gaussian smoothing of the total field,
 * Secs. 2.1 and 2.5; reductions and optional stop test, Sec. 2.4), then (for
 * Eq. 6) the inversion of the mid-space field into the static-grid field.  Waits for
 * completion and fills *stats_out if it is not NULL.
 */
int dir_register(dir_ctx* ctx, dir_stats* stats_out);

/* Enqueues the registration on the context's stream and returns without
   waiting.  dir_sync then waits and fills the stats. */
int dir_register_async(dir_ctx* ctx);
int dir_sync(dir_ctx* ctx, dir_stats* stats_out);

/*
 * The result of the registration (Sec. 2: the displacement of every static
 * voxel; Sec. 3.2 applies it to landmark points in mm).
 * Copies the registered static-grid field (3*N floats, planar, dense) to out,
 * a host pointer or, if out_on_device != 0, a device pointer.  in_mm != 0
 * multiplies each component by the voxel spacing of its axis.
 * DIR_ESTATE before the first successful dir_register.
 */
int dir_get_field(dir_ctx* ctx, float* out, int in_mm, int out_on_device);

/* As dir_get_field, but writes doubles (exact for DIR_F64 contexts). */
int dir_get_field_f64(dir_ctx* ctx, double* out, int in_mm, int out_on_device);

/*
 * The quantities of the Sec. 2.4 stopping criterion: the relative norm
 * l(n) = sum|du(n+1)| / sum|u(n)| is out[3t+1] / out[3t+2].
 * Per-iteration reductions of the last registration, in the order run
 * (coarsest level first): out[3*t + 0] = mean (W - S)^2 (for Eq. 6 the mean
 * squared difference of the two warped images), out[3*t + 1] = sum |du|,
 * out[3*t + 2] = sum |u| before the update, all over the voxels of the level
 * at which iteration t ran.  Writes min(max_iters, iterations run) rows to the
 * host array out and returns that count, or a negative error.
 */
int dir_get_history(dir_ctx* ctx, double* out, int max_iters);

/*
 * The correlation coefficient of the warped moving image with S (Eq. 6: of the
 * two warped images) at every iteration of the last registration, before the
 * update, in the order run (coarsest level first): the similarity measure that
 * Sec. 2.4 contrasts with the relative norm and Sec. 3.3 (Fig. 3) plots
 * against the iterations.  Its sums are reduced on the device in the force
 * pass (FP32 within a block, FP64 across blocks); the quotient is formed here.
 * Writes min(max_iters, iterations run) values (NaN where an image is
 * constant) to the host array out and returns that count; DIR_EUNSUPPORTED
 * unless the context was created with correlation = 1 or stop_mode = 2,
 * DIR_ESTATE before the first registration.
 */
int dir_get_correlation(dir_ctx* ctx, double* out, int max_iters);

/*
 * Warps an image on the static grid's dims by the registered field, with the
 * software trilinear interpolation of Sec. 2.5 (clamped coordinates):
 * img_out(x) = img_in(x + u(x)).  With img_in = M this is the deformed moving
 * image that the paper compares with S (Sec. 3.3).  img_in and
 * img_out are dense volumes of dtype dt (DIR_F32 in this build), both host or
 * both device (on_device != 0).
 */
int dir_warp(dir_ctx* ctx, const void* img_in, void* img_out, dir_dtype dt, int on_device);

/*
 * Batched registration: one CUDA graph that runs the registrations of n
 * contexts (each created with dir_create, params.timing 0, none pending),
 * replayed by one graph launch on cuda_stream.  The contexts stay owned by the
 * caller and must outlive the batch; after dir_batch_run each context's field,
 * history and warp are available as after dir_register, bit for bit the same.
 * dir_batch_run waits for the batch and reports its device time in *ms_out
 * (may be NULL).  Multi-job batching of this kind is beyond the paper, which
 * registers one pair at a time (each of its steps runs per pair here too).
 *
 * Two forms:
 *  - grouped (the default where every context allows it: FP32 field, sigma
 *    with radius 3, stop_mode 0, fuse 2 or 3, the same levels and iteration
 *    counts): every iteration of a pyramid level is one x/y launch and one
 *    z + force launch over the bricks of all the contexts at that level (up
 *    to 16 per launch, grouped by force law and image storage) in the split
 *    schedule of params.fuse, so the fixed latencies of a launch are paid
 *    once per step for the whole chunk.  Each chunk runs on its own graph
 *    branch (`branches` is then the number of chunks).  The pyramid, the
 *    first force pass and the last smoothing of each level run per context;
 *  - branches (flags & DIR_BATCH_BRANCHES, or when the contexts do not
 *    qualify): each context's own registration on one of `branches`
 *    concurrent graph branches (longest job first onto the least loaded).
 */
#define DIR_BATCH_BRANCHES 1
typedef struct dir_batch dir_batch;
int dir_batch_create(dir_batch** out, dir_ctx* const* ctxs, int n, int branches, int flags,
                     void* cuda_stream);
int dir_batch_run(dir_batch* batch, float* ms_out);
/* 1 if the batch was captured in the grouped form, 0 for branches, -1 for NULL */
int dir_batch_grouped(const dir_batch* batch);
void dir_batch_destroy(dir_batch* batch);  /* NULL-safe */

/*
 * Launch-shape autotuning for one context, after a finished dir_register:
 * for each pyramid level, times the force kernel with 1, 2, 4 and 8 voxels
 * per thread along z and the smoothing kernel with several z chunks (on
 * levels of the split schedule, the z + force kernel and the x/y kernel)
 * (`reps` launches each), keeps the fastest of each for the context's later
 * registrations (and batches built afterwards), and writes them to
 * shapes_out[2*l], shapes_out[2*l+1] for level l (finest = 0) if not NULL.
 * The registered field is kept.
 */
int dir_autotune(dir_ctx* ctx, int reps, int* shapes_out);

/*
 * Registration that allocates no device memory, for callers that cannot call
 * cudaMalloc while they run: a host whose memory pool owns the whole device, a
 * real-time loop or plug-in callback where allocation is forbidden.  The paper
 * has no counterpart; it is the same pyramid and iterations as dir_create +
 * dir_register + dir_get_field, with every scratch buffer taken from one
 * static device array of 48 MiB that the library reserves on each device it is
 * used on (for as long as the library stays loaded).
 *   static_img, moving_img  DEVICE pointers, dense float volumes of dims
 *   dims                    {nx, ny, nz}; the pyramid, two fields and the
 *                           reduction rows must fit the 48 MiB (about 1.5 M
 *                           voxels in single precision with 3 levels, e.g.
 *                           128 x 128 x 90; half that in DIR_F64);
 *                           larger requests fail with DIR_EINVAL and a message
 *                           in dir_last_error(NULL), before any device work
 *   params                  as for dir_create; timing must be 0; use_graph is
 *                           ignored (kernels are launched directly)
 *   field_out               DEVICE pointer, 3*N floats: the static-grid field in voxels
 *   stats_out               NULL, or iterations run and voxel-updates
 * The first call on a device looks up the array's device address (no
 * allocation), so make it before capturing the stream into a CUDA graph.  The
 * work runs on cuda_stream and the call waits for it.  Every call shares the
 * array: calls whose work could overlap on the GPU (other streams or threads)
 * race and must be serialised by the caller.
 */
int dir_register_noalloc(const float* static_img, const float* moving_img, const int dims[3],
                         dir_variant variant, const dir_params* params, float* field_out,
                         void* cuda_stream, dir_stats* stats_out);

/*
 * Exercises the failure path of the bounded device-side waits that every
 * TMA-fed kernel of the library uses (a kernel whose copy never lands gives
 * up, flags the context's error word and returns; the call then reports
 * DIR_ETIMEOUT).  One block waits on a shared-memory mbarrier that nothing
 * completes -- no copy is involved and nothing faults -- for limit_ms, gives
 * up, and records that in a device word that the call reads back.
 *   cuda_stream  a cudaStream_t, or NULL for the legacy default stream
 *   limit_ms     how long the wait lasts before it gives up, 1 .. 2000
 * Returns DIR_ETIMEOUT when the wait gave up as designed (the expected
 * outcome; the device stays usable), DIR_EINVAL for a limit out of range,
 * DIR_ECUDA on a CUDA error, DIR_OK if the wait were ever satisfied.
 * Waits for the stream.
 */
int dir_check_wait_timeout(void* cuda_stream, double limit_ms);

/* Frees ctx and everything it owns.  NULL-safe. */
void dir_destroy(dir_ctx* ctx);

/* Static description of a status code. */
const char* dir_status_string(int status);

/* Description of the last failure on ctx (empty if none); ctx may be NULL for
   the last dir_create failure of this thread. */
const char* dir_last_error(const dir_ctx* ctx);

/* Library build identifier (compute capability targeted, version). */
const char* dir_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DIR_H */
