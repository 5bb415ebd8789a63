/*
 * gl_map.h -- C ABI of the GB300 optimiser of the Gaussian-LIC photo-realistic
 * map (arXiv 2404.06926, Sec. III-A and III-C).
 *
 * One optimisation step for one keyframe view is: project every Gaussian
 * (Eq. 1-3) and colour it from its SH; bin it into screen tiles with
 * (tile | depth) keys and a device radix sort; composite each tile front to
 * back (Eq. 4-7); apply the view's 3x4 exposure affine; score the L1 + D-SSIM
 * loss (Eq. 9); back-propagate to every Gaussian attribute (and to the camera
 * pose and the exposure); and apply Adam, optionally only to the Gaussians
 * visible in the view (sparse Adam, Sec. III-D 2).
 *
 * Conventions shared by every call:
 *   - Every entry point returns gl_status; GL_OK is 0.  Nothing aborts.  On
 *     failure gl_last_error() returns a thread-local message.
 *   - Poses are world->camera: x_c = R_cw x_w + t_cw (Eq. 2), R_cw row-major.
 *   - Intrinsics are a pinhole (Eq. 2's pi_c) on undistorted images: pixel
 *     (u, v) has its centre at integer coordinates (u, v).
 *   - Images are H x W x 3 float RGB (row-major, channel last).
 *   - Quaternions are (w, x, y, z) and need not be unit length.
 *   - Pointers documented "device" must be CUDA device memory of the current
 *     device; "host or device" pointers are classified with
 *     cudaPointerGetAttributes.  The caller owns every buffer it passes; the
 *     library copies whatever it keeps beyond the call.
 *   - Work is enqueued on the stream given at creation; calls return once the
 *     work is enqueued unless they copy results to host memory, in which case
 *     they synchronise that stream first.
 *   - An object (gl_map, gl_ctx) is used by one host thread at a time.
 */
#ifndef GL_MAP_H
#define GL_MAP_H

#include <stdint.h>

#if defined(__GNUC__)
#define GL_API __attribute__((visibility("default")))
#else
#define GL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GL_OK = 0,
    GL_ERR_INVALID = 1,   /* bad argument: NaN/Inf pose, non-positive focal, bad size */
    GL_ERR_OOM = 2,       /* device allocation failed                                 */
    GL_ERR_CUDA = 3,      /* a CUDA call failed (message in gl_last_error)            */
    GL_ERR_CAPACITY = 4,  /* more than 2^32-1 (Gaussian, tile) instances in one view  */
    GL_ERR_TIMEOUT = 5,   /* a bounded device wait gave up                            */
    GL_ERR_BUSY = 6,      /* the serving queue is full                                */
    GL_ERR_NOT_FOUND = 7  /* unknown keyframe id                                      */
} gl_status;

/* Pinhole intrinsics pi_c (Eq. 2). */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
} gl_intrinsics;

/* Camera pose {R_cw, t_cw}, world -> camera (Eq. 2). */
typedef struct {
    float R_cw[9];
    float t_cw[3];
} gl_pose;

/* A keyframe as the mapping module receives it (Sec. III-C): an id, a pose,
 * intrinsics and an undistorted image.  `image` is H*W*3 float RGB in [0,1],
 * host or device; it may be NULL in gl_optimize_step when the id was
 * registered with gl_map_add_keyframe, whose stored copy is then used. */
typedef struct {
    int64_t id;
    gl_pose pose;
    gl_intrinsics K;
    const float* image;
} gl_keyframe;

/* Hyper-parameters.  The paper's values (Sec. IV-A): lambda = 0.2,
 * tau = 0.99, o_a = 0.1, o_b = 0.7, R = 1e4, N_s = 1e5; learning rates "as
 * vanilla 3DGS, not decayed".  gl_config_default() fills every field. */
typedef struct {
    int32_t sh_degree;      /* 0..3 (the paper uses 3)                      */
    int32_t tile_size;      /* 8, 16 or 32                                  */
    int32_t sparse_adam;    /* 1: Adam touches only Gaussians visible in the
                               step's views; 0: all Gaussians ("w/o acc")  */
    int32_t reserved0;
    uint64_t seed;          /* sky sampling (SplitMix64 counter generator)  */
    float lambda_dssim, tau, opacity_fg, opacity_sky, sky_radius;
    int32_t reserved1;
    int64_t n_sky;          /* sky Gaussians created by gl_map_create       */
    float lr_pos, lr_sh_dc, lr_sh_rest, lr_opacity, lr_scale, lr_rot, lr_exposure;
    float adam_b1, adam_b2, adam_eps;
    int64_t capacity_hint;  /* initial Gaussian capacity                    */
    float lr_window_exp;    /* Gaussian learning rates of an n-view window
                               step are scaled by n^lr_window_exp: 0 keeps
                               the paper's rates for any window (default);
                               0.5 is square-root scaling for the mean
                               gradient's lower variance.  Not in the paper. */
    int32_t reserved2;
} gl_config;

/* Gaussian parameters in caller memory, one array per attribute, row-major:
 * means n*3, log_scales n*3, quats n*4 (w,x,y,z), logits n (opacity =
 * sigmoid(logit)), sh n*K*3 with K = (sh_degree+1)^2, coefficient-major and
 * channel-minor (Sec. III-A: position, scale, rotation, opacity, SH).  Each
 * array starts on a 16-byte boundary (GL_ERR_INVALID otherwise). */
typedef struct {
    int64_t n;
    int32_t sh_degree;
    int32_t reserved;
    float* means;
    float* log_scales;
    float* quats;
    float* logits;
    float* sh;
} gl_gaussians;

/* ---------------------------------------------------------------------- */
/* Library                                                                 */
/* ---------------------------------------------------------------------- */

/* Thread-local message of the last failing call on this thread ("" if none). */
GL_API const char* gl_last_error(void);

/* ABI version of this header (major * 100 + minor). */
GL_API int32_t gl_version(void);

/* Fill `cfg` with the paper's values and the proposed readings of the
 * constants it leaves open (tile 16, SH degree 3, sparse Adam on). */
GL_API gl_status gl_config_default(gl_config* cfg);

/* ---------------------------------------------------------------------- */
/* Map API (Sec. III-C)                                                    */
/* ---------------------------------------------------------------------- */
typedef struct gl_map gl_map;

/* Create a map on the current device; `cuda_stream` (cudaStream_t, may be
 * NULL for the legacy default stream) orders all of its work.  Creates
 * cfg->n_sky sky Gaussians (Sec. III-C 1): points uniform by area on the
 * upper hemisphere (z >= 0) of radius cfg->sky_radius about the origin,
 * white DC colour, opacity o_b, isotropic scale = distance to the nearest
 * other sky point.  The map owns all device state and releases it in
 * gl_map_destroy.  Errors: GL_ERR_INVALID (bad config), GL_ERR_OOM. */
GL_API gl_status gl_map_create(const gl_config* cfg, void* cuda_stream, gl_map** out);

/* Release every device allocation of the map (after its stream drains). */
GL_API gl_status gl_map_destroy(gl_map* map);

/* Number of Gaussians in the map. */
GL_API gl_status gl_map_size(gl_map* map, int64_t* n_out);

/* Map initialisation and expansion (Sec. III-C 1-2, Eq. 8).  xyz and rgb
 * are n*3 floats (host or device) of coloured LiDAR / visual points in the
 * world frame.  Each kept point becomes a Gaussian centred on it with SH DC
 * from its colour, higher SH zero, opacity o_a, identity rotation and
 * isotropic scale d/f (d = depth in `pose`, f = K->fx).  Points at depth
 * <= 0.2 m are never kept.  use_mask = 0 keeps every other point (the first
 * frame); use_mask = 1 renders the opacity map O (Eq. 7) from (pose, K) and
 * keeps a point only if it lands inside the image on a pixel (nearest pixel
 * centre) with O < cfg->tau.  `kind` (0 LiDAR, 1 visual) is recorded per
 * Gaussian.  New Gaussians start with zero Adam moments.  *n_added (host)
 * receives the number kept.  Errors: GL_ERR_INVALID, GL_ERR_OOM. */
GL_API gl_status gl_map_add_points(gl_map* map, const float* xyz, const float* rgb, int64_t n,
                            int32_t kind, const gl_pose* pose, const gl_intrinsics* K,
                            int32_t use_mask, int64_t* n_added);

/* Register a keyframe: copies its image to device memory owned by the map
 * and creates its exposure E = [I | 0] (Sec. III-C 3).  Re-registering an
 * id replaces its image and pose and keeps its exposure. */
GL_API gl_status gl_map_add_keyframe(gl_map* map, const gl_keyframe* kf);

/* Render the map from (pose, K) (Eq. 5-7).  E34 (host, 12 floats, row-major
 * [A | b]) applies C_hat = A C + b to the colour; NULL means identity.
 * out_rgb (H*W*3), out_depth (H*W, nullable) and out_opacity (H*W,
 * nullable) are host or device. */
GL_API gl_status gl_render(gl_map* map, const gl_pose* pose, const gl_intrinsics* K, const float* E34,
                    float* out_rgb, float* out_depth, float* out_opacity);

/* One optimisation step (Sec. III-C 3, Eq. 9).  n_views = 1 is the paper's
 * single-view step: forward, loss with the view's exposure, backward, Adam
 * on the Gaussians (sparse or dense per the config) and on the view's
 * exposure.  n_views > 1 renders and back-propagates all views as one
 * window and takes one Adam step on the mean of their losses.  out_loss
 * (host, nullable) receives the mean loss.  Images in host memory (pinned
 * or pageable) are copied to the device on a stream of the map's own while
 * the step's binning and forward run, and only the loss waits for them;
 * the call returns when the step is done, so the caller may reuse them
 * then.  Errors: GL_ERR_INVALID, GL_ERR_NOT_FOUND (image NULL and id not
 * registered), GL_ERR_CAPACITY. */
GL_API gl_status gl_optimize_step(gl_map* map, const gl_keyframe* views, int32_t n_views,
                           float* out_loss);

/* How optimisation steps execute (none of this is in the paper; none of it
 * changes a result except tile_size, which sets the binning tiles and so
 * the 3-sigma tile rectangles of Sec. III-A):
 *   use_graphs       1: after one eager step of a given shape (views and
 *                    their sizes, map size, the fields below) the step is
 *                    captured into a CUDA graph and later steps of that
 *                    shape replay it.  Binning then reads nothing back: the
 *                    instance buffers keep 25% headroom, a step whose
 *                    instances do not fit updates nothing, is detected when
 *                    the replay ends and is re-run eagerly (growing them).
 *                    Graph steps synchronise the map's stream once, at the
 *                    end.  Ignored while timers are on.
 *   persistent       1: both raster kernels run one grid of resident warps
 *                    that take (tile, pixel block) units from a counter.
 *   batch_depth      records a warp stages per batch: 32, 64, 128 or 256
 *                    (128 and 256 take one pixel per lane).
 *   pixels_per_lane  1, 2 or 4 pixels of a column per lane; 4 x this must
 *                    not exceed the tile size.
 *   tile_size        0: gl_config's; else 8, 16 or 32.
 *   deterministic    1: the backward writes each pixel block's sums per
 *                    (Gaussian, tile) instance and adds them per Gaussian
 *                    in a fixed order instead of with float atomics, so a
 *                    step's results are bit-identical from run to run (at
 *                    the cost of one more pass over 40 bytes per instance
 *                    and pixel block); batch_depth is then 32.
 *   exact_cull       1 (default): a (Gaussian, tile) pair of the 3-sigma
 *                    rectangle gets an instance only if the Gaussian can
 *                    reach alpha >= 1/255 at a pixel centre of the tile
 *                    (closed-form minimum of its quadratic form over the
 *                    tile, with a 2^-7 slack); renders are bit-identical
 *                    either way, the instance lists (and contributor
 *                    positions) shorter.
 *   segment          0, or a power of two in 64..65536: a tile whose list
 *                    holds at least 2 x segment Gaussians is rendered and
 *                    back-propagated as segments of `segment` consecutive
 *                    Gaussians by separate warps; the transmittance is then
 *                    a product of per-segment products, equal to the
 *                    single running product up to float rounding.
 *   per_gaussian     1: per-Gaussian backward (Sec. III-D 1): each lane
 *                    of a warp owns Gaussians of the pixel block's list and
 *                    sums their gradients in its registers while the
 *                    pixels' transmittance and blended colour pass from
 *                    lane to lane; 0: per-pixel backward (lanes own pixels,
 *                    each Gaussian's sums folded across the warp).  The
 *                    per-Gaussian backward works on 8 x 4 pixel blocks with
 *                    32-record batches whatever pixels_per_lane and
 *                    batch_depth say (those still drive the forward).
 * Apart from deterministic = 1, results differ between runs only by the
 * order of the backward's float atomics.
 * gl_map_create starts with {0, 0, 32, 1, 0, 0, 0, 1, 0}.  Errors: GL_ERR_INVALID. */
typedef struct {
    int32_t use_graphs;
    int32_t persistent;
    int32_t batch_depth;
    int32_t pixels_per_lane;
    int32_t tile_size;
    int32_t deterministic;
    int32_t segment;
    int32_t exact_cull;
    int32_t per_gaussian;
} gl_exec_config;

GL_API gl_status gl_map_set_exec(gl_map* map, const gl_exec_config* exec);
GL_API gl_status gl_map_get_exec(gl_map* map, gl_exec_config* exec);

/* Autotuner: `views` holds n_views / window windows of `window` views each
 * (as gl_optimize_step takes them; several windows make the timing
 * representative of steps over different views).  Coordinate descent from
 * {graphs, persistent, batch depth 32, 1 pixel per lane, segment 1024,
 * per-pixel backward}: the tile size (8/16/32), the segment length
 * (0/256/512/1024), persistence, the batch depth (32/64/128/256), the pixels per
 * lane (1/2/4) and the backward (per pixel / per Gaussian) in turn take the
 * value whose `reps` rounds of one step per window are fastest (CUDA
 * events) with the other knobs fixed; deterministic and exact_cull stay as
 * set.  The Gaussians, their Adam moments, the views' exposures and the
 * step counters are put back after each trial.  With keep_tile_size != 0 only
 * gl_config's tile size is tried.  The fastest candidate is installed with
 * gl_map_set_exec and returned in *best, its device time per step in
 * *best_ms (nullable).  The map ends as it started.  Errors: as
 * gl_optimize_step; GL_ERR_INVALID if n_views is not 1..64 whole windows;
 * GL_ERR_OOM for the state snapshot. */
GL_API gl_status gl_map_autotune(gl_map* map, const gl_keyframe* views, int32_t n_views, int32_t window,
                                 int32_t reps, int32_t keep_tile_size, gl_exec_config* best, float* best_ms);

/* Change the configuration of an existing map: learning rates, Adam
 * constants, lambda_dssim, tau, opacity_fg, sparse_adam, tile_size and
 * lr_window_exp take effect from the next call; sh_degree must equal the
 * map's; seed, n_sky, sky_radius, opacity_sky and capacity_hint only act at
 * creation and are kept.  Errors: GL_ERR_INVALID (the map is unchanged). */
GL_API gl_status gl_map_set_config(gl_map* map, const gl_config* cfg);
GL_API gl_status gl_map_get_config(gl_map* map, gl_config* cfg);

/* Checkpoint (not in the paper): the whole optimisation state -- the
 * Gaussians and their kinds (LiDAR, visual, sky), both Adam moments, the
 * Adam step counter, and every keyframe (id, pose, intrinsics, exposure E
 * with its Adam moments and step count, and its stored image when
 * with_images != 0) -- in one host byte buffer: a header (magic "GLMAPCK1",
 * version 1, SH degree, counts), the parameter arrays, the moments, the
 * kinds, then the keyframes by ascending id; little-endian, as both target
 * hosts are.  gl_map_checkpoint_size gives the bytes gl_map_save writes.
 * gl_map_load replaces the map's contents with such a buffer (same SH
 * degree); it validates the whole buffer first and leaves the map untouched
 * on GL_ERR_INVALID.  Pageable or pinned host memory; synchronous.
 * Errors: GL_ERR_INVALID (null, short buffer, wrong magic/version/degree,
 * bad keyframe camera), GL_ERR_OOM. */
GL_API gl_status gl_map_checkpoint_size(gl_map* map, int32_t with_images, int64_t* bytes);
GL_API gl_status gl_map_save(gl_map* map, int32_t with_images, void* host_buf, int64_t bytes);
GL_API gl_status gl_map_load(gl_map* map, const void* host_buf, int64_t bytes);

/* Copy the Gaussians (out->n must be >= the map size; pointers host or
 * device; out->sh_degree must equal the map's).  *n_out gets the size. */
GL_API gl_status gl_map_get_params(gl_map* map, gl_gaussians* out, int64_t* n_out);

/* Replace all Gaussians with `in` (host or device) and zero Adam state. */
GL_API gl_status gl_map_set_params(gl_map* map, const gl_gaussians* in);

/* Copy Adam's first (which = 1) or second (which = 2) moments. */
GL_API gl_status gl_map_get_moments(gl_map* map, int32_t which, gl_gaussians* out);

/* Exposure E (12 floats, host) of keyframe `id`. */
GL_API gl_status gl_map_get_exposure(gl_map* map, int64_t id, float* E34_out);

/* ---------------------------------------------------------------------- */
/* Instrumentation (not in the paper, which reports only run times,      */
/* Table II): per-phase CUDA-event timers and counts of the last view.    */
/* ---------------------------------------------------------------------- */
#define GL_NUM_PHASES 10

typedef struct {
    int64_t n_gaussians;   /* map size                                          */
    int64_t n_visible;     /* Gaussians with a non-zero screen radius, last view */
    int64_t n_instances;   /* (Gaussian, tile) instances of the last view        */
    int64_t sum_contrib;   /* sum over pixels of the contributor count, i.e. the
                              (pixel, Gaussian) pairs the backward walks         */
    int64_t pixels;        /* pixels of the last view                           */
    int64_t steps;         /* optimisation steps taken (Adam step counter)      */
    double phase_ms[GL_NUM_PHASES];     /* summed device time per phase         */
    int64_t phase_calls[GL_NUM_PHASES]; /* timed launches per phase             */
    int64_t graph_captures;  /* step graphs captured                             */
    int64_t graph_replays;   /* steps run by replaying a graph                   */
    int64_t graph_reruns;    /* replays whose instances overflowed (re-run eagerly) */
    /* Summed over the steps taken since the timers were last switched on (the
     * steps whose phases phase_ms times), over all their views:            */
    int64_t timed_steps;     /* steps                                             */
    int64_t timed_views;     /* views                                             */
    int64_t timed_visible;   /* (view, Gaussian) pairs with a non-zero radius     */
    int64_t timed_instances; /* (Gaussian, tile) instances                        */
    int64_t timed_contrib;   /* (pixel, Gaussian) pairs the backward walks        */
    int64_t timed_pixels;    /* pixels                                            */
} gl_stats;

/* Turn the per-phase timers on (1) or off (0); either way they restart from
 * zero.  When on, every phase of every call is bracketed by CUDA events on
 * the map's stream (no extra synchronisation). */
GL_API gl_status gl_map_set_timing(gl_map* map, int32_t enable);

/* Counts of the last rendered view, the accumulated phase times and the
 * counts summed over the timed steps.  Synchronises the map's stream. */
GL_API gl_status gl_map_get_stats(gl_map* map, gl_stats* out);

/* Name of phase i (0 <= i < GL_NUM_PHASES), e.g. "raster_backward". */
GL_API const char* gl_phase_name(int32_t i);

/* Number of kernels this library has launched in this process so far. */
GL_API int64_t gl_kernel_launch_count(void);

/* Self-test of the bounded device waits (no GPU fault, no hang): runs one
 * radix-sort scatter pass as the CTA of tile 1 of a two-tile sort whose tile
 * 0 is never published, so its look-back wait has nothing to find and must
 * give up after its poll limit (about a second).  *expired (host) receives
 * 1 if the pass gave up and raised its flag, 0 otherwise; the pass writes
 * only its own scratch buffers, which are freed before returning.
 * Synchronous; uses device 0's current context.  Errors: GL_ERR_INVALID
 * (null expired), GL_ERR_OOM, GL_ERR_CUDA. */
GL_API gl_status gl_selftest_bounded_wait(int32_t* expired);

/* ---------------------------------------------------------------------- */
/* Serving loop (not in the paper, which runs the mapping thread of        */
/* Sec. III-C beside tracking): a request loop over one map that keeps    */
/* the map on the device, serialises the requests that change it and      */
/* batches novel-view renders.                                             */
/*                                                                         */
/* Mutating requests (KEYFRAME_UPDATE, OPTIMIZE) run on the map's stream   */
/* in submission order; each one that succeeds commits a new map version   */
/* (1, 2, ...; 0 is the map as the server found it).  After each commit    */
/* the Gaussians are copied into one of two snapshot buffers.  RENDER      */
/* requests read the snapshot of the latest committed version at the time */
/* they are admitted; all renders admitted together (up to                 */
/* render_batch) are rendered by one multi-view launch on the server's own */
/* stream, so their work overlaps the mutations' on the device.  A        */
/* request is admitted only while the device has free memory for it (its  */
/* estimated need plus reserve_bytes); it waits otherwise and fails with   */
/* GL_ERR_OOM only if it cannot fit with nothing else in flight.           */
/*                                                                         */
/* KEYFRAME_UPDATE (Sec. III-C 2-3): add the points through the opacity     */
/* mask of the keyframe's view (gl_map_add_points, use_mask = 1, or all    */
/* points if the map is empty), register the keyframe (gl_map_add_keyframe) */
/* and take n_steps optimisation steps.  OPTIMIZE: n_steps steps.  Each     */
/* step uses `window` distinct registered keyframes (1 = the plain step),  */
/* drawn by a SplitMix64 counter generator seeded with `seed` over the     */
/* registered ids in ascending order, so a request's steps depend only on */
/* the map version it starts from and its own fields.                      */
/* ---------------------------------------------------------------------- */
typedef struct gl_server gl_server;

enum { GL_REQ_KEYFRAME_UPDATE = 1, GL_REQ_OPTIMIZE = 2, GL_REQ_RENDER = 3 };

typedef struct {
    int32_t queue_capacity;      /* pending requests before GL_ERR_BUSY (default 256)  */
    int32_t render_batch;        /* renders per batched launch (default 8, <= 64)       */
    int64_t reserve_bytes;       /* device memory kept free (default 1 GiB)             */
    int32_t record_versions;     /* 1: keep a checkpoint (gl_map_save layout, with      */
                                 /*    images) of every committed version, for tests    */
    int32_t max_gaussians;       /* > 0: keyframe updates add at most this many minus   */
                                 /*    the map size (a prefix of their points); 0: no cap */
} gl_server_config;

typedef struct {
    int32_t kind;                /* GL_REQ_*                                            */
    int32_t n_steps;             /* optimisation steps (KEYFRAME_UPDATE, OPTIMIZE)      */
    int32_t window;              /* keyframes per step (>= 1)                           */
    int32_t point_kind;          /* 0 LiDAR, 1 visual (KEYFRAME_UPDATE)                 */
    uint64_t seed;               /* keyframe sampling                                   */
    const float* xyz;            /* KEYFRAME_UPDATE: n_points * 3, host; copied at      */
    const float* rgb;            /*   submission                                        */
    int64_t n_points;
    gl_keyframe keyframe;        /* KEYFRAME_UPDATE: id, pose, K, host image (copied);  */
                                 /* RENDER: pose and K (image ignored)                  */
    float* out_rgb;              /* RENDER: H*W*3, host or device, written before the   */
                                 /*   request completes; caller keeps it valid          */
} gl_request;

typedef struct {
    int32_t status;              /* gl_status of the request                            */
    int32_t kind;
    int64_t version;             /* RENDER: version read; others: version committed     */
    double t_submit, t_admit, t_done;   /* seconds since gl_server_create               */
    float loss;                  /* mean loss of the request's last optimisation step   */
    int32_t batch;               /* RENDER: renders in its launch                       */
    int64_t n_added;             /* KEYFRAME_UPDATE: Gaussians added                    */
} gl_result;

typedef struct {
    int64_t submitted[4], completed[4], failed[4];   /* indexed by GL_REQ_* (0 unused)   */
    double p50_ms[4], p99_ms[4], mean_ms[4];         /* latency submit -> done           */
    int64_t steps;               /* optimisation steps taken                            */
    double steps_per_s;          /* steps / (last completion - first submission)        */
    double renders_per_s;
    double mean_render_batch;
    int64_t memory_waits;        /* admissions deferred for device memory               */
    int64_t busy_rejects;        /* submissions refused with GL_ERR_BUSY                */
    int64_t version;             /* latest committed version                            */
    int64_t map_size;
    int64_t points_capped;       /* points left out by max_gaussians                    */
} gl_server_stats;

/* gl_server_config_default fills the defaults above. */
GL_API gl_status gl_server_config_default(gl_server_config* cfg);
/* Start the loop's two worker threads over `map`.  While the server lives,
 * the map must not be used directly.  Errors: GL_ERR_INVALID, GL_ERR_OOM. */
GL_API gl_status gl_server_create(gl_map* map, const gl_server_config* cfg, gl_server** out);
/* Queue a request; *ticket identifies it.  Errors: GL_ERR_INVALID (bad
 * request), GL_ERR_BUSY (queue full). */
GL_API gl_status gl_server_submit(gl_server* srv, const gl_request* req, uint64_t* ticket);
/* Wait up to timeout_s seconds (< 0: forever) for a request and take its
 * result (each ticket can be taken once).  Errors: GL_ERR_TIMEOUT,
 * GL_ERR_NOT_FOUND (unknown or already taken). */
GL_API gl_status gl_server_wait(gl_server* srv, uint64_t ticket, double timeout_s, gl_result* out);
/* Wait until every submitted request has completed. */
GL_API gl_status gl_server_drain(gl_server* srv);
GL_API gl_status gl_server_get_stats(gl_server* srv, gl_server_stats* out);
/* With record_versions: the checkpoint of committed version v (v = 0 is
 * the map as the server found it).  *bytes gets its size; buf (nullable)
 * receives it if cap is large enough.  Errors: GL_ERR_NOT_FOUND. */
GL_API gl_status gl_server_get_version(gl_server* srv, int64_t v, void* buf, int64_t cap, int64_t* bytes);
/* Drain, stop the workers and free the server (not the map). */
GL_API gl_status gl_server_destroy(gl_server* srv);

/* ---------------------------------------------------------------------- */
/* Stateless differentiable API (one view), for autograd wrappers and     */
/* tests.  A gl_ctx owns the scratch of one forward/backward pair.         */
/* ---------------------------------------------------------------------- */
typedef struct gl_ctx gl_ctx;

GL_API gl_status gl_ctx_create(void* cuda_stream, gl_ctx** out);
GL_API gl_status gl_ctx_destroy(gl_ctx* ctx);

/* Raster execution of this context's calls: batch_depth, pixels_per_lane,
 * persistent, deterministic, segment, exact_cull and per_gaussian as in
 * gl_exec_config (defaults 32, 1, 0, 0, 0, 1, 0; use_graphs
 * and tile_size are ignored: the tile size is each call's argument).  A
 * pixels_per_lane above tile_size / 4 is lowered to it.  Errors:
 * GL_ERR_INVALID. */
GL_API gl_status gl_ctx_set_exec(gl_ctx* ctx, const gl_exec_config* exec);

/* Forward (Eq. 1-7) of the Gaussians `g` (device arrays) seen from the pose
 * exp(xi^) T_cw with T_cw = `pose` and xi = twist6 (host, 6 floats: a
 * twist (rho, phi), translation part first; NULL means xi = 0, i.e. `pose`
 * itself), with square tiles of side tile_size (8, 16 or 32).  exp is the
 * SE(3) exponential, evaluated in double precision inside the library.
 * Writes the device images out_rgb (H*W*3), out_depth (H*W, nullable) and
 * out_opacity (H*W, nullable), and keeps the per-view state (records,
 * sorted instances, per-pixel final transmittance and contributor count)
 * in `ctx` for gl_rasterize_backward.  Errors: GL_ERR_INVALID (also for a
 * non-finite twist), GL_ERR_CAPACITY, GL_ERR_OOM. */
GL_API gl_status gl_rasterize_forward(gl_ctx* ctx, const gl_gaussians* g, const gl_pose* pose,
                                      const float* twist6, const gl_intrinsics* K, int32_t tile_size,
                                      float* out_rgb, float* out_depth, float* out_opacity);

/* Backward of the last gl_rasterize_forward on `ctx` (same `g`, unchanged).
 * dL_drgb (H*W*3, device) is required; dL_ddepth and dL_dopacity (H*W,
 * device) may be NULL.  Per-pixel transmittance is recomputed from the
 * stored final value, not stored per pair.  Writes gradients for every
 * attribute into `grad` (device arrays shaped like `g`; Gaussians outside
 * the view get 0) and, if grad_pose6 (device, 6 floats) is not NULL, the
 * gradient dL/dxi w.r.t. the forward's twist: J_l(xi)^T g, where g is the
 * gradient w.r.t. a left perturbation d of the rendered pose,
 * exp(d^) exp(xi^) T_cw, at d = 0, and J_l the SE(3) left Jacobian (so at
 * xi = 0 it is g itself). */
GL_API gl_status gl_rasterize_backward(gl_ctx* ctx, const gl_gaussians* g, const float* dL_drgb,
                                       const float* dL_ddepth, const float* dL_dopacity,
                                       gl_gaussians* grad, float* grad_pose6);

/* Photometric loss, Eq. 9: L = (1-lambda) mean|E[C] - C_bar| + lambda
 * (1 - mean SSIM(E[C], C_bar)), SSIM with an 11x11 Gaussian window of
 * sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2, averaged over pixels
 * and channels.  rgb, target (H*W*3), E34 (12) are device.  Writes the
 * device scalar loss_out (1 float; may be NULL), the device gradients
 * dL_drgb (H*W*3; required) and dL_dE (12; may be NULL). */
GL_API gl_status gl_photometric_loss(gl_ctx* ctx, const float* rgb, const float* target, const float* E34,
                              int32_t width, int32_t height, float lambda_dssim,
                              float* loss_out, float* dL_drgb, float* dL_dE);

/* The photometric loss above without any device allocation.  The paper has
 * no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory while they run: a real-time tracking or serving
 * thread for which cudaMalloc's implicit device-wide synchronisation would
 * stall the other work on the GPU, or a process whose device memory is all
 * owned by another allocator (a framework's caching allocator, a fixed
 * memory budget).  Arguments and results are those of gl_photometric_loss
 * (loss_out and dL_dE may be NULL, dL_drgb is required), with the stream
 * passed directly (cudaStream_t, NULL for the legacy default stream)
 * instead of through a gl_ctx.
 * Scratch: the per-tile partial sums live in one fixed array inside the
 * library (917,504 bytes), which every GPU that loads the library holds
 * until the process exits.  Limit: at most 16,384 tiles of 32x32 pixels
 * (e.g. 4096 x 4096); larger images are rejected with GL_ERR_INVALID before
 * any work is enqueued.  First call on each device: it looks up the array's
 * device address and raises the loss kernel's shared-memory limit, and the
 * CUDA runtime loads the library's device code (with the array) on that
 * device if nothing has loaded it yet -- a one-time allocation made by the
 * runtime, not by this call.  Make that first call at set-up, before any
 * real-time section and before any stream capture; later calls allocate
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 * All calls share the array, which keeps the last call's contents; calls
 * that overlap on the GPU (on different streams, or from different threads)
 * race on it, so serialise them. */
GL_API gl_status gl_photometric_loss_noalloc(const float* rgb, const float* target, const float* E34,
                                             int32_t width, int32_t height, float lambda_dssim,
                                             float* loss_out, float* dL_drgb, float* dL_dE,
                                             void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Introspection of the last forward on a ctx (tests; not a user API).     */
/* All outputs are device arrays; n = number of Gaussians of the forward.  */
/* ---------------------------------------------------------------------- */

/* radius (n int32), rect (n*4 int32: x0, y0, x1, y1 tiles, half open),
 * mean2d (n*2), conic (n*3: A, B, C of Sigma'^-1), opacity (n), rgb (n*3),
 * depth (n).  Any pointer may be NULL. */
GL_API gl_status gl_ctx_get_preprocess(gl_ctx* ctx, int32_t* radius, int32_t* rect, float* mean2d,
                                float* conic, float* opacity, float* rgb, float* depth);

/* Number of (Gaussian, tile) instances of the last forward (host out). */
GL_API gl_status gl_ctx_num_instances(gl_ctx* ctx, int64_t* I_out);

/* Sorted instances: keys (I u64, tile << 32 | float bits of depth), vals
 * (I u32 Gaussian index) and ranges (num_tiles * 2 u32, [start, end)). */
GL_API gl_status gl_ctx_get_instances(gl_ctx* ctx, uint64_t* keys, uint32_t* vals, uint32_t* ranges);

/* Per-pixel final transmittance (H*W float) and contributor count (H*W
 * u32: 1 + position, in the tile's list, of the last Gaussian blended). */
GL_API gl_status gl_ctx_get_pixel_state(gl_ctx* ctx, float* T_final, uint32_t* n_contrib);

#ifdef __cplusplus
}
#endif
#endif /* GL_MAP_H */
