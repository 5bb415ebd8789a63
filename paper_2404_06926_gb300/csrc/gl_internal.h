// gl_internal.h -- host-side internals shared by the translation units of the
// library: grow-only device buffers, the per-view context and the kernel
// launchers.  Not part of the public ABI (include/gl_map.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gl_common.cuh"
#include "../../include/gl_map.h"

namespace gl {

void set_error(const std::string& msg);

#define GL_CUDA_TRY(expr)                                                         \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) {                                                  \
            ::gl::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));  \
            return _e == cudaErrorMemoryAllocation ? GL_ERR_OOM : GL_ERR_CUDA;     \
        }                                                                         \
    } while (0)

#define GL_TRY(expr)                         \
    do {                                     \
        gl_status _s = (expr);               \
        if (_s != GL_OK) return _s;          \
    } while (0)

// Kernel launch accounting (process-wide).
void count_launches(int64_t n);

// Streaming multiprocessors of the current device (looked up once per device).
int sm_count();

// Raise the dynamic shared-memory limit of kernel `fn` to `bytes` on the
// current device, once per (kernel, device); safe from several host threads.
gl_status ensure_smem_limit(const void* fn, int bytes);

// Phases timed by the optional CUDA-event profiler.
enum Phase {
    PH_PREPROCESS = 0, PH_DEPTH_SORT, PH_SCAN_DUP, PH_TILE_SORT, PH_RANGES, PH_RASTER_FWD, PH_LOSS,
    PH_RASTER_BWD, PH_PARAMS, PH_EXPAND, PH_COUNT
};

// Event-pair timers: begin/end record events on the stream; harvest() waits
// for them and accumulates elapsed time per phase.  Events are pooled.
struct Prof {
    bool on = false;
    struct Pending { int phase; cudaEvent_t a, b; };
    Pending* pend = nullptr;
    int npend = 0, cap = 0;
    cudaEvent_t* pool = nullptr;
    int npool = 0, poolcap = 0;
    double ms[PH_COUNT] = {0};
    int64_t calls[PH_COUNT] = {0};
    cudaEvent_t begin(cudaStream_t s);
    void end(int phase, cudaEvent_t a, cudaStream_t s);
    void harvest();
    void reset();
    void prefill(int count);
    void release();
};

// RAII bracket of one phase (no-op when the profiler is off or null).
struct PhaseScope {
    Prof* p;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseScope(Prof* p_, int ph, cudaStream_t s_) : p(p_), phase(ph), s(s_)
    {
        if (p && p->on) a = p->begin(s);
    }
    void close()
    {
        if (p && p->on && a) p->end(phase, a, s);
        p = nullptr;
    }
    ~PhaseScope() { close(); }
};

// Grow-only device allocation.  Contents are not preserved on growth.
// While a thread captures a CUDA graph (AllocFreeze in scope) a reserve that
// would have to grow fails with GL_ERR_CAPACITY instead of reallocating a
// buffer that captured work already points at.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    gl_status reserve(size_t need);
    void release();
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

struct AllocFreeze {
    AllocFreeze();
    ~AllocFreeze();
};
bool alloc_frozen();

constexpr int kMaxViews = 64;   // views in one step (a keyframe window)
constexpr int kDescRing = 8;    // pinned upload slots for view descriptors

// Per-view inputs of the loss and the exposure update, set by the caller.
struct ViewExtra {
    const float* target = nullptr;
    float* E = nullptr;
    float* Em = nullptr;
    float e_bc1 = 1.f, e_bc2 = 1.f;
    float weight = 1.f;
};

// Per-step scalars uploaded with the view descriptors (read on the device by
// steps replayed from a CUDA graph).
struct StepScalars {
    float ibc1 = 1.f, isbc2 = 1.f;   // Adam bias corrections 1/(1-b1^t), 1/sqrt(1-b2^t)
    float pad[14] = {};
};
static_assert(sizeof(StepScalars) == 64, "descriptor block layout");

// Scratch of one step over V views: projected records (per view and
// Gaussian, index v * n + g), binning over the concatenated tiles of all
// views, and per-pixel state over the concatenated pixels.
struct View {
    int V = 0;
    int64_t n = 0;            // Gaussians (per view)
    int Ts = 16, ntiles = 0, nltiles = 0;   // totals over the views
    int64_t P = 0;            // pixels over the views
    int W = 0, H = 0, TX = 0, TY = 0;       // view 0 (single-view helpers)
    Cam cam{};                // view 0
    int64_t I = 0;            // (Gaussian, tile) instances over the views
    ViewDesc hdesc[kMaxViews];
    StepScalars hscal;
    DevBuf desc;              // device copy of [hscal][hdesc[0..V)]
    char* hpin = nullptr;     // pinned upload ring (kDescRing blocks of that layout)
    cudaEvent_t pin_ev[kDescRing] = {};
    bool pin_used[kDescRing] = {};
    int pin_slot = 0;
    // per (view, Gaussian)
    DevBuf rec0, rec1, rec2, rec3;  // float4: (u,v,A',C'), (B',log2 o,z,o), (r,g,b,-), alpha box
    DevBuf radius;            // int
    DevBuf rect;              // int4 (x0,y0,x1,y1), tiles local to the view
    DevBuf touched;           // u32
    DevBuf dkey, gidx;        // u32 depth key (sort input); u32 index (sort output buffer)
    DevBuf dkey2, gidx2;      // sort ping-pong
    DevBuf dup_off;           // u32 offset of the Gaussian's first instance
    DevBuf kmask;             // u64 kept-tile mask of the rectangle (all ones if it is not culled)
    DevBuf g2d;               // float[10] screen-space gradient accumulators
    // scan
    DevBuf bsum;              // u64 per scan block: instance offset, then duplication-part offset
    DevBuf count;             // u64[16]: I (0 after an overflow), overflow flag, N (depth
                              // sort), instances needed, view-count scratch [4..5],
                              // work items [6], segment items [7], bounded device
                              // waits that gave up [8] (bit 0: radix-sort look-back,
                              // bit 1: parameter staging; sticky until
                              // sort_wait_status reads it), Gaussians left after
                              // the depth sort drops the culled ones [9],
                              // duplication parts [10]
    // per instance
    DevBuf itile, ival, itile2, ival2;  // u32 global tile id, u32 instance id (sort; input ids implied)
    DevBuf iowner;            // u32 owning (view, Gaussian) per instance id
    DevBuf srec0, srec1, srec2, srec3;  // records in sorted-instance order
    DevBuf sgid;              // u32 owning (view, Gaussian) per sorted instance
    DevBuf hist;              // radix histograms
    DevBuf ranges;            // uint2 per global tile
    DevBuf tile_order;        // u32 tile launch order (heaviest first)
    // per pixel (concatenated over views)
    DevBuf Tfin, ncon;        // float, u32
    DevBuf rgb, depth, opac;  // internal render targets when needed
    // sorted-order results of the last forward (pointers into the buffers above)
    const uint32_t* sorted_g = nullptr;
    const uint32_t* sorted_tile = nullptr;
    const uint32_t* sorted_inst = nullptr;
    uint64_t* h_count = nullptr;          // pinned copy of count[0..8]
    Prof* prof = nullptr;                 // optional phase timers
    // raster execution: records per lane per batch (1: 32, 2: 64), pixels per
    // lane (1, 2, 4), persistent grid with a unit counter in `work`
    int nb = 1, pd = 1;
    bool persistent = false;
    DevBuf work;              // int[2] unit counters (forward, backward)
    // deterministic backward: per (instance, pixel block) sums, reduced per
    // (view, Gaussian) in a fixed order (floats: instances x blocks x 10)
    bool det = false;
    DevBuf gpart;
    // segmented raster: tiles whose list holds >= 2 seg records are split
    // into segments of seg records (seg a power of two; 0: never split)
    int seg = 0;
    // exact tile culling: only tiles where the Gaussian can reach alpha >=
    // 1/255 at a pixel centre get an instance
    bool cull = true;
    // per-Gaussian backward: lanes own Gaussians, pixel states travel the warp
    bool pg = false;
    DevBuf items;             // uint2 per work item: (tile, segment), heaviest first
    DevBuf segstate;          // 8 floats per (segment item, pixel of its tile), see gl_raster.cu
    const ViewDesc* d_desc() const
    {
        return reinterpret_cast<const ViewDesc*>(desc.as<const char>() + sizeof(StepScalars));
    }
    const float* d_scal() const { return desc.as<const float>(); }
    static constexpr size_t kDescBlock = sizeof(StepScalars) + sizeof(ViewDesc) * kMaxViews;
    // Fill hdesc and the tile / pixel totals for V views (host only).
    void set_views(const Cam* cams, const ViewExtra* extra, int V, int Ts);
    gl_status init();
    gl_status upload_descs(cudaStream_t s);
    void release();
};

struct gl_ctx_impl {
    cudaStream_t stream = nullptr;
    View view;
    gl_exec_config exec{0, 0, 32, 1, 0, 0, 0, 1, 0};
    DevBuf pose_part;   // per-block pose partials
    DevBuf loss_part;   // per-block loss partials
    float pose_jac[36] = {};   // J_l of the last forward's twist (row-major 6 x 6)
    int has_forward = 0;
    int deg = 0;
};

// ---------------------------------------------------------------------------
// Launchers (each returns GL_OK or an error; all work on `stream`).
// ---------------------------------------------------------------------------

// Describe V views (cameras, tiles, pixel offsets, loss inputs), upload the
// descriptors, then preprocess + depth sort + scan + duplicate + tile sort +
// ranges + tile order + record permutation over all of them.  Synchronises
// once to size the instance buffers.
// sync_free: the descriptors were set and uploaded by the caller (set_views,
// upload_descs) and nothing is read back: instances beyond the current
// capacity set the overflow flag (count[1]), every later kernel of the step
// sees zero instances, and the Adam updates skip themselves; the caller
// checks the flag after the step.  Used for steps captured in a CUDA graph.
gl_status bin_views(View& v, const GParams& p, const Cam* cams, const ViewExtra* extra, int V, int Ts,
                    cudaStream_t s, bool sync_free = false);
// The single-view case.
gl_status bin_view(View& v, const GParams& p, const Cam& cam, int Ts, cudaStream_t s);

// Forward raster of a binned view into (rgb, depth, opacity) device images
// (depth/opacity may be null) plus T_final / n_contrib in `v`.
// extras: also blend depth and opacity (needed for those outputs and for a
// later backward with depth or opacity gradients on split tiles).
gl_status raster_forward(View& v, float* rgb, float* depth, float* opac, cudaStream_t s, bool extras = true);

// Upper bound of the work items of a binned step (every tile once, plus one
// per seg records of the instance capacity).
int64_t work_items_bound(const View& v);
// Build the work items of a binned step (after the tile order).
gl_status build_items(View& v, cudaStream_t s);

// Records gathered into sorted-instance order (after binning).
// nmax bounds the instance count (which is read on the device).
gl_status permute_records(View& v, int64_t nmax, cudaStream_t s);

// Backward raster: per-Gaussian screen-space gradients into v.g2d.
gl_status raster_backward(View& v, const float* dL_drgb, const float* dL_ddepth,
                          const float* dL_dopac, cudaStream_t s);

// Chain rule from per-instance 2-D gradients to parameters.
struct AdamArgs {
    GMut m, v;                 // moments
    float lr_pos, lr_dc, lr_rest, lr_op, lr_scale, lr_rot;
    float b1, b2, eps, ibc1, isbc2;  // 1/(1-b1^t), 1/sqrt(1-b2^t)
    int sparse;
    const float* bc = nullptr;       // if set: (ibc1, isbc2) read on the device
    const uint64_t* abort = nullptr; // if set and abort[1] != 0: no update
};
// mode 0: write gradients into `grad` (+ pose partials if pose_part != null).
gl_status params_backward(View& v, const GParams& p, GMut grad, float* pose_part, int npart,
                          cudaStream_t s);
// mode 1: fused Adam update of `upd` (same storage as p) with moments.
gl_status params_adam(View& v, const GParams& p, GMut upd, const AdamArgs& a, cudaStream_t s);
int pose_partials_needed(int64_t n);
// Sum the per-block pose partials (the gradient g of a left perturbation of
// the rendered pose) and write J^T g, J the 6 x 6 row-major left Jacobian of
// the forward's twist (the identity for a zero twist).
gl_status pose_reduce(const float* part, int npart, const float jac[36], float* out6, cudaStream_t s);

// Photometric loss (Eq. 9) of one view given by value (no descriptor upload):
// writes dL/drgb and per-tile partials; then the final reduction writes loss
// and dL/dE.
int loss_partials_needed(int W, int H);
gl_status photometric_loss(const float* rgb, const float* target, const float* E, int W, int H,
                           float lambda, float* dL_drgb, float* part, float* loss_out,
                           float* dE_out, cudaStream_t s);
// The same over all views of `v` (targets, exposures and weights from the
// descriptors): dL/drgb over the concatenated pixels (already weighted),
// loss per view into loss_v[V], and the exposure Adam step of views with Em.
// With abort set and abort[1] != 0, the exposure update is skipped.
gl_status photometric_loss_views(const View& v, const float* rgb, float lambda, float* dL_drgb, float* part,
                                 float* loss_v, float b1, float b2, float eps, float lr, cudaStream_t s,
                                 const uint64_t* abort = nullptr);

// Apply C_hat = A C + b (E34 by value) from src to dst (device images).
gl_status apply_exposure(const float* src, float* dst, const float E[12], int64_t P,
                         cudaStream_t s);

// Stable radix sort of (u32 key, u32 value) pairs over bits [0, bits); n on
// the device, at most n_max; scratch sized for max(n_max, n_reserve) keys;
// ctl[8] is raised if a look-back wait gave up.  Returns in *out_k/*out_v the
// buffers holding the result.  index_values: the input values are 0..n-1 and
// v0 is not read (it still serves as an output buffer).  n_kept (device, may
// be null): keys 0xffffffff are dropped from the result, whose length is
// written to *n_kept.
gl_status radix_sort_u32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                         const uint64_t* n_dev, int64_t n_max, int64_t n_reserve, int bits, DevBuf& scratch,
                         uint64_t* ctl, uint32_t** out_k, uint32_t** out_v, cudaStream_t s,
                         bool index_values = false, uint64_t* n_kept = nullptr);
// Bytes of the counters copied to View::h_count (count[0..8]).
constexpr size_t kCountCopy = 9 * sizeof(uint64_t);
// GL_ERR_TIMEOUT (once) if a radix-sort pass gave up a look-back wait, as
// seen in the host copy of the counters taken before the caller's last
// synchronisation; GL_OK otherwise.
gl_status sort_wait_status(View& v, cudaStream_t s);
// Runs one sort pass whose look-back can never complete (see
// gl_selftest_bounded_wait); *expired = 1 if it gave up and raised its flag.
gl_status sort_wait_selftest(int32_t* expired);

// Add the counts of the step just enqueued on `v` to acc[0..4) on the device
// (no synchronisation): visible (view, Gaussian) pairs, instances,
// contributor sum over the pixels, pixels.
gl_status accumulate_view_counts(const View& v, uint64_t* acc, cudaStream_t s);

// Visible Gaussians and the summed contributor count of the last view.
gl_status view_counts(const View& v, int64_t* n_visible, int64_t* sum_contrib, cudaStream_t s);

// Projected quantities of the last view in plain form (null outputs skipped).
gl_status export_preprocess(const View& v, float* mean2d, float* conic, float* opacity, float* rgb,
                            float* depth, cudaStream_t s);

// Sorted instances as (tile << 32 | depth bits) keys and owning Gaussians.
gl_status export_instances(const View& v, uint64_t* keys, uint32_t* vals, cudaStream_t s);

// The map's raster execution knobs (batch depth, pixels per lane,
// persistence, segment length; pixels per lane capped by the tile size Ts)
// applied to another view's scratch.
void map_exec_knobs(const gl_map* m, View& v, int Ts);

// Validated camera of a pose and intrinsics (finite pose, positive focal
// lengths, image size 1..16384); GL_ERR_INVALID otherwise.
gl_status camera_from(const gl_pose* pose, const gl_intrinsics* K, Cam& cam);

// Hooks into a map for the serving loop (the map's own code is in gl_capi.cu).
cudaStream_t map_stream(const gl_map* m);
int map_sh_degree(const gl_map* m);
int map_tile_size(const gl_map* m);
int64_t map_size_now(const gl_map* m);
int64_t map_capacity(const gl_map* m);
// Copy the live Gaussians into dst[0..5) (means, log-scales, quats, logits,
// SH; grown as needed) on the map's stream, then record `done` there.
gl_status map_snapshot(gl_map* m, DevBuf* dst, int64_t* n_out, cudaEvent_t done);
GParams snapshot_params(const gl_map* m, const DevBuf* src, int64_t n);
// Registered keyframes that hold an image, by ascending id (image = null).
void map_keyframes(const gl_map* m, std::vector<gl_keyframe>& out);

// Map-side kernels.
gl_status sky_create(float* means, float* log_scales, float* quats, float* logits, float* sh,
                     int K, int64_t n, double radius, uint64_t seed, float opacity,
                     cudaStream_t s);
gl_status expand_points(const float* xyz, const float* rgb, int64_t n, const Cam& cam,
                        const float* opacity_map, float tau, int use_mask, float opacity_fg,
                        int K, GMut dst, int64_t dst_offset, int64_t dst_cap, DevBuf& flags,
                        DevBuf& scan, int64_t* n_added, cudaStream_t s);

}  // namespace gl
