// gl_server.cu -- the serving loop over one map: a mutation worker that runs
// keyframe updates and optimisation requests in submission order on the
// map's stream, and a render worker that renders every admitted novel view
// of the latest committed version in one multi-view launch on its own
// stream.  Snapshots of the Gaussians (two buffers) decouple the two, so
// the device runs renders while the map is being optimised.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "gl_internal.h"

using namespace gl;

namespace {

constexpr int kKinds = 4;

struct Req {
    uint64_t ticket = 0;
    gl_request r{};
    std::vector<float> xyz, rgb, image;   // owned copies of the caller's host/device data
    double t_submit = 0.0, t_admit = 0.0;
};

struct Snap {
    DevBuf arr[5];
    int64_t n = 0;
    int64_t version = -1;
    int readers = 0;
    cudaEvent_t ready = nullptr;
};

// SplitMix64 (Steele, Lea and Flood, 2014): state += golden gamma, then the
// variant-13 finaliser.
uint64_t splitmix64(uint64_t& s)
{
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Copy n floats from host or device memory into a host vector.
gl_status take_copy(const float* src, size_t n, std::vector<float>& dst)
{
    dst.resize(n);
    if (n == 0) return GL_OK;
    cudaPointerAttributes a{};
    const bool dev = cudaPointerGetAttributes(&a, src) == cudaSuccess &&
                     (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev) {
        GL_CUDA_TRY(cudaMemcpy(dst.data(), src, 4 * n, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(dst.data(), src, 4 * n);
    }
    return GL_OK;
}

double pct(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q / 100.0 * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct gl_server {
    gl_map* map = nullptr;
    gl_server_config cfg{};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req*> mut_q, ren_q;
    std::unordered_map<uint64_t, gl_result> done;
    std::unordered_set<uint64_t> open;       // submitted, result not yet taken
    uint64_t next_ticket = 1;
    int64_t pending = 0;                      // submitted, not completed
    bool stop = false;
    Snap snap[2];
    int latest = -1;
    int64_t version = 0;
    std::vector<std::vector<uint8_t>> versions;
    // admitted work in flight, for memory admission (a worker still waiting
    // for admission does not count: two waiting workers would otherwise wait
    // for each other)
    int mut_running = 0, ren_running = 0;
    double mut_scratch_hw = 0.0, ren_scratch_hw = 0.0;   // largest scratch estimates admitted
    double inst_per_px = 2.0;                              // instances per pixel, from the last render
    // statistics
    std::vector<double> lat[kKinds];
    int64_t submitted[kKinds] = {}, completed[kKinds] = {}, failed[kKinds] = {};
    int64_t steps = 0, renders = 0, render_batches = 0, memory_waits = 0, busy_rejects = 0, points_capped = 0;
    double first_submit = -1.0, last_done = 0.0;
    // render side
    cudaStream_t rstream = nullptr;
    View rview;
    DevBuf rgb;
    std::thread tm, tr;
    int device = 0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

size_t free_bytes()
{
    size_t f = 0, t = 0;
    if (cudaMemGetInfo(&f, &t) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return f;
}

// Device bytes per Gaussian for parameters + both moments.
double bytes_per_gaussian(int deg)
{
    const int K = (deg + 1) * (deg + 1);
    return 3.0 * 4.0 * (3 + 3 + 4 + 1 + 3 * K);
}

// Scratch of one step over views of P pixels in total (per-(view, Gaussian)
// records and binning, per-instance and per-pixel buffers).
double step_scratch(double views, double n, double P, double inst_per_px)
{
    return views * n * 170.0 + P * 110.0 + inst_per_px * P * 1.25 * 90.0;
}

void finish(gl_server* s, Req* q, const gl_result& res)
{
    std::lock_guard<std::mutex> lk(s->mu);
    const int k = q->r.kind;
    if (res.status == GL_OK) {
        s->completed[k]++;
        s->lat[k].push_back((res.t_done - res.t_submit) * 1e3);
    } else {
        s->failed[k]++;
    }
    s->last_done = std::max(s->last_done, res.t_done);
    s->done[q->ticket] = res;
    s->pending--;
    delete q;
    s->cv.notify_all();
}

// Admission: wait until the device has `need` bytes beyond the reserve free.
// Returns false when it cannot fit while the other worker has no admitted
// work in flight (nothing will be freed), or after 30 s.  On true the
// caller's worker counts as running.
bool admit_memory(gl_server* s, double need, bool render_side)
{
    const double deadline = s->now() + 30.0;
    for (;;) {
        const double f = (double)free_bytes();
        std::unique_lock<std::mutex> lk(s->mu);
        if (f >= need + (double)s->cfg.reserve_bytes) {
            (render_side ? s->ren_running : s->mut_running)++;
            return true;
        }
        const bool others = render_side ? s->mut_running > 0 : s->ren_running > 0;
        if (!others || s->now() > deadline) return false;
        s->memory_waits++;
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

gl_status publish(gl_server* s)
{
    int slot;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        slot = s->latest < 0 ? 0 : 1 - s->latest;
        s->cv.wait(lk, [&] { return s->snap[slot].readers == 0; });
    }
    int64_t n = 0;
    GL_TRY(map_snapshot(s->map, s->snap[slot].arr, &n, s->snap[slot].ready));
    std::lock_guard<std::mutex> lk(s->mu);
    s->snap[slot].n = n;
    s->snap[slot].version = s->version;
    s->latest = slot;
    s->cv.notify_all();
    return GL_OK;
}

gl_status record_version(gl_server* s)
{
    if (!s->cfg.record_versions) return GL_OK;
    int64_t b = 0;
    GL_TRY(gl_map_checkpoint_size(s->map, 1, &b));
    std::vector<uint8_t> buf((size_t)b);
    GL_TRY(gl_map_save(s->map, 1, buf.data(), b));
    std::lock_guard<std::mutex> lk(s->mu);
    s->versions.push_back(std::move(buf));
    return GL_OK;
}

gl_status run_steps(gl_server* s, const gl_request& r, float* loss)
{
    if (r.n_steps <= 0) return GL_OK;
    std::vector<gl_keyframe> kfs;
    map_keyframes(s->map, kfs);
    if (kfs.empty()) { set_error("no keyframe with an image to optimise on"); return GL_ERR_NOT_FOUND; }
    const int K = (int)kfs.size();
    const int w = std::min(r.window, K);
    std::vector<int> idx(K);
    std::vector<gl_keyframe> views(w);
    uint64_t st = r.seed;
    for (int i = 0; i < r.n_steps; i++) {
        for (int j = 0; j < K; j++) idx[j] = j;
        for (int j = 0; j < w; j++) {   // partial Fisher-Yates draw of w distinct keyframes
            const int pick = j + (int)(splitmix64(st) % (uint64_t)(K - j));
            std::swap(idx[j], idx[pick]);
            views[j] = kfs[idx[j]];
        }
        GL_TRY(gl_optimize_step(s->map, views.data(), w, loss));
        std::lock_guard<std::mutex> lk(s->mu);
        s->steps++;
    }
    return GL_OK;
}

gl_status run_mutation(gl_server* s, Req* q, gl_result& res)
{
    const gl_request& r = q->r;
    if (r.kind == GL_REQ_KEYFRAME_UPDATE) {
        const gl_keyframe& kf = r.keyframe;
        int64_t added = 0;
        int64_t np = r.n_points;
        if (s->cfg.max_gaussians > 0) {
            const int64_t room = std::max<int64_t>(0, (int64_t)s->cfg.max_gaussians - map_size_now(s->map));
            if (np > room) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->points_capped += np - room;
                np = room;
            }
        }
        if (np > 0) {
            const int use_mask = map_size_now(s->map) > 0 ? 1 : 0;
            GL_TRY(gl_map_add_points(s->map, q->xyz.data(), q->rgb.data(), np, r.point_kind, &kf.pose, &kf.K,
                                     use_mask, &added));
        }
        res.n_added = added;
        gl_keyframe k = kf;
        k.image = q->image.data();
        GL_TRY(gl_map_add_keyframe(s->map, &k));
    }
    float loss = 0.f;
    GL_TRY(run_steps(s, r, r.n_steps > 0 ? &loss : nullptr));
    res.loss = loss;
    return GL_OK;
}

void mutation_worker(gl_server* s)
{
    cudaSetDevice(s->device);
    const int deg = map_sh_degree(s->map);
    for (;;) {
        Req* q;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->mut_q.empty(); });
            if (s->mut_q.empty()) return;
            q = s->mut_q.front();
        }
        const gl_request& r = q->r;
        // bytes this request may allocate: map growth (capacity doubles),
        // its keyframe image and expansion scratch, and step scratch beyond
        // what earlier requests already grew
        const double n = (double)map_size_now(s->map);
        const double cap = (double)map_capacity(s->map);
        double need = 0.0;
        if (r.kind == GL_REQ_KEYFRAME_UPDATE) {
            if (n + (double)r.n_points > cap)
                need += std::max(n + (double)r.n_points, 2.0 * cap) * bytes_per_gaussian(deg);
            need += 12.0 * r.keyframe.K.width * r.keyframe.K.height + 40.0 * (double)r.n_points;
        }
        const double P = r.kind == GL_REQ_KEYFRAME_UPDATE ? (double)r.keyframe.K.width * r.keyframe.K.height
                                                          : 1280.0 * 1024.0;
        const double scratch = step_scratch(r.window, n + (double)r.n_points, P * r.window, s->inst_per_px);
        need += std::max(0.0, scratch - s->mut_scratch_hw);
        gl_result res{};
        res.kind = r.kind;
        res.t_submit = q->t_submit;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->mut_q.pop_front();
        }
        const bool fits = admit_memory(s, need, false);
        res.t_admit = s->now();
        gl_status st = GL_OK;
        if (!fits) {
            set_error("request does not fit in device memory");
            st = GL_ERR_OOM;
        } else {
            s->mut_scratch_hw = std::max(s->mut_scratch_hw, scratch);
            st = run_mutation(s, q, res);
            if (st == GL_OK) {
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->version++;
                    res.version = s->version;
                }
                st = publish(s);
                if (st == GL_OK) st = record_version(s);
            }
        }
        if (fits) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->mut_running--;
            s->cv.notify_all();
        }
        res.status = st;
        res.t_done = s->now();
        finish(s, q, res);
    }
}

void render_worker(gl_server* s)
{
    cudaSetDevice(s->device);
    const int Ts = map_tile_size(s->map);
    for (;;) {
        std::vector<Req*> batch;
        int slot = -1;
        int64_t ver = 0;
        double need = 0.0, scratch = 0.0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->ren_q.empty(); });
            if (s->ren_q.empty()) return;
            const int take = std::min<int>((int)s->ren_q.size(), s->cfg.render_batch);
            for (int i = 0; i < take; i++) {
                batch.push_back(s->ren_q.front());
                s->ren_q.pop_front();
            }
        }
        double P = 0.0;
        for (Req* q : batch) P += (double)q->r.keyframe.K.width * q->r.keyframe.K.height;
        const double n = (double)map_size_now(s->map);
        scratch = step_scratch((double)batch.size(), n, P, s->inst_per_px) + 12.0 * P;
        need = std::max(0.0, scratch - s->ren_scratch_hw);
        const bool fits = admit_memory(s, need, true);
        const double t_admit = s->now();
        gl_status st = GL_OK;
        if (!fits) {
            set_error("render batch does not fit in device memory");
            st = GL_ERR_OOM;
        } else {
            std::lock_guard<std::mutex> lk(s->mu);
            slot = s->latest;
            s->snap[slot].readers++;
            ver = s->snap[slot].version;
        }
        if (st == GL_OK) {
            s->ren_scratch_hw = std::max(s->ren_scratch_hw, scratch);
            const int V = (int)batch.size();
            std::vector<Cam> cams(V);
            for (int i = 0; i < V; i++) camera_from(&batch[i]->r.keyframe.pose, &batch[i]->r.keyframe.K, cams[i]);
            const GParams p = snapshot_params(s->map, s->snap[slot].arr, s->snap[slot].n);
            st = cudaStreamWaitEvent(s->rstream, s->snap[slot].ready, 0) == cudaSuccess ? GL_OK : GL_ERR_CUDA;
            if (st == GL_OK) st = s->rgb.reserve(12 * (size_t)P);
            map_exec_knobs(s->map, s->rview, Ts);
            if (st == GL_OK) st = bin_views(s->rview, p, cams.data(), nullptr, V, Ts, s->rstream);
            if (st == GL_OK) st = raster_forward(s->rview, s->rgb.as<float>(), nullptr, nullptr, s->rstream, false);
            size_t off = 0;
            for (int i = 0; i < V && st == GL_OK; i++) {
                const size_t b = 12 * (size_t)cams[i].W * cams[i].H;
                if (cudaMemcpyAsync(batch[i]->r.out_rgb, s->rgb.as<char>() + off, b, cudaMemcpyDefault,
                                    s->rstream) != cudaSuccess)
                    st = GL_ERR_CUDA;
                off += b;
            }
            if (cudaStreamSynchronize(s->rstream) != cudaSuccess && st == GL_OK) st = GL_ERR_CUDA;
            if (st == GL_OK) st = sort_wait_status(s->rview, s->rstream);
            if (st == GL_ERR_CUDA) {
                set_error(cudaGetErrorString(cudaGetLastError()));
            } else if (P > 0 && s->rview.I > 0) {
                s->inst_per_px = std::max(0.5, (double)s->rview.I / P);
            }
            std::lock_guard<std::mutex> lk(s->mu);
            s->snap[slot].readers--;
            s->renders += V;
            s->render_batches++;
            s->cv.notify_all();
        }
        if (fits) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->ren_running--;
            s->cv.notify_all();
        }
        const double t_done = s->now();
        for (Req* q : batch) {
            gl_result res{};
            res.kind = GL_REQ_RENDER;
            res.status = st;
            res.version = ver;
            res.t_submit = q->t_submit;
            res.t_admit = t_admit;
            res.t_done = t_done;
            res.batch = (int32_t)batch.size();
            finish(s, q, res);
        }
    }
}

}  // namespace

extern "C" gl_status gl_server_config_default(gl_server_config* c)
{
    if (!c) { set_error("null argument"); return GL_ERR_INVALID; }
    std::memset(c, 0, sizeof(*c));
    c->queue_capacity = 256;
    c->render_batch = 8;
    c->reserve_bytes = int64_t(1) << 30;
    c->record_versions = 0;
    return GL_OK;
}

extern "C" gl_status gl_server_create(gl_map* map, const gl_server_config* cfg, gl_server** out)
{
    if (!map || !out) { set_error("null argument"); return GL_ERR_INVALID; }
    gl_server_config c;
    if (cfg) c = *cfg;
    else gl_server_config_default(&c);
    if (c.queue_capacity < 1 || c.render_batch < 1 || c.render_batch > kMaxViews || c.reserve_bytes < 0 ||
        c.max_gaussians < 0) {
        set_error("invalid server config");
        return GL_ERR_INVALID;
    }
    std::unique_ptr<gl_server> s(new gl_server());
    s->map = map;
    s->cfg = c;
    s->t0 = std::chrono::steady_clock::now();
    GL_CUDA_TRY(cudaGetDevice(&s->device));
    // renders are latency-bound and small: their stream gets the highest
    // priority, so their CTAs go first whenever SM slots free up
    int prio_lo = 0, prio_hi = 0;
    GL_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    GL_CUDA_TRY(cudaStreamCreateWithPriority(&s->rstream, cudaStreamNonBlocking, prio_hi));
    for (Snap& sn : s->snap) GL_CUDA_TRY(cudaEventCreateWithFlags(&sn.ready, cudaEventDisableTiming));
    GL_TRY(s->rview.init());
    GL_TRY(publish(s.get()));
    GL_TRY(record_version(s.get()));
    GL_CUDA_TRY(cudaStreamSynchronize(map_stream(map)));
    gl_server* raw = s.release();
    raw->tm = std::thread(mutation_worker, raw);
    raw->tr = std::thread(render_worker, raw);
    *out = raw;
    return GL_OK;
}

extern "C" gl_status gl_server_submit(gl_server* s, const gl_request* req, uint64_t* ticket)
{
    if (!s || !req || !ticket) { set_error("null argument"); return GL_ERR_INVALID; }
    const gl_request& r = *req;
    if (r.kind != GL_REQ_KEYFRAME_UPDATE && r.kind != GL_REQ_OPTIMIZE && r.kind != GL_REQ_RENDER) {
        set_error("unknown request kind");
        return GL_ERR_INVALID;
    }
    if (r.kind != GL_REQ_RENDER && (r.n_steps < 0 || r.window < 1 || r.window > kMaxViews)) {
        set_error("n_steps must be >= 0 and window in 1..64");
        return GL_ERR_INVALID;
    }
    if (r.kind != GL_REQ_OPTIMIZE) {
        Cam c;
        GL_TRY(camera_from(&r.keyframe.pose, &r.keyframe.K, c));
    }
    if (r.kind == GL_REQ_RENDER && !r.out_rgb) { set_error("render needs out_rgb"); return GL_ERR_INVALID; }
    if (r.kind == GL_REQ_KEYFRAME_UPDATE) {
        if (r.n_points < 0 || (r.n_points > 0 && (!r.xyz || !r.rgb)) || !r.keyframe.image ||
            (r.point_kind != 0 && r.point_kind != 1)) {
            set_error("keyframe update needs points (n >= 0, kind 0/1) and an image");
            return GL_ERR_INVALID;
        }
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->pending >= s->cfg.queue_capacity) {
            s->busy_rejects++;
            set_error("serving queue is full");
            return GL_ERR_BUSY;
        }
    }
    std::unique_ptr<Req> q(new Req());
    q->r = r;
    if (r.kind == GL_REQ_KEYFRAME_UPDATE) {
        GL_TRY(take_copy(r.xyz, 3 * (size_t)r.n_points, q->xyz));
        GL_TRY(take_copy(r.rgb, 3 * (size_t)r.n_points, q->rgb));
        GL_TRY(take_copy(r.keyframe.image, 3 * (size_t)r.keyframe.K.width * r.keyframe.K.height, q->image));
        q->r.xyz = q->r.rgb = nullptr;
        q->r.keyframe.image = nullptr;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->pending >= s->cfg.queue_capacity) {
        s->busy_rejects++;
        set_error("serving queue is full");
        return GL_ERR_BUSY;
    }
    q->ticket = s->next_ticket++;
    q->t_submit = s->now();
    if (s->first_submit < 0) s->first_submit = q->t_submit;
    s->submitted[r.kind]++;
    s->pending++;
    s->open.insert(q->ticket);
    *ticket = q->ticket;
    if (r.kind == GL_REQ_RENDER) s->ren_q.push_back(q.release());
    else s->mut_q.push_back(q.release());
    s->cv.notify_all();
    return GL_OK;
}

extern "C" gl_status gl_server_wait(gl_server* s, uint64_t ticket, double timeout_s, gl_result* out)
{
    if (!s || !out) { set_error("null argument"); return GL_ERR_INVALID; }
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->open.count(ticket)) { set_error("unknown ticket or result already taken"); return GL_ERR_NOT_FOUND; }
    auto ready = [&] { return s->done.count(ticket) > 0; };
    if (timeout_s < 0) {
        s->cv.wait(lk, ready);
    } else if (!s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        set_error("request still running");
        return GL_ERR_TIMEOUT;
    }
    *out = s->done[ticket];
    s->done.erase(ticket);
    s->open.erase(ticket);
    return GL_OK;
}

extern "C" gl_status gl_server_drain(gl_server* s)
{
    if (!s) { set_error("null argument"); return GL_ERR_INVALID; }
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait(lk, [&] { return s->pending == 0; });
    return GL_OK;
}

extern "C" gl_status gl_server_get_stats(gl_server* s, gl_server_stats* out)
{
    if (!s || !out) { set_error("null argument"); return GL_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    for (int k = 0; k < kKinds; k++) {
        out->submitted[k] = s->submitted[k];
        out->completed[k] = s->completed[k];
        out->failed[k] = s->failed[k];
        out->p50_ms[k] = pct(s->lat[k], 50.0);
        out->p99_ms[k] = pct(s->lat[k], 99.0);
        double sum = 0.0;
        for (double x : s->lat[k]) sum += x;
        out->mean_ms[k] = s->lat[k].empty() ? 0.0 : sum / (double)s->lat[k].size();
    }
    const double span = s->first_submit >= 0 ? s->last_done - s->first_submit : 0.0;
    out->steps = s->steps;
    out->steps_per_s = span > 0 ? (double)s->steps / span : 0.0;
    out->renders_per_s = span > 0 ? (double)s->renders / span : 0.0;
    out->mean_render_batch = s->render_batches ? (double)s->renders / (double)s->render_batches : 0.0;
    out->memory_waits = s->memory_waits;
    out->busy_rejects = s->busy_rejects;
    out->version = s->version;
    out->map_size = map_size_now(s->map);
    out->points_capped = s->points_capped;
    return GL_OK;
}

extern "C" gl_status gl_server_get_version(gl_server* s, int64_t v, void* buf, int64_t cap, int64_t* bytes)
{
    if (!s || !bytes) { set_error("null argument"); return GL_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(s->mu);
    if (v < 0 || v >= (int64_t)s->versions.size()) { set_error("version not recorded"); return GL_ERR_NOT_FOUND; }
    const auto& b = s->versions[(size_t)v];
    *bytes = (int64_t)b.size();
    if (buf && cap >= (int64_t)b.size()) std::memcpy(buf, b.data(), b.size());
    return GL_OK;
}

extern "C" gl_status gl_server_destroy(gl_server* s)
{
    if (!s) return GL_OK;
    gl_server_drain(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->tm.joinable()) s->tm.join();
    if (s->tr.joinable()) s->tr.join();
    cudaStreamSynchronize(s->rstream);
    for (Snap& sn : s->snap) {
        for (DevBuf& b : sn.arr) b.release();
        if (sn.ready) cudaEventDestroy(sn.ready);
    }
    s->rview.release();
    s->rgb.release();
    cudaStreamDestroy(s->rstream);
    delete s;
    return GL_OK;
}
