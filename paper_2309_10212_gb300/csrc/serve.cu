// serve.cu -- the render request loop (continuous batching) over the C ABI.
//
// The paper renders one view progressively (Sec. 3, 4); a service renders a
// stream of requests, each a (volume, image size, camera, isovalue).  This
// scheduler keeps a pool of renderers (each with its block cache, wavefront
// buffers and captured pass graphs on the device), admits queued requests
// whenever an in-flight slot (a CUDA stream) is free and the device memory
// budget allows the renderer they need, merges queued requests of the same
// volume and image size into one batched render (views of one wavefront that
// share the speculation budget and the cache), and runs each admitted render
// on its own stream so that renders overlap on the GPU.  Results are the
// framebuffers of the requests, copied to caller buffers, plus latency
// timestamps: arrival, admission, first pass completed (read from the
// renderer's pass mirror in mapped host memory) and final image.
//
// Host code only; every device step is a library render.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "spr_common.cuh"

using namespace spr;

namespace {

struct PoolEntry {
    spr_renderer *r = nullptr;
    int vol = 0, W = 0, H = 0;
    int nv = 0;             // view capacity (a render may use fewer views)
    size_t bytes = 0;       // device bytes charged to the budget
    bool busy = false;
    uint64_t last_used = 0; // admission tick of its last render
    int64_t renders = 0;
};

struct Pending {
    int64_t id;
    spr_request q;
    double t_arrival;
};

struct Flight {
    PoolEntry *pe = nullptr;
    int stream = -1;
    std::vector<Pending> reqs;
    double t_admit = 0.0, t_first = -1.0;
    cudaEvent_t done = nullptr;   // after the render and the output copies
};

struct VolEntry {
    spr_volume *v = nullptr;
    size_t cache_per_view = 0;
};

}  // namespace

struct spr_server {
    spr_server_desc d{};
    std::chrono::steady_clock::time_point t0;
    std::vector<VolEntry> vols;
    std::deque<Pending> pending;
    std::vector<PoolEntry *> pool;
    std::vector<Flight> flights;
    std::vector<cudaStream_t> streams;
    std::vector<char> stream_busy;
    std::vector<cudaEvent_t> free_events;
    std::deque<spr_result> results;
    size_t mem_used = 0;
    int64_t next_id = 0;
    uint64_t tick = 0;
    int64_t renders = 0, renderers_created = 0, renderers_destroyed = 0, done = 0;
};

namespace {

double now_s(const spr_server *s)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

void destroy_entry(spr_server *s, PoolEntry *pe)
{
    spr_destroy_renderer(pe->r);
    s->mem_used -= std::min(s->mem_used, pe->bytes);
    ++s->renderers_destroyed;
    delete pe;
}

size_t cache_for(const spr_server *s, int vol, int nv)
{
    return std::max<size_t>(s->vols[vol].cache_per_view * (size_t)nv, 8 * 256);
}

int estimate(const spr_server *s, int vol, int W, int H, int nv, size_t *need)
{
    return spr_renderer_memory_estimate(s->vols[vol].v, W, H, nv, cache_for(s, vol, nv), s->d.spec_mode, s->d.k,
                                        need);
}

bool has_pending(const spr_server *s, int vol, int W, int H)
{
    for (const Pending &p : s->pending)
        if (p.q.volume == vol && p.q.width == W && p.q.height == H) return true;
    return false;
}

int same_shape_count(const spr_server *s, const PoolEntry *e)
{
    int n = 0;
    for (const PoolEntry *pe : s->pool) n += pe->vol == e->vol && pe->W == e->W && pe->H == e->H;
    return n;
}

// Release idle renderers, least recently used first, until `need` more bytes
// fit the budget: first second copies of a shape (the pool keeps one warm
// renderer per shape where it can), then renderers no queued request
// wants, then (`any`) the rest.
bool make_room(spr_server *s, size_t need, bool any)
{
    // release nothing unless releasing every eligible idle renderer would
    // make room (otherwise warm caches would be lost for no admission)
    size_t idle = 0;
    for (PoolEntry *pe : s->pool)
        if (!pe->busy && (any || same_shape_count(s, pe) >= 2 || !has_pending(s, pe->vol, pe->W, pe->H)))
            idle += pe->bytes;
    if (s->mem_used - std::min(s->mem_used, idle) + need > s->d.memory_bytes) return false;
    for (int round = 0; round < (any ? 3 : 2); ++round)
        while (s->mem_used + need > s->d.memory_bytes) {
            PoolEntry *lru = nullptr;
            for (PoolEntry *pe : s->pool) {
                if (pe->busy) continue;
                if (round == 0 && same_shape_count(s, pe) < 2) continue;
                if (round == 1 && has_pending(s, pe->vol, pe->W, pe->H)) continue;
                if (!lru || pe->last_used < lru->last_used) lru = pe;
            }
            if (!lru) break;
            s->pool.erase(std::find(s->pool.begin(), s->pool.end(), lru));
            destroy_entry(s, lru);
        }
    return s->mem_used + need <= s->d.memory_bytes;
}

int create_entry(spr_server *s, int vol, int W, int H, int nv, size_t need, PoolEntry **out)
{
    spr_renderer *r = nullptr;
    SPR_TRY(spr_create_renderer(s->vols[vol].v, W, H, &r));
    int rc;
    if ((rc = spr_set_cache_budget(r, cache_for(s, vol, nv))) ||
        (rc = spr_set_speculation(r, s->d.spec_mode, s->d.k, s->d.k_max)) || (rc = spr_set_view_count(r, nv))) {
        spr_destroy_renderer(r);
        return rc;
    }
    PoolEntry *pe = new (std::nothrow) PoolEntry();
    if (!pe) {
        spr_destroy_renderer(r);
        return set_error(SPR_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    pe->r = r;
    pe->vol = vol;
    pe->W = W;
    pe->H = H;
    pe->nv = nv;
    pe->bytes = need;
    s->mem_used += need;
    s->pool.push_back(pe);
    ++s->renderers_created;
    *out = pe;
    return SPR_OK;
}

// A renderer for a batch of up to *nv requests of (vol, W, H).  An idle
// pooled renderer of that shape is taken first (the batch shrinks to its
// view capacity).  Otherwise a new one is created when it fits the budget;
// when a renderer of the shape is busy, none is released for a new one (it
// frees up within one render); when none exists, idle renderers are
// released, least recently used first.  *out = nullptr: wait.
int acquire(spr_server *s, int vol, int W, int H, int *nv, PoolEntry **out)
{
    *out = nullptr;
    PoolEntry *best = nullptr;
    bool busy_same = false;
    for (PoolEntry *pe : s->pool) {
        if (pe->vol != vol || pe->W != W || pe->H != H) continue;
        if (pe->busy) {
            busy_same = true;
            continue;
        }
        // the smallest capacity that holds the batch, else the largest one
        if (!best || (best->nv < *nv ? pe->nv > best->nv : (pe->nv >= *nv && pe->nv < best->nv))) best = pe;
    }
    if (best) {
        *nv = std::min(*nv, best->nv);
        *out = best;
        return SPR_OK;
    }
    size_t need = 0;
    // a batch larger than the budget allows shrinks (the requests left out
    // stay queued)
    for (;;) {
        SPR_TRY(estimate(s, vol, W, H, *nv, &need));
        if (need <= s->d.memory_bytes || *nv == 1) break;
        --*nv;
    }
    if (need > s->d.memory_bytes)
        return set_error(SPR_ERR_OUT_OF_MEMORY, "a %dx%d render of volume %d needs %zu bytes, above the budget", W,
                         H, vol, need);
    if (s->mem_used + need > s->d.memory_bytes) {
        if (busy_same) {
            // a smaller batch that fits now, else wait for the busy renderer
            while (*nv > 1 && s->mem_used + need > s->d.memory_bytes) {
                --*nv;
                SPR_TRY(estimate(s, vol, W, H, *nv, &need));
            }
            if (s->mem_used + need > s->d.memory_bytes) return SPR_OK;
        } else if (!make_room(s, need, true)) {
            return SPR_OK;
        }
    }
    return create_entry(s, vol, W, H, *nv, need, out);
}

void finish_request(spr_server *s, const Pending &p, int status, int passes, int batch, double t_admit,
                    double t_first, double t_done, const spr_render_stats *rs)
{
    spr_result res;
    memset(&res, 0, sizeof res);
    res.id = p.id;
    res.status = status;
    res.passes = passes;
    res.batch = batch;
    res.t_arrival = p.t_arrival;
    res.t_admit = t_admit;
    res.t_first_pass = t_first;
    res.t_done = t_done;
    if (rs) {
        res.blocks_decoded = rs->blocks_decoded;
        res.entries = rs->entries;
        res.ms_device = rs->ms_total;
    }
    s->results.push_back(res);
    ++s->done;
}

// Copy view v of the renderer's framebuffer to the request's buffers.
int enqueue_outputs(spr_renderer *r, int v, const spr_request &q, cudaStream_t st)
{
    spr_framebuffer fb;
    SPR_TRY(spr_get_framebuffer(r, &fb));
    const size_t n = (size_t)q.width * q.height, off = n * (size_t)v;
    if (q.depth) SPR_CUDA_TRY(cudaMemcpyAsync(q.depth, fb.depth + off, 4 * n, cudaMemcpyDeviceToDevice, st));
    if (q.rgba) SPR_CUDA_TRY(cudaMemcpyAsync(q.rgba, fb.rgba + off, 4 * n, cudaMemcpyDeviceToDevice, st));
    if (q.block) SPR_CUDA_TRY(cudaMemcpyAsync(q.block, fb.block + off, 4 * n, cudaMemcpyDeviceToDevice, st));
    if (q.status) SPR_CUDA_TRY(cudaMemcpyAsync(q.status, fb.status + off, n, cudaMemcpyDeviceToDevice, st));
    return SPR_OK;
}

// Start one render: the oldest queued request whose shape (volume, image
// size) can get a renderer now, batched with the queued requests of that
// shape behind it (oldest first, up to max_batch and the renderer's view
// capacity).  Requests of one shape start in arrival order; a shape whose
// renderers are all busy does not hold up the others.  *started = false when
// no stream is free or no queued shape can start.
int admit_one(spr_server *s, bool *started)
{
    *started = false;
    if (s->pending.empty()) return SPR_OK;
    int si = -1;
    for (int i = 0; i < (int)s->streams.size(); ++i)
        if (!s->stream_busy[i]) {
            si = i;
            break;
        }
    if (si < 0) return SPR_OK;
    std::vector<size_t> take;
    PoolEntry *pe = nullptr;
    int nv = 0;
    std::vector<uint64_t> tried;
    for (size_t h = 0; h < s->pending.size() && !pe; ++h) {
        const spr_request &head = s->pending[h].q;
        const uint64_t key = ((uint64_t)head.volume << 42) ^ ((uint64_t)head.width << 21) ^ (uint64_t)head.height;
        if (std::find(tried.begin(), tried.end(), key) != tried.end()) continue;
        tried.push_back(key);
        take.clear();
        for (size_t i = h; i < s->pending.size() && (int)take.size() < s->d.max_batch; ++i) {
            const spr_request &q = s->pending[i].q;
            if (q.volume == head.volume && q.width == head.width && q.height == head.height) take.push_back(i);
        }
        nv = (int)take.size();
        int rc = acquire(s, head.volume, head.width, head.height, &nv, &pe);
        if (rc != SPR_OK) {
            // this shape can never fit the budget: fail its requests
            const double t = now_s(s);
            for (size_t k = take.size(); k-- > 0;) {
                finish_request(s, s->pending[take[k]], rc, 0, 1, t, -1.0, t, nullptr);
                s->pending.erase(s->pending.begin() + (std::ptrdiff_t)take[k]);
            }
            *started = true;
            return SPR_OK;
        }
    }
    if (!pe) return SPR_OK;   // wait for a renderer or memory
    take.resize(nv);
    Flight f;
    f.pe = pe;
    f.stream = si;
    for (size_t k : take) f.reqs.push_back(s->pending[k]);
    for (size_t k = take.size(); k-- > 0;) s->pending.erase(s->pending.begin() + (std::ptrdiff_t)take[k]);
    cudaStream_t st = s->streams[si];
    int rc = spr_set_view_count(pe->r, nv);
    for (int v = 0; v < nv && rc == SPR_OK; ++v) {
        const spr_request &q = f.reqs[v].q;
        rc = spr_set_view(pe->r, v, q.eye, q.p00, q.du, q.dv, q.iso);
    }
    if (rc == SPR_OK) rc = spr_render_submit(pe->r, st, s->d.max_passes);
    if (rc == SPR_OK)
        for (int v = 0; v < nv && rc == SPR_OK; ++v) rc = enqueue_outputs(pe->r, v, f.reqs[v].q, st);
    if (rc == SPR_OK) {
        if (s->free_events.empty()) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                rc = set_error(SPR_ERR_CUDA, "event creation failed");
            else
                s->free_events.push_back(e);
        }
    }
    if (rc == SPR_OK) {
        f.done = s->free_events.back();
        s->free_events.pop_back();
        if (cudaEventRecord(f.done, st) != cudaSuccess) rc = set_error(SPR_ERR_CUDA, "event record failed");
    }
    const double t = now_s(s);
    if (rc != SPR_OK) {
        // the renderer is in an unknown state: collect what was submitted,
        // drop it from the pool and fail the batch
        spr_render_collect(pe->r, nullptr, nullptr);
        s->pool.erase(std::find(s->pool.begin(), s->pool.end(), pe));
        destroy_entry(s, pe);
        for (const Pending &p : f.reqs) finish_request(s, p, rc, 0, nv, t, -1.0, t, nullptr);
        *started = true;
        return SPR_OK;
    }
    f.t_admit = t;
    pe->busy = true;
    pe->last_used = ++s->tick;
    ++pe->renders;
    ++s->renders;
    s->stream_busy[si] = 1;
    s->flights.push_back(f);
    *started = true;
    return SPR_OK;
}

// Advance the in-flight renders: first-pass times, completions.
int progress(spr_server *s)
{
    for (size_t i = 0; i < s->flights.size();) {
        Flight &f = s->flights[i];
        int32_t passes = 0, rdone = 0;
        SPR_TRY(spr_render_query(f.pe->r, &passes, &rdone));
        const double t = now_s(s);
        if (f.t_first < 0.0 && passes >= 1) f.t_first = t;
        cudaError_t e = cudaEventQuery(f.done);
        if (e == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (e != cudaSuccess) return set_error(SPR_ERR_CUDA, "render event: %s", cudaGetErrorString(e));
        spr_render_stats rs;
        memset(&rs, 0, sizeof rs);
        int rc = spr_render_collect(f.pe->r, &rs, nullptr);
        if (f.t_first < 0.0) f.t_first = t;   // finished between two polls
        size_t mem = 0;
        if (spr_renderer_memory(f.pe->r, &mem) == SPR_OK && mem > 0) {
            s->mem_used = s->mem_used - std::min(s->mem_used, f.pe->bytes) + mem;
            f.pe->bytes = mem;
        }
        for (const Pending &p : f.reqs)
            finish_request(s, p, rc, rs.passes, (int)f.reqs.size(), f.t_admit, f.t_first, t, &rs);
        f.pe->busy = false;
        s->stream_busy[f.stream] = 0;
        s->free_events.push_back(f.done);
        s->flights.erase(s->flights.begin() + (std::ptrdiff_t)i);
    }
    return SPR_OK;
}

}  // namespace

extern "C" int spr_server_create(const spr_server_desc *d, spr_server **out)
{
    clear_error();
    if (!d || !out) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (d->max_inflight < 1 || d->max_inflight > 64)
        return set_error(SPR_ERR_INVALID_ARG, "max_inflight = %d outside [1, 64]", d->max_inflight);
    if (d->max_batch < 1 || d->max_batch > 64)
        return set_error(SPR_ERR_INVALID_ARG, "max_batch = %d outside [1, 64]", d->max_batch);
    if (d->max_passes < 1) return set_error(SPR_ERR_INVALID_ARG, "max_passes must be positive");
    if (d->spec_mode != SPR_SPEC_FIXED && d->spec_mode != SPR_SPEC_ADAPTIVE)
        return set_error(SPR_ERR_INVALID_ARG, "unknown speculation mode %d", d->spec_mode);
    if (d->k < 1 || d->k > SPR_K_LIMIT || d->k_max < 1 || d->k_max > SPR_K_LIMIT)
        return set_error(SPR_ERR_INVALID_ARG, "k and k_max must lie in [1, %d]", SPR_K_LIMIT);
    spr_server *s = new (std::nothrow) spr_server();
    if (!s) return set_error(SPR_ERR_OUT_OF_MEMORY, "host allocation failed");
    s->d = *d;
    s->t0 = std::chrono::steady_clock::now();
    s->streams.resize(d->max_inflight, nullptr);
    s->stream_busy.assign(d->max_inflight, 0);
    for (auto &st : s->streams)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            spr_server_destroy(s);
            return set_error(SPR_ERR_CUDA, "stream creation failed");
        }
    *out = s;
    return SPR_OK;
}

extern "C" int spr_server_destroy(spr_server *s)
{
    clear_error();
    if (!s) return SPR_OK;
    for (auto &st : s->streams)
        if (st) cudaStreamSynchronize(st);
    for (Flight &f : s->flights) {
        spr_render_collect(f.pe->r, nullptr, nullptr);
        if (f.done) cudaEventDestroy(f.done);
    }
    for (PoolEntry *pe : s->pool) destroy_entry(s, pe);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    for (auto &st : s->streams)
        if (st) cudaStreamDestroy(st);
    delete s;
    return SPR_OK;
}

extern "C" int spr_server_add_volume(spr_server *s, spr_volume *vol, size_t cache_bytes_per_view, int32_t *volume_id)
{
    clear_error();
    if (!s || !vol || !volume_id) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    if (cache_bytes_per_view < 8 * 256)
        return set_error(SPR_ERR_CACHE_TOO_SMALL, "cache of %zu bytes per view is below 8 slots", cache_bytes_per_view);
    VolEntry ve;
    ve.v = vol;
    ve.cache_per_view = cache_bytes_per_view;
    s->vols.push_back(ve);
    *volume_id = (int32_t)s->vols.size() - 1;
    return SPR_OK;
}

extern "C" int spr_server_reserve(spr_server *s, int32_t volume, int32_t width, int32_t height, int32_t n_views)
{
    clear_error();
    if (!s) return set_error(SPR_ERR_INVALID_ARG, "NULL server");
    if (volume < 0 || volume >= (int)s->vols.size()) return set_error(SPR_ERR_INVALID_ARG, "unknown volume %d", volume);
    if (width < 1 || height < 1 || n_views < 1 || n_views > s->d.max_batch)
        return set_error(SPR_ERR_INVALID_ARG, "bad shape %dx%d x%d", width, height, n_views);
    size_t need = 0;
    SPR_TRY(estimate(s, volume, width, height, n_views, &need));
    if (s->mem_used + need > s->d.memory_bytes)
        return set_error(SPR_ERR_OUT_OF_MEMORY, "reserving %zu bytes would exceed the budget (%zu of %zu used)", need,
                         s->mem_used, s->d.memory_bytes);
    PoolEntry *pe = nullptr;
    return create_entry(s, volume, width, height, n_views, need, &pe);
}

extern "C" double spr_server_clock(const spr_server *s)
{
    return s ? now_s(s) : 0.0;
}

extern "C" int spr_server_submit(spr_server *s, const spr_request *q, int64_t *id)
{
    clear_error();
    if (!s || !q) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    if (q->volume < 0 || q->volume >= (int)s->vols.size())
        return set_error(SPR_ERR_INVALID_ARG, "unknown volume %d", q->volume);
    if (q->width < 1 || q->height < 1 || (int64_t)q->width * q->height * s->d.max_batch > (int64_t)1 << 28)
        return set_error(SPR_ERR_INVALID_ARG, "bad image size %dx%d", q->width, q->height);
    for (int a = 0; a < 3; ++a) {
        double e = q->eye[a];
        if (!(e == e) || e * 256.0 != (double)(int64_t)(e * 256.0) || e >= 16384.0 || e <= -16384.0)
            return set_error(SPR_ERR_INVALID_ARG, "eye[%d] must be a multiple of 1/256 below 16384", a);
    }
    if (!(q->iso == q->iso)) return set_error(SPR_ERR_INVALID_ARG, "bad isovalue");
    Pending p;
    p.id = s->next_id++;
    p.q = *q;
    p.t_arrival = q->t_arrival >= 0.0 ? q->t_arrival : now_s(s);
    s->pending.push_back(p);
    if (id) *id = p.id;
    return SPR_OK;
}

extern "C" int spr_server_poll(spr_server *s, spr_result *out, int max_out, int *n_out)
{
    clear_error();
    if (!s || (max_out > 0 && !out) || !n_out) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    *n_out = 0;
    SPR_TRY(progress(s));
    for (;;) {
        bool started = false;
        SPR_TRY(admit_one(s, &started));
        if (!started) break;
    }
    int n = 0;
    while (n < max_out && !s->results.empty()) {
        out[n++] = s->results.front();
        s->results.pop_front();
    }
    *n_out = n;
    return SPR_OK;
}

extern "C" int spr_server_info(const spr_server *s, spr_server_stats *out)
{
    clear_error();
    if (!s || !out) return set_error(SPR_ERR_INVALID_ARG, "NULL argument");
    memset(out, 0, sizeof *out);
    out->pending = (int64_t)s->pending.size();
    out->in_flight = (int64_t)s->flights.size();
    out->renderers = (int64_t)s->pool.size();
    out->memory_used = s->mem_used;
    out->renders = s->renders;
    out->requests_done = s->done;
    out->renderers_created = s->renderers_created;
    out->renderers_destroyed = s->renderers_destroyed;
    return SPR_OK;
}
