// he_server.cu -- continuous-batching request loop for encrypted MatMults.
//
// Requests (an encoded matrix resident on the device, an input and an output ciphertext) are
// admitted in arrival order while the bytes they pin fit the HBM budget.  A server serves one or
// more rings (a context family at one level: the first given at creation, more added with
// he_server_add_ring), each with two batch "lanes".  A scheduler thread packs a ring's admitted
// requests into the slots of a free lane and launches the lane's captured batch graph (empty
// slots are skipped by every kernel); while one lane runs, the next requests are packed into the
// other, so arrivals during a launch join the next one and their work overlaps the launch in
// flight, and the rings' lanes run side by side on their own streams.  A request that finds its
// ring idle and alone runs as one plain call.  Completion is observed with
// CUDA events; no kernel waits on anything.  Plain mode serves one request per
// he_matmult_plain_cipher call instead (in order per ring), the baseline a serving measurement is
// compared with.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "he_internal.cuh"

namespace {

double now_s() { return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count(); }

struct Req {
    const he_ptmat *pm = nullptr;
    const he_plan *plan = nullptr;
    he_ct in{}, out{};
    size_t bytes = 0;
    int ring = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int state = 0;  // 0 queued, 1 admitted, 2 running, 3 done, 4 failed
    int status = HE_OK;
    cudaEvent_t ready = nullptr;  // inputs ready on the ring context's stream
};

struct Lane {
    he_batch *b = nullptr;
    bool busy = false;
    std::vector<int64_t> ids;
};

struct Ring {
    he_ctx *ctx = nullptr;
    int level = 0;
    Lane lanes[2];
    cudaEvent_t plain_done = nullptr;  // plain mode, or a lone request in batched mode: the call in flight on ctx's stream
    Lane solo;                         // batched mode: a lone request run as one call (see schedule_batched)
    std::deque<int64_t> admitted;
};

}  // namespace

struct he_server {
    int slots = 0, plain = 0;
    size_t budget = 0, in_use = 0;
    std::vector<Ring> rings;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Req> reqs;
    std::vector<cudaEvent_t> event_pool;
    std::thread worker;
    bool started = false, stop = false;
    int64_t next_id = 1;
    int64_t launches = 0, completed = 0;
};

namespace {

cudaEvent_t take_event(he_server *s) {
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

void finish(he_server *s, int64_t id, int status) {
    Req &r = s->reqs[id];
    r.state = status == HE_OK ? 3 : 4;
    r.status = status;
    r.t_done = now_s();
    s->in_use -= r.bytes;
    s->completed++;
    if (r.ready) {
        s->event_pool.push_back(r.ready);
        r.ready = nullptr;
    }
}

bool ring_busy(const he_server *s, const Ring &g) { return s->plain ? g.lanes[0].busy : (g.lanes[0].busy || g.lanes[1].busy || g.solo.busy); }

// run request id as one he_matmult_plain_cipher call on the ring context's stream (the lock released
// around it: the call may tune a matrix's loop kernel, synchronising); its completion is recorded
// in g.plain_done and tracked by `ln`
bool run_single(he_server *s, Ring &g, Lane &ln, int64_t id, std::unique_lock<std::mutex> &lock) {
    Req &r = s->reqs[id];
    r.state = 2;
    r.t_start = now_s();
    // only this thread touches r's inputs meanwhile, and map references stay valid across inserts
    const he_plan *plan = r.plan;
    const he_ptmat *pm = r.pm;
    he_ct in = r.in, out = r.out;
    lock.unlock();
    int rc = he_matmult_plain_cipher(g.ctx, plan, pm, &in, 1, &out, 1);
    lock.lock();
    if (rc != HE_OK) {
        finish(s, id, rc);
    } else {
        cudaEventRecord(g.plain_done, g.ctx->stream);
        ln.ids.assign(1, id);
        ln.busy = true;
        s->launches++;
    }
    return true;
}

// one ring's plain-mode pass: one request per he_matmult_plain_cipher call, strictly in order
bool schedule_plain(he_server *s, Ring &g, std::unique_lock<std::mutex> &lock) {
    bool changed = false;
    Lane &ln = g.lanes[0];
    if (ln.busy) {
        if (cudaEventQuery(g.plain_done) != cudaSuccess) return false;
        for (int64_t id : ln.ids) finish(s, id, HE_OK);
        ln.ids.clear();
        ln.busy = false;
        changed = true;
    }
    if (g.admitted.empty()) return changed;
    const int64_t id = g.admitted.front();
    g.admitted.pop_front();
    return run_single(s, g, ln, id, lock);
}

// one ring's batched pass: completions, then every free lane takes up to `slots` admitted
// requests.  A lone request with nothing of its ring on the GPU runs as one plain call instead
// (a batch launch would carry one job and its empty slots; at low load this keeps its latency
// that of the plain path), and requests arriving meanwhile go to the lanes.
bool schedule_batched(he_server *s, Ring &g, std::unique_lock<std::mutex> &lock) {
    bool changed = false;
    for (Lane &ln : g.lanes) {
        if (ln.busy && cudaEventQuery(ln.b->ev_out) == cudaSuccess) {
            for (int64_t id : ln.ids) finish(s, id, HE_OK);
            ln.ids.clear();
            ln.busy = false;
            changed = true;
        }
    }
    if (g.solo.busy && cudaEventQuery(g.plain_done) == cudaSuccess) {
        for (int64_t id : g.solo.ids) finish(s, id, HE_OK);
        g.solo.ids.clear();
        g.solo.busy = false;
        changed = true;
    }
    if (g.admitted.size() == 1 && !g.lanes[0].busy && !g.lanes[1].busy && !g.solo.busy) {
        const int64_t id = g.admitted.front();
        g.admitted.pop_front();
        return run_single(s, g, g.solo, id, lock);
    }
    for (Lane &ln : g.lanes) {
        if (ln.busy || g.admitted.empty()) continue;
        he_batch *b = ln.b;
        const int n = (int)std::min<size_t>(g.admitted.size(), (size_t)s->slots);
        for (int j = 0; j < s->slots; ++j) b->h_jobs[j] = MMJob{};
        const double t = now_s();
        for (int j = 0; j < n; ++j) {
            const int64_t id = g.admitted.front();
            g.admitted.pop_front();
            Req &r = s->reqs[id];
            MMJob &jb = b->h_jobs[j];
            jb.ct = r.in.data;
            jb.out = r.out.data;
            jb.pts = r.pm->data;
            jb.keys = r.pm->d_keys;
            jb.galois = r.pm->d_galois;
            jb.m_prime = (int32_t)r.pm->plan.m_prime;
            r.state = 2;
            r.t_start = t;
            cudaStreamWaitEvent(b->stream, r.ready, 0);
            ln.ids.push_back(id);
        }
        int rc = batch_launch(g.ctx, b);
        if (rc != HE_OK) {
            for (int64_t id : ln.ids) finish(s, id, rc);
            ln.ids.clear();
        } else {
            ln.busy = true;
            s->launches++;
        }
        changed = true;
    }
    return changed;
}

// one scheduling pass; returns true when something changed.  Called with s->mu held by `lock`
// (released around a plain-mode product).
bool schedule(he_server *s, std::unique_lock<std::mutex> &lock) {
    bool changed = false;
    // admission, in arrival order, while the budget allows
    while (!s->queue.empty() && s->in_use + s->reqs[s->queue.front()].bytes <= s->budget) {
        const int64_t id = s->queue.front();
        s->queue.pop_front();
        Req &r = s->reqs[id];
        s->in_use += r.bytes;
        r.state = 1;
        s->rings[r.ring].admitted.push_back(id);
        changed = true;
    }
    for (Ring &g : s->rings) changed |= s->plain ? schedule_plain(s, g, lock) : schedule_batched(s, g, lock);
    return changed;
}

void worker_main(he_server *s) {
    // the scheduler's launches, events and graph replays belong to the contexts' device, whatever
    // device the thread that made the server had current
    cudaSetDevice(s->rings[0].ctx->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        const bool changed = schedule(s, lock);
        if (changed) s->cv.notify_all();
        bool idle = s->queue.empty();
        for (const Ring &g : s->rings) idle = idle && g.admitted.empty() && !ring_busy(s, g);
        if (s->stop && idle) break;
        if (!changed) s->cv.wait_for(lock, std::chrono::microseconds(idle ? 200 : 10));
    }
    s->cv.notify_all();
}

int ring_init(he_server *s, Ring &g, he_ctx *ctx, int level) {
    g.ctx = ctx;
    g.level = level;
    if (cudaEventCreateWithFlags(&g.plain_done, cudaEventDisableTiming) != cudaSuccess) return HE_ECUDA;
    if (s->plain) return HE_OK;
    for (Lane &ln : g.lanes) {
        int rc = batch_create_impl(ctx, s->slots, level, nullptr, &ln.b);
        if (rc != HE_OK) return rc;
        // a lane usually runs few requests: its ModUp, ModDown and rescale as clusters
        ln.b->stage_form = 1;
    }
    return HE_OK;
}

void ring_free(Ring &g) {
    for (Lane &ln : g.lanes) {
        he_batch_free(ln.b);
        ln.b = nullptr;
    }
    if (g.plain_done) cudaEventDestroy(g.plain_done);
    g.plain_done = nullptr;
}

}  // namespace

extern "C" {

int he_server_create(he_ctx *ctx, int slots, int level, size_t hbm_budget_bytes, int plain, he_server **out) {
    if (!ctx || !out || slots < 1 || slots > 4096 || level < 1 || level >= ctx->L || hbm_budget_bytes == 0) return HE_EINVAL;
    *out = nullptr;
    he_server *s = new (std::nothrow) he_server();
    if (!s) return HE_ENOMEM;
    s->slots = plain ? 1 : slots;
    s->plain = plain != 0;
    s->budget = hbm_budget_bytes;
    s->rings.reserve(8);
    s->rings.emplace_back();
    int rc = ring_init(s, s->rings[0], ctx, level);
    if (rc != HE_OK) {
        ring_free(s->rings[0]);
        delete s;
        return rc;
    }
    *out = s;
    return HE_OK;
}

int he_server_add_ring(he_server *s, he_ctx *ctx, int level) {
    if (!s || !ctx || level < 1 || level >= ctx->L) return HE_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->started || s->rings.size() >= 8) return HE_EINVAL;
    for (const Ring &g : s->rings)
        if (same_family(g.ctx, ctx) && g.level == level) return HE_EINVAL;  // already served
    s->rings.emplace_back();
    int rc = ring_init(s, s->rings.back(), ctx, level);
    if (rc != HE_OK) {
        ring_free(s->rings.back());
        s->rings.pop_back();
    }
    return rc;
}

int he_server_submit(he_server *s, const he_plan *plan, const he_ptmat *pm, const he_ct *in, he_ct *out, int64_t *request_id) {
    if (!s || !plan || !pm || !in || !out || !request_id || !in->data || !out->data) return HE_EINVAL;
    if (pm->plan.row_blocks != 1 || pm->plan.col_blocks != 1 || pm->plan.m != plan->m || pm->plan.n != plan->n) return HE_EINVAL;
    if (pm->plan.baby && !s->plain) return HE_EINVAL;  // the batch lanes run the diagonal method's loop kernel
    int ring = -1;
    for (size_t i = 0; i < s->rings.size(); ++i)
        if (same_family(pm->ctx, s->rings[i].ctx) && pm->level == s->rings[i].level) ring = (int)i;
    if (ring < 0) {
        for (const Ring &g : s->rings)
            if (same_family(pm->ctx, g.ctx)) return HE_ELEVEL;
        return HE_EINVAL;
    }
    Ring &g = s->rings[ring];
    if (in->level != g.level) return HE_ELEVEL;
    he_ctx *ctx = g.ctx;
    const size_t N = ctx->n;
    const size_t bytes = (size_t)pm->plan.m_prime * pm->ext * N * 8 + 2 * (size_t)(g.level + 1) * N * 8 + 2 * (size_t)g.level * N * 8;
    if (bytes > s->budget) return HE_EBUDGET;
    int rc = pm->plan.baby ? HE_OK : ptmat_bind_keys(ctx, const_cast<he_ptmat *>(pm));
    if (rc != HE_OK) return rc;
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return HE_EINVAL;
    if (!s->started) {  // the scheduler starts with the first request, once the rings are fixed
        s->worker = std::thread(worker_main, s);
        s->started = true;
    }
    const int64_t id = s->next_id++;
    Req &r = s->reqs[id];
    r.pm = pm;
    r.plan = plan;
    r.in = *in;
    r.out = *out;
    r.ring = ring;
    r.out.level = g.level - 1;
    r.out.scale = in->scale * pm->scale / (double)ctx->primes[g.level];
    r.bytes = bytes;
    r.t_submit = now_s();
    r.ready = take_event(s);
    if (!r.ready || cudaEventRecord(r.ready, ctx->stream) != cudaSuccess) {
        s->reqs.erase(id);
        return HE_ECUDA;
    }
    s->queue.push_back(id);
    *request_id = id;
    out->level = r.out.level;
    out->scale = r.out.scale;
    s->cv.notify_all();
    return HE_OK;
}

int he_server_wait(he_server *s, int64_t id, int64_t timeout_us, double *latency_s) {
    if (!s) return HE_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return HE_EINVAL;
    // a reference, not the iterator: submit may insert (and rehash) while the wait releases the lock
    Req &r = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    while (r.state < 3) {
        if (s->cv.wait_until(lock, deadline) == std::cv_status::timeout && r.state < 3) return HE_ETIMEOUT;
    }
    if (latency_s) *latency_s = r.t_done - r.t_submit;
    const int status = r.status;
    // a finished request's entry (its event is already back in the pool) is dropped, so a
    // long-running server's table holds only requests not yet waited for
    s->reqs.erase(id);
    return status;
}

int he_server_stats(he_server *s, int64_t *completed, int64_t *launches, size_t *bytes_in_use) {
    if (!s) return HE_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (completed) *completed = s->completed;
    if (launches) *launches = s->launches;
    if (bytes_in_use) *bytes_in_use = s->in_use;
    return HE_OK;
}

void he_server_free(he_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Ring &g : s->rings) ring_free(g);
    for (auto &kv : s->reqs)
        if (kv.second.ready) cudaEventDestroy(kv.second.ready);
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    delete s;
}

}  // extern "C"
