// ar_serve.cu -- the request server of libar: continuous batching of
// abstract-render requests over resident scenes.
//
// A server owns n_slots slots.  Each slot is a host worker thread with its own
// non-blocking CUDA stream and its own grow-only workspace, so the requests
// that occupy different slots run their pipelines (prep, binning, render)
// concurrently on the device.  Submitted requests wait in a bounded FIFO; a
// slot that becomes free admits the oldest request whose workspace fits the
// device-memory budget next to what the other slots hold.  A request behind
// the head of the queue is admitted first only if it also leaves room for the
// head ("backfilling"), so that large requests are never starved by small ones.
//
// Memory accounting: a slot holds max(its workspace capacity, the estimate of
// the request it runs).  The estimate of a request is the workspace of one of
// its cell batches (records are about a third of it; the batch size follows
// from the per-request limit), capped at the budget.  When a request does not
// fit and idle slots keep large workspaces, those are released first.
//
// Overlap on the device: every slot has a high- and a low-priority stream.  A
// request of at most kSmallCells cells runs on the high-priority one, a larger
// one on the low-priority one, and the slots' workspaces launch the first
// per-pixel sweep of a batch as one CTA per segment (Workspace::interleave),
// so that a large request's CTAs finish one by one and the blocks of a small
// request that arrives meanwhile are scheduled as SMs free up, instead of
// waiting for the large request's persistent sweep to end.
//
// Timeouts and cancellation: with a timeout set, a request still queued when
// it expires is completed with AR_ETIMEOUT without running, and one whose GPU
// work has not finished by then (a host watchdog polls its stream) is
// completed with AR_ETIMEOUT while the slot waits for that work to drain
// before it admits another request.  A cancelled request leaves the queue at
// once; a running one is completed with AR_ECANCELED when its work ends.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ar.h"
#include "ar_common.cuh"
#include "ar_host.h"
#include "ar_launch.h"

namespace ar {

using Clock = std::chrono::steady_clock;

struct ServeRequest {
    uint64_t ticket = 0;
    ar_scene *scene = nullptr;
    ar_intrinsics intr;
    ar_nominal_pose pose;
    std::vector<ar_pose_box> cells;
    float *out_lo = nullptr, *out_hi = nullptr;
    int64_t est = 0;     // workspace estimate (bytes)
    int64_t limit = 0;   // workspace limit the request renders under
    Clock::time_point t_submit, t_done;
    bool done = false;
    bool cancel = false;  // cancelled while running: completed as AR_ECANCELED
    int status = AR_OK;
    std::string error;
};

struct ServeSlot {
    std::thread worker;
    cudaStream_t stream = nullptr;       // low priority: large requests
    cudaStream_t stream_hi = nullptr;    // high priority: small requests
    Workspace ws;
    ServeRequest *running = nullptr;
};

constexpr size_t kQueueCap = 1024;
constexpr size_t kSmallCells = 4;  // requests of at most this many cells run at high priority

// Workspace estimate of one request: the records, keys and boxes of one cell
// batch times three (bins and sort buffers take about two thirds), capped by
// the budget and by the scene's workspace limit (which sizes its batches).
static void estimate(const ar_scene *s, const ar_pose_box *cells, int n_cells, int64_t budget, int64_t &est,
                     int64_t &limit)
{
    int m_active = 0;
    for (int k = 0; k < MAXV; ++k) {
        bool act = false;
        for (int c = 0; c < n_cells; ++c) act = act || cells[c].hi[k] > cells[c].lo[k];
        m_active += act;
    }
    const int M = m_active <= 1 ? 1 : (m_active <= 4 ? 4 : 6);
    const int64_t per_cell = (int64_t)(sizeof(float) * rec_width(M) + 64) * s->n;
    const int64_t want = 3 * per_cell * n_cells + 96 * s->n;
    limit = want < budget ? want : budget;
    if (limit > s->ws_limit) limit = s->ws_limit;  // the scene's own batch limit
    if (limit < (int64_t)1 << 20) limit = (int64_t)1 << 20;
    est = limit;
}

}  // namespace ar

using namespace ar;

struct ar_server {
    int device = 0;
    int64_t budget = 0;
    std::vector<ServeSlot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServeRequest *> pending;
    std::unordered_map<uint64_t, ServeRequest *> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    double timeout_ms = 0.0;  // 0: none
};

namespace ar {

static int64_t held_by(const ServeSlot &sl)
{
    int64_t h = (int64_t)sl.ws.bytes();
    if (sl.running && sl.running->est > h) h = sl.running->est;
    return h;
}

static double ms_since(Clock::time_point t) { return std::chrono::duration<double, std::milli>(Clock::now() - t).count(); }

// Under the lock: complete the queued requests whose timeout has passed.
static void expire_queued(ar_server *sv)
{
    if (!(sv->timeout_ms > 0.0)) return;
    for (auto it = sv->pending.begin(); it != sv->pending.end();) {
        ServeRequest *r = *it;
        if (ms_since(r->t_submit) > sv->timeout_ms) {
            r->t_done = Clock::now();
            r->status = AR_ETIMEOUT;
            r->error = "request timed out in the queue";
            r->done = true;
            it = sv->pending.erase(it);
        } else {
            ++it;
        }
    }
}

// Under the lock: pick the request slot k admits next, or null.
static ServeRequest *pick(ar_server *sv, int k)
{
    expire_queued(sv);
    if (sv->pending.empty()) return nullptr;
    int64_t others = 0;
    for (int j = 0; j < (int)sv->slots.size(); ++j)
        if (j != k) others += held_by(sv->slots[j]);
    int64_t mine = (int64_t)sv->slots[k].ws.bytes();
    auto fits = [&](const ServeRequest *r, int64_t reserve) {
        const int64_t need = r->est > mine ? r->est : mine;
        return others + need + reserve <= sv->budget;
    };
    ServeRequest *head = sv->pending.front();
    if (fits(head, 0)) {
        sv->pending.pop_front();
        return head;
    }
    // the head waits for memory: release idle workspaces (this slot's own
    // included) if that helps
    bool trimmed = false;
    for (int j = 0; j < (int)sv->slots.size(); ++j) {
        ServeSlot &o = sv->slots[j];
        if (!o.running && o.ws.bytes() > 0) {
            cudaStreamSynchronize(o.stream);
            cudaStreamSynchronize(o.stream_hi);
            o.ws.release();
            trimmed = true;
        }
    }
    if (trimmed) {
        mine = 0;
        others = 0;
        for (int j = 0; j < (int)sv->slots.size(); ++j)
            if (j != k) others += held_by(sv->slots[j]);
        if (fits(head, 0)) {
            sv->pending.pop_front();
            return head;
        }
    }
    // backfill: a later request that fits next to the head's reservation
    for (auto it = sv->pending.begin() + 1; it != sv->pending.end(); ++it) {
        if (fits(*it, head->est)) {
            ServeRequest *r = *it;
            sv->pending.erase(it);
            return r;
        }
    }
    return nullptr;
}

static void complete(ar_server *sv, ServeRequest *r, int code, const std::string &err)
{
    r->t_done = Clock::now();
    r->status = r->cancel ? AR_ECANCELED : code;
    r->error = r->cancel ? std::string("request cancelled") : err;
    r->done = true;
}

static void worker_main(ar_server *sv, int k)
{
    cudaSetDevice(sv->device);
    ServeSlot &sl = sv->slots[k];
    sl.ws.interleave = true;
    std::unique_lock<std::mutex> lock(sv->mu);
    for (;;) {
        ServeRequest *r = nullptr;
        // wake now and then to expire queued requests under a timeout
        while (!sv->stop && (r = pick(sv, k)) == nullptr) sv->cv.wait_for(lock, std::chrono::milliseconds(5));
        if (!r) break;  // stopping and nothing admitted
        sl.running = r;
        const double timeout = sv->timeout_ms;
        lock.unlock();
        cudaStream_t st = r->cells.size() <= kSmallCells ? sl.stream_hi : sl.stream;
        ar_render_stats stats;
        int code = render_core(r->scene, sl.ws, &r->intr, &r->pose, r->cells.data(), (int32_t)r->cells.size(), 0,
                               r->out_lo, r->out_hi, st, false, &stats, false, r->limit);
        std::string err = code ? ar_last_error() : std::string();
        // watchdog: poll the stream until its work is done or the timeout passes
        bool timed_out = false;
        for (;;) {
            const cudaError_t q = cudaStreamQuery(st);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) {
                if (code == AR_OK) {
                    code = AR_EDEVICE;
                    err = cudaGetErrorString(q);
                }
                cudaGetLastError();
                break;
            }
            if (!timed_out && timeout > 0.0 && ms_since(r->t_submit) > timeout) {
                // report the timeout now; the slot keeps waiting for its work
                timed_out = true;
                lock.lock();
                complete(sv, r, AR_ETIMEOUT, "request did not finish within the server's timeout");
                lock.unlock();
            }
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
        if (!timed_out && code == AR_OK && timeout > 0.0 && ms_since(r->t_submit) > timeout) {
            code = AR_ETIMEOUT;
            err = "request did not finish within the server's timeout";
        }
        lock.lock();
        if (!timed_out) complete(sv, r, code, err);
        sl.running = nullptr;
        sv->cv.notify_all();  // memory freed: other slots may admit now
    }
}

}  // namespace ar

static int serve_fail(int code, const char *msg) { return set_last_error(code, msg); }

int ar_serve_create(int64_t hbm_budget_bytes, int32_t n_slots, ar_server **out)
{
    if (!out) return serve_fail(AR_EINVAL, "out is null");
    *out = nullptr;
    if (hbm_budget_bytes < ((int64_t)1 << 20)) return serve_fail(AR_EINVAL, "budget below 1 MiB");
    if (n_slots < 1 || n_slots > 64) return serve_fail(AR_EINVAL, "n_slots must be in [1, 64]");
    ar_server *sv = new ar_server();
    cudaGetDevice(&sv->device);
    sv->budget = hbm_budget_bytes;
    sv->slots.resize(n_slots);
    int prio_lo = 0, prio_hi = 0;  // numerically lower is higher priority
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    for (auto &sl : sv->slots) {
        if (cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
            cudaStreamCreateWithPriority(&sl.stream_hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
            cudaGetLastError();
            for (auto &o : sv->slots) {
                if (o.stream) cudaStreamDestroy(o.stream);
                if (o.stream_hi) cudaStreamDestroy(o.stream_hi);
            }
            delete sv;
            return serve_fail(AR_EDEVICE, "stream creation failed");
        }
    }
    for (int k = 0; k < n_slots; ++k) sv->slots[k].worker = std::thread(worker_main, sv, k);
    *out = sv;
    return AR_OK;
}

int ar_serve_destroy(ar_server *sv)
{
    if (!sv) return serve_fail(AR_EINVAL, "server is null");
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        // requests still queued are dropped; running ones finish
        for (ServeRequest *r : sv->pending) {
            sv->tickets.erase(r->ticket);
            delete r;
        }
        sv->pending.clear();
    }
    sv->cv.notify_all();
    for (auto &sl : sv->slots)
        if (sl.worker.joinable()) sl.worker.join();
    cudaSetDevice(sv->device);
    for (auto &sl : sv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.stream_hi) cudaStreamSynchronize(sl.stream_hi);
        sl.ws.release();
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.stream_hi) cudaStreamDestroy(sl.stream_hi);
    }
    for (auto &kv : sv->tickets) delete kv.second;
    delete sv;
    return AR_OK;
}

int ar_serve_submit(ar_server *sv, ar_scene *scene, const ar_intrinsics *intr, const ar_nominal_pose *pose,
                    const ar_pose_box *cells, int32_t n_cells, float *out_lower, float *out_upper,
                    uint64_t *ticket)
{
    if (!sv || !scene || !ticket) return serve_fail(AR_EINVAL, "null argument");
    int r = validate_call(intr, pose, cells, n_cells, 0);
    if (r) return r;
    if (!out_lower || !out_upper) return serve_fail(AR_EINVAL, "null output");
    if (scene->device != sv->device) return serve_fail(AR_EINVAL, "scene and server are on different devices");
    ServeRequest *q = new ServeRequest();
    q->scene = scene;
    q->intr = *intr;
    q->pose = *pose;
    q->cells.assign(cells, cells + n_cells);
    q->out_lo = out_lower;
    q->out_hi = out_upper;
    estimate(scene, cells, n_cells, sv->budget, q->est, q->limit);
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        if (sv->stop) {
            delete q;
            return serve_fail(AR_EINVAL, "server is stopping");
        }
        if (sv->pending.size() >= kQueueCap) {
            delete q;
            return serve_fail(AR_EAGAIN, "request queue is full");
        }
        q->ticket = sv->next_ticket++;
        q->t_submit = Clock::now();
        sv->tickets[q->ticket] = q;
        sv->pending.push_back(q);
        *ticket = q->ticket;
    }
    sv->cv.notify_all();
    return AR_OK;
}

int ar_serve_set_timeout(ar_server *sv, double timeout_ms)
{
    if (!sv) return serve_fail(AR_EINVAL, "server is null");
    if (!(timeout_ms >= 0.0)) return serve_fail(AR_EINVAL, "timeout must be >= 0 (0: none)");
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->timeout_ms = timeout_ms;
    return AR_OK;
}

int ar_serve_cancel(ar_server *sv, uint64_t ticket)
{
    if (!sv) return serve_fail(AR_EINVAL, "server is null");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return serve_fail(AR_EINVAL, "unknown or retired ticket");
    ServeRequest *q = it->second;
    if (q->done) return AR_OK;
    for (auto p = sv->pending.begin(); p != sv->pending.end(); ++p)
        if (*p == q) {
            sv->pending.erase(p);
            q->cancel = true;
            complete(sv, q, AR_ECANCELED, "");
            return AR_OK;
        }
    q->cancel = true;  // running: completed as cancelled when its work ends
    return AR_OK;
}

int ar_serve_poll(ar_server *sv, uint64_t ticket, int *done, double *latency_ms)
{
    if (!sv || !done) return serve_fail(AR_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    expire_queued(sv);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return serve_fail(AR_EINVAL, "unknown or retired ticket");
    ServeRequest *q = it->second;
    *done = q->done ? 1 : 0;
    if (!q->done) {
        if (latency_ms) *latency_ms = -1.0;
        return AR_OK;
    }
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    const int status = q->status;
    if (status != AR_OK) set_last_error(status, q->error.c_str());
    sv->tickets.erase(it);
    delete q;
    return status;
}
