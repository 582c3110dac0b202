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
    int status = AR_OK;
    std::string error;
};

struct ServeSlot {
    std::thread worker;
    cudaStream_t stream = nullptr;
    Workspace ws;
    ServeRequest *running = nullptr;
};

constexpr size_t kQueueCap = 1024;

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
};

namespace ar {

static int64_t held_by(const ServeSlot &sl)
{
    int64_t h = (int64_t)sl.ws.bytes();
    if (sl.running && sl.running->est > h) h = sl.running->est;
    return h;
}

// Under the lock: pick the request slot k admits next, or null.
static ServeRequest *pick(ar_server *sv, int k)
{
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

static void worker_main(ar_server *sv, int k)
{
    cudaSetDevice(sv->device);
    ServeSlot &sl = sv->slots[k];
    std::unique_lock<std::mutex> lock(sv->mu);
    for (;;) {
        ServeRequest *r = nullptr;
        sv->cv.wait(lock, [&] { return sv->stop || (r = pick(sv, k)) != nullptr; });
        if (!r) break;  // stopping and nothing admitted
        sl.running = r;
        lock.unlock();
        ar_render_stats st;
        int code = render_core(r->scene, sl.ws, &r->intr, &r->pose, r->cells.data(), (int32_t)r->cells.size(), 0,
                               r->out_lo, r->out_hi, sl.stream, false, &st, false, r->limit);
        std::string err = code ? ar_last_error() : std::string();
        if (cudaStreamSynchronize(sl.stream) != cudaSuccess && code == AR_OK) {
            code = AR_EDEVICE;
            err = cudaGetErrorString(cudaGetLastError());
        }
        lock.lock();
        r->t_done = Clock::now();
        r->status = code;
        r->error = err;
        r->done = true;
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
    for (auto &sl : sv->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto &o : sv->slots)
                if (o.stream) cudaStreamDestroy(o.stream);
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
        sl.ws.release();
        if (sl.stream) cudaStreamDestroy(sl.stream);
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

int ar_serve_poll(ar_server *sv, uint64_t ticket, int *done, double *latency_ms)
{
    if (!sv || !done) return serve_fail(AR_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(sv->mu);
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
