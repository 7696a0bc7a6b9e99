// Re-solve server: requests (a grid, control bounds, V0, horizon) are queued,
// admitted into batch slots when a slot and enough of the device-memory
// budget are free, and stepped together with whatever else is in flight
// (continuous batching: the batch advances a few steps per tick and new
// requests join between ticks).  Results stay on the device until the
// caller fetches them, which frees the slot.
//
// This is the serving side of the paper's real-time claim (Sec. I and
// Sec. IV-C: the BRT of a changed environment is re-computed at 5 Hz, i.e.
// within 200 ms); the scheme and the kernels are the batch path's.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "hj_internal.h"

namespace {

enum ReqState : int32_t { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3 };

struct Request {
    int64_t id;
    int32_t n[4];
    double lo[4], hi[4], params[2];
    double T, cfl;
    std::vector<double> v0;  // host copy until admission
    bool xy = false;         // v0 holds the N1*N2 (x, y) field only
    int32_t slot = -1;
    ReqState state = REQ_QUEUED;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int64_t steps = 0;
    hj_status error = HJ_OK;  // why admission failed (REQ_FAILED)
};

double now_s(const std::chrono::steady_clock::time_point &t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct hj_server {
    hj_batch *batch = nullptr;
    int32_t steps_per_tick = 8;
    int64_t next_id = 1;
    std::deque<int64_t> queue;
    std::map<int64_t, Request> reqs;
    std::chrono::steady_clock::time_point t0;
    int64_t ticks = 0, batch_steps = 0;
};

namespace {

hj_status sfail(hj_status s, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    hj_internal_set_error(buf);
    return s;
}

}  // namespace

extern "C" {

hj_status hj_server_create(int32_t max_slots, size_t memory_budget, int32_t steps_per_tick, void *cuda_stream,
                           hj_server **out)
{
    hj_internal_set_error("");
    if (!out) return sfail(HJ_ERR_INVALID_ARG, "out is NULL");
    if (steps_per_tick < 1) return sfail(HJ_ERR_INVALID_ARG, "steps_per_tick must be >= 1");
    hj_server *s = new (std::nothrow) hj_server();
    if (!s) return sfail(HJ_ERR_OOM, "host allocation failed");
    hj_status st = hj_batch_create(max_slots, memory_budget, cuda_stream, &s->batch);
    if (st != HJ_OK) {
        delete s;
        return st;
    }
    s->steps_per_tick = steps_per_tick;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return HJ_OK;
}

void hj_server_destroy(hj_server *s)
{
    if (!s) return;
    hj_batch_destroy(s->batch);
    delete s;
}

double hj_server_clock(const hj_server *s) { return s ? now_s(s->t0) : 0.0; }

static hj_status submit(hj_server *s, const int32_t n[4], const double lo[4], const double hi[4],
                        const double params[2], const double *v0, bool xy, double T, double cfl, int64_t *request_id)
{
    if (!s || !n || !lo || !hi || !params || !v0 || !request_id) return sfail(HJ_ERR_INVALID_ARG, "NULL argument");
    for (int d = 0; d < 4; ++d)
        if (n[d] < 3) return sfail(HJ_ERR_INVALID_ARG, "N%d = %d < 3", d + 1, n[d]);
    if (!isfinite(T) || T < 0) return sfail(HJ_ERR_INVALID_ARG, "T must be finite and >= 0");
    if (!isfinite(cfl) || !(cfl > 0) || cfl > 1) return sfail(HJ_ERR_INVALID_ARG, "cfl must be in (0, 1]");
    const size_t cells = xy ? (size_t)n[0] * n[1] : (size_t)n[0] * n[1] * n[2] * n[3];
    Request r;
    r.xy = xy;
    r.id = s->next_id++;
    memcpy(r.n, n, sizeof(r.n));
    memcpy(r.lo, lo, sizeof(r.lo));
    memcpy(r.hi, hi, sizeof(r.hi));
    memcpy(r.params, params, sizeof(r.params));
    r.T = T;
    r.cfl = cfl;
    try {
        r.v0.assign(v0, v0 + cells);
    } catch (...) {
        return sfail(HJ_ERR_OOM, "host allocation failed");
    }
    r.t_submit = now_s(s->t0);
    const int64_t id = r.id;
    s->queue.push_back(id);
    s->reqs.emplace(id, std::move(r));
    *request_id = id;
    return HJ_OK;
}

hj_status hj_server_submit(hj_server *s, const int32_t n[4], const double lo[4], const double hi[4],
                           const double params[2], const double *v0, double T, double cfl, int64_t *request_id)
{
    hj_internal_set_error("");
    return submit(s, n, lo, hi, params, v0, false, T, cfl, request_id);
}

hj_status hj_server_submit_xy(hj_server *s, const int32_t n[4], const double lo[4], const double hi[4],
                              const double params[2], const double *v0_xy, double T, double cfl,
                              int64_t *request_id)
{
    hj_internal_set_error("");
    return submit(s, n, lo, hi, params, v0_xy, true, T, cfl, request_id);
}

hj_status hj_server_tick(hj_server *s, int32_t *completed, int32_t *running, int32_t *queued)
{
    hj_internal_set_error("");
    if (!s) return sfail(HJ_ERR_INVALID_ARG, "server is NULL");
    // 1. admit queued requests in arrival order while slots and memory last
    while (!s->queue.empty()) {
        Request &r = s->reqs[s->queue.front()];
        int32_t slot = -1;
        hj_status st = hj_batch_add(s->batch, r.n, r.lo, r.hi, r.params, &slot);
        if (st == HJ_ERR_OOM) break;  // wait for running requests to be fetched
        if (st == HJ_OK) {
            st = r.xy ? hj_batch_set_initial_value_xy(s->batch, slot, r.v0.data(), r.v0.size())
                      : hj_batch_set_initial_value(s->batch, slot, r.v0.data(), r.v0.size());
            if (st == HJ_OK) st = hj_batch_set_horizon(s->batch, slot, r.T, r.cfl);
            if (st != HJ_OK) hj_batch_remove(s->batch, slot);
        }
        if (st == HJ_ERR_CUDA || st == HJ_ERR_TIMEOUT) return st;  // the device is in trouble
        if (st != HJ_OK) {  // this request cannot run (unsupported grid, NaN in V0, ...)
            r.state = REQ_FAILED;
            r.error = st;
            r.t_done = now_s(s->t0);
            std::vector<double>().swap(r.v0);
            s->queue.pop_front();
            continue;
        }
        std::vector<double>().swap(r.v0);
        r.slot = slot;
        r.state = REQ_RUNNING;
        r.t_admit = now_s(s->t0);
        s->queue.pop_front();
    }
    // 2. step everything in flight
    int32_t nrun = 0;
    for (auto &kv : s->reqs)
        if (kv.second.state == REQ_RUNNING) ++nrun;
    if (nrun > 0) {
        hj_batch_stats bs;
        hj_status st = hj_batch_advance(s->batch, s->steps_per_tick, &bs);
        if (st != HJ_OK) return st;
        s->batch_steps += bs.steps;
    }
    ++s->ticks;
    // 3. collect the requests that reached their horizon (one state pull)
    int32_t done = 0;
    nrun = 0;
    hj_status st = hj_batch_refresh(s->batch);
    if (st != HJ_OK) return st;
    const double t_now = now_s(s->t0);
    for (auto &kv : s->reqs) {
        Request &r = kv.second;
        if (r.state != REQ_RUNNING) continue;
        int64_t steps = 0;
        if (hj_batch_cached_done(s->batch, r.slot, &steps)) {
            r.state = REQ_DONE;
            r.t_done = t_now;
            r.steps = steps;
            ++done;
        } else {
            ++nrun;
        }
    }
    if (completed) *completed = done;
    if (running) *running = nrun;
    if (queued) *queued = (int32_t)s->queue.size();
    return HJ_OK;
}

hj_status hj_server_request_info(const hj_server *s, int64_t id, hj_request_info *info)
{
    hj_internal_set_error("");
    if (!s || !info) return sfail(HJ_ERR_INVALID_ARG, "NULL argument");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(HJ_ERR_INVALID_ARG, "unknown request %lld", (long long)id);
    const Request &r = it->second;
    memset(info, 0, sizeof(*info));
    info->state = r.state;
    info->slot = r.slot;
    info->steps = r.steps;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
    return HJ_OK;
}

static hj_status fetch(hj_server *s, int64_t id, void *out, hj_precision dtype, bool host, size_t count)
{
    if (!s || !out) return sfail(HJ_ERR_INVALID_ARG, "NULL argument");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(HJ_ERR_INVALID_ARG, "unknown request %lld", (long long)id);
    Request &r = it->second;
    if (r.state == REQ_FAILED) {
        const hj_status e = r.error;
        s->reqs.erase(it);
        return sfail(e, "request %lld was not admitted: %s", (long long)id, hj_status_string(e));
    }
    if (r.state != REQ_DONE) return sfail(HJ_ERR_STATE, "request %lld is not done", (long long)id);
    hj_status st = host ? hj_batch_read_value(s->batch, r.slot, (double *)out, count)
                        : hj_batch_read_value_device(s->batch, r.slot, out, dtype, count);
    if (st != HJ_OK) return st;
    st = hj_batch_remove(s->batch, r.slot);
    s->reqs.erase(it);
    return st;
}

hj_status hj_server_fetch(hj_server *s, int64_t id, double *out, size_t count)
{
    hj_internal_set_error("");
    return fetch(s, id, out, HJ_FP64, true, count);
}

hj_status hj_server_fetch_device(hj_server *s, int64_t id, void *out_device, hj_precision dtype, size_t count)
{
    hj_internal_set_error("");
    if (dtype != HJ_FP64 && dtype != HJ_FP32) return sfail(HJ_ERR_INVALID_ARG, "unknown dtype");
    return fetch(s, id, out_device, dtype, false, count);
}

hj_status hj_server_stats(const hj_server *s, int64_t *ticks, int64_t *batch_steps)
{
    hj_internal_set_error("");
    if (!s) return sfail(HJ_ERR_INVALID_ARG, "server is NULL");
    if (ticks) *ticks = s->ticks;
    if (batch_steps) *batch_steps = s->batch_steps;
    return HJ_OK;
}

}  // extern "C"
