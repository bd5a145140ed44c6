// Continuous-batching request server over device-resident ensembles.
//
// Requests (host buffers) queue in arrival order and are served in parts of at most
// kPartRows rows.  A scheduler thread fills a wave whenever an execution slot is free:
// it walks the queue taking one part from each request in turn (round robin), so a
// large request cannot hold back the requests behind it, until the wave has
// max_wave parts or kWaveWork row-trees of work or the next part's device buffers
// (consumer rows and phi) would exceed the remaining device-memory budget.  A wave is
// host-to-device copies, ONE batch-graph launch for all its parts (wdf_batch_explain,
// each slot owns its own batch object), device-to-host copies of phi, then an event.
// Waves of different slots run concurrently on their own streams, so requests that
// arrive while others are on the GPU start as soon as a slot and memory free up.
// Completion is detected by polling the slot events; a request completes when its last
// part does, and its latency is measured from submit to then.  Every row is computed by
// exactly the same per-row code whatever else shares its wave, so a request's phi does
// not depend on the mix or on how it was cut into parts.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "wdf_objects.h"
#include "woodelf.h"

namespace {

using Clock = std::chrono::steady_clock;

wdf_status fail(wdf_status s, const std::string &msg) {
    wdf::set_last_error(msg);
    return s;
}

constexpr int64_t kPartRows = 8192;         // rows per part of a request
constexpr int64_t kWaveWork = 16ll << 20;    // row-trees per wave (rows x trees of the ensemble)
constexpr int64_t kSmallWork = 1ll << 20;    // largest request (row-trees) of the express slot
constexpr int64_t kExpressWaveWork = 4ll << 20;  // row-trees per express wave: short waves
constexpr int kExpressMinSlots = 4;              // slot 0 is the express slot from this many slots on
constexpr int kMaxSkips = 8;                 // fills that may pass over a request that does not fit

struct Request {
    uint64_t ticket = 0;
    int ens = 0;
    const float *C = nullptr;
    float *phi = nullptr;
    int64_t n = 0, ldc = 0, ldp = 0;
    int F = 0;
    Clock::time_point t_submit;
    int64_t next = 0;      // first row not yet in a wave
    int64_t finished = 0;  // rows whose wave has completed
    int skips = 0;         // fills in a row that passed it over for lack of device memory
    bool failed = false;
};

// Rows [r0, r0 + n) of one request.
struct Part {
    uint64_t ticket = 0;
    int ens = 0;
    const float *C = nullptr;
    float *phi = nullptr;
    int64_t n = 0, ldc = 0, ldp = 0;
    int F = 0;
    int64_t bytes = 0;  // device bytes while in flight
    float *d_C = nullptr, *d_phi = nullptr;
};

struct Wave {
    std::vector<Part> parts;
    int slot = -1;
    int64_t bytes = 0;
    bool failed = false;  // a launch step failed: its parts are reported failed
};

}  // namespace

struct wdf_server {
    wdf_ctx *ctx = nullptr;
    std::vector<wdf_ensemble *> ens;
    int64_t budget = 0;
    int max_wave = 0;
    int n_slots = 0;
    std::vector<wdf_batch *> batch;  // one per slot
    std::vector<cudaStream_t> stream;
    std::vector<cudaEvent_t> done_ev;
    std::vector<Wave> wave;          // per slot, empty when free
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<uint64_t, Request> active;  // submitted and not yet complete
    std::deque<uint64_t> pending;        // tickets with rows not yet in a wave, in arrival order
    std::map<uint64_t, int> state;       // 0 queued, 1 in flight, 2 done, 3 failed
    std::map<uint64_t, double> done_ms;  // latency of each completed request
    uint64_t next_ticket = 1;
    int64_t in_use = 0;
    bool stop = false;
    std::string error;
    std::vector<double> lat_ms;
    int64_t submitted = 0, completed = 0, rows_done = 0, waves = 0;
    Clock::time_point t_first, t_last;
    std::thread worker;
};

namespace {

void run(wdf_server *s);

// Launch one wave on its slot (called by the worker without the lock held).  If a step
// fails part-way, the device buffers already taken are released in stream order (after
// whatever copies were already queued) and the slot's event is still recorded, so the
// caller reports the wave's parts only after the slot's stream has finished with their
// host buffers.  recorded is false only if even the event could not be recorded; the
// stream has then been synchronised before returning.
cudaError_t launch_wave(wdf_server *s, Wave &w, bool *recorded) {
    wdf::TraceRange trace_("wdf_server wave");
    cudaStream_t st = s->stream[(size_t)w.slot];
    std::vector<int32_t> idx;
    std::vector<const float *> C;
    std::vector<float *> phi;
    std::vector<int64_t> n, ldc, ldp;
    cudaError_t err = cudaSuccess;
    for (Part &r : w.parts) {
        const size_t row_bytes = (size_t)r.F * sizeof(float);
        err = cudaMallocAsync((void **)&r.d_C, r.n * row_bytes, st);
        if (err != cudaSuccess) {
            r.d_C = nullptr;
            break;
        }
        err = cudaMallocAsync((void **)&r.d_phi, r.n * row_bytes, st);
        if (err != cudaSuccess) {
            r.d_phi = nullptr;
            break;
        }
        err = cudaMemcpy2DAsync(r.d_C, row_bytes, r.C, (size_t)r.ldc * sizeof(float), row_bytes, (size_t)r.n,
                                cudaMemcpyHostToDevice, st);
        if (err != cudaSuccess) break;
        idx.push_back(r.ens);
        C.push_back(r.d_C);
        phi.push_back(r.d_phi);
        n.push_back(r.n);
        ldc.push_back(r.F);
        ldp.push_back(r.F);
    }
    if (err == cudaSuccess) {
        const wdf_status bs = wdf_batch_explain(s->batch[(size_t)w.slot], (int32_t)idx.size(), idx.data(), C.data(),
                                                n.data(), ldc.data(), phi.data(), ldp.data(), st);
        if (bs != WDF_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->error = wdf_last_error();
            err = cudaErrorUnknown;
        }
    }
    for (Part &r : w.parts) {
        if (err == cudaSuccess) {
            const size_t row_bytes = (size_t)r.F * sizeof(float);
            err = cudaMemcpy2DAsync(r.phi, (size_t)r.ldp * sizeof(float), r.d_phi, row_bytes, row_bytes,
                                    (size_t)r.n, cudaMemcpyDeviceToHost, st);
        }
        // released in stream order whatever happened above
        if (r.d_C) cudaFreeAsync(r.d_C, st);
        if (r.d_phi) cudaFreeAsync(r.d_phi, st);
        r.d_C = r.d_phi = nullptr;
    }
    *recorded = cudaEventRecord(s->done_ev[(size_t)w.slot], st) == cudaSuccess;
    if (!*recorded) cudaStreamSynchronize(st);
    return err;
}

// A part's rows are done (ok or failed): the request completes with its last part.
void finish_part(wdf_server *s, const Part &p, bool ok, Clock::time_point now) {
    auto it = s->active.find(p.ticket);
    if (it == s->active.end()) return;
    Request &r = it->second;
    r.finished += p.n;
    if (!ok) r.failed = true;
    if (r.finished < r.n) return;
    s->state[r.ticket] = r.failed ? 3 : 2;
    const double ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
    s->lat_ms.push_back(ms);
    s->done_ms[r.ticket] = ms;
    s->rows_done += r.n;
    ++s->completed;
    s->active.erase(it);
}

// Work of a request's remaining rows in row-trees (rows x trees of its ensemble).
int64_t remaining_work(const wdf_server *s, const Request &r) {
    return (r.n - r.next) * (int64_t)s->ens[(size_t)r.ens]->pk.T;
}

// Fill a wave for a free slot from the queue, one part per request per pass.  The
// express slot (slot 0 when there are four or more) takes only requests whose remaining
// work is at most kSmallWork, in waves of at most kExpressWaveWork, so a small request
// never waits behind the large parts that occupy the other slots.  A part that does not fit the remaining device budget is
// skipped (a smaller one further back may fit), but once a request has been passed over
// kMaxSkips times the fill stops at it, so that memory frees up for it and a stream of
// narrow requests cannot hold a wide one back indefinitely.
Wave fill_wave(wdf_server *s, int slot) {
    Wave w;
    w.slot = slot;
    const bool express = s->n_slots >= kExpressMinSlots && slot == 0;
    const int64_t wave_work = express ? kExpressWaveWork : kWaveWork;
    int64_t work = 0;
    bool added = true, blocked = false;
    while (added && !blocked && (int)w.parts.size() < s->max_wave && work < wave_work) {
        added = false;
        for (auto it = s->pending.begin();
             it != s->pending.end() && (int)w.parts.size() < s->max_wave && work < wave_work;) {
            Request &r = s->active[*it];
            if (express && remaining_work(s, r) > kSmallWork) {
                ++it;
                continue;
            }
            const int64_t rows = std::min(kPartRows, r.n - r.next);
            const int64_t bytes = 2 * rows * (int64_t)r.F * (int64_t)sizeof(float);
            if (s->in_use + w.bytes + bytes > s->budget) {
                if (++r.skips > kMaxSkips) {
                    blocked = true;
                    break;
                }
                ++it;  // does not fit now; a smaller part further back may
                continue;
            }
            r.skips = 0;
            Part p;
            p.ticket = r.ticket;
            p.ens = r.ens;
            p.C = r.C + r.next * r.ldc;
            p.phi = r.phi + r.next * r.ldp;
            p.n = rows;
            p.ldc = r.ldc;
            p.ldp = r.ldp;
            p.F = r.F;
            p.bytes = bytes;
            w.parts.push_back(p);
            w.bytes += bytes;
            work += rows * (int64_t)s->ens[(size_t)r.ens]->pk.T;
            r.next += rows;
            s->state[r.ticket] = 1;
            added = true;
            if (r.next == r.n)
                it = s->pending.erase(it);
            else
                ++it;
        }
    }
    return w;
}

void run(wdf_server *s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // reap finished waves
        bool any_inflight = false;
        for (int k = 0; k < s->n_slots; ++k) {
            Wave &w = s->wave[(size_t)k];
            if (w.parts.empty()) continue;
            const cudaError_t q = cudaEventQuery(s->done_ev[(size_t)k]);
            if (q == cudaErrorNotReady) {
                any_inflight = true;
                continue;
            }
            const auto now = Clock::now();
            for (const Part &p : w.parts) finish_part(s, p, q == cudaSuccess && !w.failed, now);
            if (q != cudaSuccess) s->error = std::string("wave failed: ") + cudaGetErrorString(q);
            s->t_last = now;
            s->in_use -= w.bytes;
            w = Wave();
            s->cv_done.notify_all();
        }
        // fill free slots from the queue
        bool launched = false;
        for (int k = 0; k < s->n_slots && !s->pending.empty(); ++k) {
            if (!s->wave[(size_t)k].parts.empty()) continue;
            Wave w = fill_wave(s, k);
            if (w.parts.empty()) {
                if (s->n_slots >= kExpressMinSlots && k == 0) continue;  // no small request: try the others
                break;                                    // no part fits until memory frees up
            }
            s->in_use += w.bytes;
            ++s->waves;
            lk.unlock();
            bool recorded = true;
            const cudaError_t e = launch_wave(s, w, &recorded);
            lk.lock();
            if (e != cudaSuccess) {
                if (s->error.empty() || e != cudaErrorUnknown)
                    s->error = std::string("launch failed: ") + cudaGetErrorString(e);
                w.failed = true;
            }
            if (!recorded) {  // the stream was synchronised: report the parts now
                const auto now = Clock::now();
                for (const Part &p : w.parts) finish_part(s, p, !w.failed, now);
                s->in_use -= w.bytes;
                s->cv_done.notify_all();
                continue;
            }
            s->wave[(size_t)k] = std::move(w);
            launched = true;
            any_inflight = true;
        }
        if (s->stop && s->pending.empty() && !any_inflight) break;
        if (!launched) {
            // poll the slot events every 50 us while waves are in flight, else sleep until work arrives
            if (any_inflight)
                s->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" {

wdf_status wdf_server_create(wdf_ctx *ctx, int32_t n_ensembles, wdf_ensemble *const *ensembles,
                             int64_t device_budget_bytes, int32_t n_slots, int32_t max_wave_requests,
                             wdf_server **out) {
    if (!ctx || !out || n_ensembles < 1 || !ensembles || device_budget_bytes <= 0 || n_slots < 1 || n_slots > 16 ||
        max_wave_requests < 1)
        return fail(WDF_EINVAL, "bad server arguments");
    *out = nullptr;
    for (int i = 0; i < n_ensembles; ++i)
        if (!ensembles[i] || ensembles[i]->ctx != ctx || !ensembles[i]->has_bg)
            return fail(WDF_EINVAL, "every ensemble must belong to the context and have a background");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    wdf_server *s = new wdf_server();
    s->ctx = ctx_retain(ctx);
    s->ens.assign(ensembles, ensembles + n_ensembles);
    s->budget = device_budget_bytes;
    s->n_slots = n_slots;
    s->max_wave = max_wave_requests;
    s->wave.assign((size_t)n_slots, Wave());
    wdf_status st = WDF_OK;
    for (int k = 0; k < n_slots && st == WDF_OK; ++k) {
        wdf_batch *b = nullptr;
        st = wdf_batch_create(ctx, n_ensembles, ensembles, &b);
        if (st != WDF_OK) break;
        s->batch.push_back(b);
        cudaStream_t str = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&str, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            st = fail(WDF_ECUDA, "stream or event creation failed");
            break;
        }
        s->stream.push_back(str);
        s->done_ev.push_back(ev);
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (st != WDF_OK) {
        for (wdf_batch *b : s->batch) wdf_batch_destroy(b);
        ctx_release(s->ctx);
        delete s;
        return st;
    }
    s->worker = std::thread(run, s);
    *out = s;
    return WDF_OK;
}

wdf_status wdf_server_submit(wdf_server *s, int32_t ensemble_index, const float *C, int64_t n, int64_t ldc,
                             float *phi, int64_t ldphi, uint64_t *ticket) {
    if (!s || !ticket) return fail(WDF_EINVAL, "null argument");
    if (ensemble_index < 0 || ensemble_index >= (int32_t)s->ens.size()) return fail(WDF_EINVAL, "ensemble index");
    const int F = s->ens[(size_t)ensemble_index]->pk.F;
    if (n < 1 || !C || !phi || ldc < F || ldphi < F) return fail(WDF_EINVAL, "bad request sizes");
    Request r;
    r.ens = ensemble_index;
    r.C = C;
    r.phi = phi;
    r.n = n;
    r.ldc = ldc;
    r.ldp = ldphi;
    r.F = F;
    if (2 * std::min(n, kPartRows) * (int64_t)F * (int64_t)sizeof(float) > s->budget)
        return fail(WDF_ENOMEM, "a part of the request is larger than the server's device-memory budget");
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return fail(WDF_EBUSY, "server is shutting down");
        r.ticket = s->next_ticket++;
        s->state[r.ticket] = 0;
        if (s->submitted == 0) s->t_first = r.t_submit;
        ++s->submitted;
        s->active[r.ticket] = r;
        s->pending.push_back(r.ticket);
    }
    s->cv_work.notify_one();
    *ticket = r.ticket;
    return WDF_OK;
}

wdf_status wdf_server_wait(wdf_server *s, uint64_t ticket, int64_t timeout_ms) {
    if (!s) return fail(WDF_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->state.find(ticket);
    if (it == s->state.end()) return fail(WDF_EINVAL, "unknown ticket");
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return s->state[ticket] >= 2; });
    if (!ok) return fail(WDF_ETIMEOUT, "request not finished within the timeout");
    if (s->state[ticket] == 3) return fail(WDF_ECUDA, s->error);
    return WDF_OK;
}

wdf_status wdf_server_poll(wdf_server *s, uint64_t ticket, int32_t *done) {
    if (!s || !done) return fail(WDF_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->state.find(ticket);
    if (it == s->state.end()) return fail(WDF_EINVAL, "unknown ticket");
    *done = it->second >= 2 ? 1 : 0;
    if (it->second == 3) return fail(WDF_ECUDA, s->error);
    return WDF_OK;
}

wdf_status wdf_server_request_ms(wdf_server *s, uint64_t ticket, double *ms) {
    if (!s || !ms) return fail(WDF_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done_ms.find(ticket);
    if (it == s->done_ms.end()) return fail(WDF_EINVAL, "unknown or unfinished ticket");
    *ms = it->second;
    return WDF_OK;
}

wdf_status wdf_server_stats(wdf_server *s, wdf_serving_stats *out) {
    if (!s || !out) return fail(WDF_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->queued = (int64_t)s->pending.size();
    out->waves = s->waves;
    out->rows_completed = s->rows_done;
    out->p50_ms = percentile(s->lat_ms, 0.50);
    out->p99_ms = percentile(s->lat_ms, 0.99);
    out->max_ms = s->lat_ms.empty() ? 0.0 : *std::max_element(s->lat_ms.begin(), s->lat_ms.end());
    const double span = s->completed ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
    out->rows_per_s = span > 0 ? (double)s->rows_done / span : 0.0;
    out->device_bytes_in_use = s->in_use;
    out->device_budget = s->budget;
    return WDF_OK;
}

wdf_status wdf_server_reset_stats(wdf_server *s) {
    if (!s) return fail(WDF_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_ms.clear();
    s->submitted = s->completed = s->rows_done = s->waves = 0;
    // completed tickets are forgotten, so a long-running server's bookkeeping stays bounded
    for (auto it = s->state.begin(); it != s->state.end();)
        it = it->second >= 2 ? s->state.erase(it) : std::next(it);
    s->done_ms.clear();
    return WDF_OK;
}

void wdf_server_destroy(wdf_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->ctx->device) cudaSetDevice(s->ctx->device);
    for (size_t k = 0; k < s->stream.size(); ++k) {
        cudaStreamSynchronize(s->stream[k]);
        cudaStreamDestroy(s->stream[k]);
        cudaEventDestroy(s->done_ev[k]);
    }
    for (wdf_batch *b : s->batch) wdf_batch_destroy(b);
    if (prev >= 0 && prev != s->ctx->device) cudaSetDevice(prev);
    ctx_release(s->ctx);
    delete s;
}

}  // extern "C"
