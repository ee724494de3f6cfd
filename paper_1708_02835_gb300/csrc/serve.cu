// Serving loop: likelihood requests from many concurrent optimisers over
// fields whose locations and measurements stay resident on the device.
//
// Requests enter a FIFO queue.  A scheduler thread admits the request at the
// head whenever an execution slot is free and its workspace fits in the HBM
// budget (fields + workspaces in flight <= budget); each admitted request is
// enqueued on its slot's own stream, so requests that arrive while others are
// running overlap with them on the GPU (continuous batching at request
// granularity).  Completion is detected by polling a CUDA event; the result
// is read from pinned host memory, the workspace is returned to the budget and
// the next request is admitted.  Latency = completion time - submit time.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "egs_internal.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Field {
    double *locs = nullptr;  // device, 2n
    double *z = nullptr;     // device, n
    int64_t n = 0;
    size_t bytes = 0;
};

struct Request {
    int64_t ticket;
    int64_t field;
    double theta[3];
    egs_precision p;
    clk::time_point submitted;
};

struct Result {
    bool done = false;
    egs_status status = EGS_OK;
    double loglik = 0.0;
    egs_info info{};
    double latency_ms = 0.0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    egs::DevStatus *h_status = nullptr;  // pinned
    int *h_err = nullptr;                // pinned
    bool busy = false;
    Request req;
    egs::EvalSetup es;
    char *ws = nullptr;
};

}  // namespace

struct egs_server {
    egs_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv_req, cv_done;
    std::deque<Request> queue;
    std::map<int64_t, Result> results;
    std::vector<Field> fields;
    std::vector<Slot> slots;
    size_t used = 0;  // bytes of fields + workspaces in flight
    size_t used_peak = 0;
    int64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    int device = 0;
    egs::Allocator alloc{};  // device memory of fields and workspaces (fixed at creation)
    // statistics
    std::vector<double> lat_ms;
    int64_t completed = 0, failed = 0, rejected = 0, fallbacks = 0;
    int inflight = 0, inflight_peak = 0;
    clk::time_point first_submit{}, last_done{};
    bool any_submit = false;
};

namespace {

// Fields live as long as the server: cudaMalloc, or the caller's hook on the
// legacy stream.
cudaError_t field_alloc(const egs::Allocator &A, double **p, size_t bytes)
{
    if (!A.alloc) return cudaMalloc((void **)p, bytes);
    cudaError_t e = egs::dev_alloc(A, (void **)p, bytes, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    return e;
}

void field_free(const egs::Allocator &A, double *p, size_t bytes)
{
    if (!p) return;
    if (!A.alloc) cudaFree(p);
    else egs::dev_free(A, p, bytes, nullptr);
}

void release_slot(egs_server *S, Slot &sl)
{
    egs::dev_free(S->alloc, sl.ws, sl.es.need, sl.stream);
    sl.ws = nullptr;
    S->used -= sl.es.need;
    sl.busy = false;
    --S->inflight;
}

void finish_slot(egs_server *S, Slot &sl)
{
    // called with S->mu held
    if (S->cfg.fallback_fp64 && sl.req.p != EGS_FP64 && !*sl.h_err && !sl.h_status->timeout) {
        const egs::DevStatus &h = *sl.h_status;
        if (h.fail_index != egs::kNoFail || !egs::mixed_result_ok(sl.es, h)) {
            // the mixed factor failed or was too inexact: answer from FP64
            Request again = sl.req;
            again.p = EGS_FP64;
            ++S->fallbacks;
            release_slot(S, sl);
            S->queue.push_front(again);
            return;
        }
    }
    Result &r = S->results[sl.req.ticket];
    r.done = true;
    const egs::DevStatus &h = *sl.h_status;
    egs::fill_info(sl.es, h, &r.info);
    if (*sl.h_err || h.timeout) {
        r.status = EGS_ERR_TIMEOUT;
        r.loglik = NAN;
    } else if (h.fail_index != egs::kNoFail) {
        r.status = EGS_ERR_NOT_PD;
        r.loglik = NAN;
    } else if (!egs::mixed_result_ok(sl.es, h)) {
        r.status = EGS_ERR_INACCURATE;
        r.loglik = NAN;
    } else {
        r.status = EGS_OK;
        r.loglik = h.result[0];
    }
    const auto now = clk::now();
    r.latency_ms = std::chrono::duration<double, std::milli>(now - sl.req.submitted).count();
    S->lat_ms.push_back(r.latency_ms);
    S->last_done = now;
    if (r.status == EGS_OK) ++S->completed;
    else ++S->failed;
    release_slot(S, sl);
}

bool admit_one(egs_server *S, std::unique_lock<std::mutex> &lk)
{
    // called with S->mu held; admits the head of the queue if possible.  The
    // lock is released while the evaluation's kernels are being enqueued.
    if (S->queue.empty()) return false;
    Slot *free_slot = nullptr;
    for (auto &sl : S->slots)
        if (!sl.busy) {
            free_slot = &sl;
            break;
        }
    if (!free_slot) return false;
    Request &rq = S->queue.front();
    const Field &f = S->fields[rq.field];
    egs_opts o{};
    o.tile = S->cfg.tile;
    o.band = S->cfg.band;
    if (rq.p == EGS_MIX_FP32 && S->cfg.xband > S->cfg.band) o.xband = S->cfg.xband;
    egs::EvalSetup es;
    if (egs::eval_setup(f.n, rq.theta, rq.p, &o, &es) != EGS_OK) {
        Result &r = S->results[rq.ticket];
        r.done = true;
        r.status = EGS_ERR_ARG;
        r.loglik = NAN;
        ++S->rejected;
        S->queue.pop_front();
        S->cv_done.notify_all();
        return true;
    }
    if (S->used + es.need > S->cfg.hbm_budget_bytes) {
        if (S->inflight > 0) return false;  // wait for memory to free up
        // nothing in flight: only resident fields hold the budget, so this
        // request can never be admitted; fail it rather than block the queue
        Result &r = S->results[rq.ticket];
        r.done = true;
        r.status = EGS_ERR_OOM;
        r.loglik = NAN;
        ++S->rejected;
        S->queue.pop_front();
        S->cv_done.notify_all();
        return true;
    }
    Slot &sl = *free_slot;
    char *ws = nullptr;
    cudaError_t e = egs::dev_alloc(S->alloc, (void **)&ws, es.need, sl.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    sl.busy = true;
    sl.req = rq;
    sl.es = es;
    sl.ws = ws;
    S->used += es.need;
    S->used_peak = std::max(S->used_peak, S->used);
    ++S->inflight;
    S->inflight_peak = std::max(S->inflight_peak, S->inflight);
    S->queue.pop_front();
    *sl.h_err = 0;
    const double *flocs = f.locs, *fz = f.z;
    lk.unlock();
    e = egs::eval_enqueue(es, flocs, fz, ws, sl.stream, nullptr, nullptr);
    if (e == cudaSuccess && es.mixed)
        e = cudaMemcpyAsync(sl.h_err, ws + es.ML.err, sizeof(int), cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.h_status, egs::eval_status(es, ws), sizeof(egs::DevStatus), cudaMemcpyDeviceToHost,
                            sl.stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
    lk.lock();
    if (e != cudaSuccess) {
        cudaStreamSynchronize(sl.stream);
        *sl.h_err = 1;
        finish_slot(S, sl);
        S->results[sl.req.ticket].status = EGS_ERR_CUDA;
        S->cv_done.notify_all();
    }
    return true;
}

void worker_loop(egs_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progress = false;
        for (auto &sl : S->slots)
            if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) {
                finish_slot(S, sl);
                progress = true;
            }
        if (progress) S->cv_done.notify_all();
        while (admit_one(S, lk)) progress = true;
        if (!progress) {
            if (S->inflight > 0) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(50));
                lk.lock();
            } else {
                S->cv_req.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
}

}  // namespace

using namespace egs;

extern "C" {

egs_status egs_serve_create(const egs_serve_config *cfg, egs_server **out)
{
    if (!cfg || !out) return set_error(EGS_ERR_ARG, "egs_serve_create: NULL argument");
    *out = nullptr;
    if (cfg->max_inflight < 1 || cfg->max_inflight > 64 || cfg->hbm_budget_bytes == 0)
        return set_error(EGS_ERR_ARG, "egs_serve_create: max_inflight in [1, 64] and a nonzero budget required");
    egs_server *S = new egs_server;
    S->cfg = *cfg;
    S->alloc = egs::current_allocator();
    cudaGetDevice(&S->device);
    S->slots.resize(cfg->max_inflight);
    for (auto &sl : S->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_status, sizeof(DevStatus));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_err, sizeof(int));
        if (e != cudaSuccess) {
            egs_serve_destroy(S);
            return cuda_error(e, "egs_serve_create");
        }
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return EGS_OK;
}

egs_status egs_serve_add_field(egs_server *S, const double *locs, const double *z, int64_t n, int64_t *field_id)
{
    if (!S || !locs || !z || !field_id || n < 1) return set_error(EGS_ERR_ARG, "egs_serve_add_field: bad arguments");
    Field f;
    f.n = n;
    f.bytes = (size_t)3 * n * sizeof(double);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->used + f.bytes > S->cfg.hbm_budget_bytes)
            return set_error(EGS_ERR_OOM, "egs_serve_add_field: field does not fit in the budget");
        S->used += f.bytes;
        S->used_peak = std::max(S->used_peak, S->used);
    }
    cudaError_t e = field_alloc(S->alloc, &f.locs, (size_t)2 * n * sizeof(double));
    if (e == cudaSuccess) e = field_alloc(S->alloc, &f.z, (size_t)n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(f.locs, locs, (size_t)2 * n * sizeof(double), cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(f.z, z, (size_t)n * sizeof(double), cudaMemcpyDefault);
    std::lock_guard<std::mutex> lk(S->mu);
    if (e != cudaSuccess) {
        S->used -= f.bytes;
        field_free(S->alloc, f.locs, (size_t)2 * n * sizeof(double));
        field_free(S->alloc, f.z, (size_t)n * sizeof(double));
        return cuda_error(e, "egs_serve_add_field");
    }
    S->fields.push_back(f);
    *field_id = (int64_t)S->fields.size() - 1;
    return EGS_OK;
}

egs_status egs_serve_submit(egs_server *S, int64_t field_id, const double theta[3], egs_precision p, int64_t *ticket)
{
    if (!S || !theta || !ticket) return set_error(EGS_ERR_ARG, "egs_serve_submit: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (field_id < 0 || field_id >= (int64_t)S->fields.size())
        return set_error(EGS_ERR_ARG, "egs_serve_submit: unknown field %lld", (long long)field_id);
    Request r;
    r.ticket = S->next_ticket++;
    r.field = field_id;
    for (int i = 0; i < 3; ++i) r.theta[i] = theta[i];
    r.p = p;
    r.submitted = clk::now();
    if (!S->any_submit) {
        S->first_submit = r.submitted;
        S->any_submit = true;
    }
    S->results[r.ticket] = Result{};
    S->queue.push_back(r);
    *ticket = r.ticket;
    S->cv_req.notify_one();
    return EGS_OK;
}

egs_status egs_serve_wait(egs_server *S, int64_t ticket, int32_t timeout_ms, double *out_loglik, egs_info *info)
{
    if (!S) return set_error(EGS_ERR_ARG, "egs_serve_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return set_error(EGS_ERR_ARG, "egs_serve_wait: unknown ticket %lld", (long long)ticket);
    auto ready = [&] { return S->results[ticket].done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return set_error(EGS_ERR_TIMEOUT, "egs_serve_wait: ticket %lld not done within %d ms", (long long)ticket,
                         timeout_ms);
    Result r = S->results[ticket];
    S->results.erase(ticket);
    if (out_loglik) *out_loglik = r.loglik;
    if (info) *info = r.info;
    if (r.status == EGS_ERR_OOM)
        return set_error(r.status, "egs_serve_wait: request %lld needs more workspace than the budget leaves beside "
                                   "the resident fields",
                         (long long)ticket);
    if (r.status != EGS_OK) return set_error(r.status, "egs_serve_wait: request %lld failed", (long long)ticket);
    return EGS_OK;
}

egs_status egs_serve_stats(egs_server *S, egs_serve_stats_t *st)
{
    if (!S || !st) return set_error(EGS_ERR_ARG, "egs_serve_stats: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof(*st));
    std::vector<double> v = S->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        const size_t i = (size_t)std::min((double)(v.size() - 1), std::ceil(q * v.size()) - 1.0);
        return v[i];
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    double sum = 0.0;
    for (double x : v) sum += x;
    st->mean_ms = v.empty() ? 0.0 : sum / v.size();
    st->completed = S->completed;
    st->failed = S->failed;
    st->rejected = S->rejected;
    st->inflight_peak = S->inflight_peak;
    st->queued = (int64_t)S->queue.size();
    st->bytes_in_use = S->used;
    st->bytes_peak = S->used_peak;
    st->fallbacks = S->fallbacks;
    const double span = S->any_submit ? std::chrono::duration<double>(S->last_done - S->first_submit).count() : 0.0;
    st->evals_per_s = span > 0 ? (double)(S->completed + S->failed) / span : 0.0;
    return EGS_OK;
}

egs_status egs_serve_destroy(egs_server *S)
{
    if (!S) return EGS_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_req.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ws) egs::dev_free(S->alloc, sl.ws, sl.es.need, sl.stream);
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.h_status) cudaFreeHost(sl.h_status);
        if (sl.h_err) cudaFreeHost(sl.h_err);
    }
    for (auto &f : S->fields) {
        field_free(S->alloc, f.locs, (size_t)2 * f.n * sizeof(double));
        field_free(S->alloc, f.z, (size_t)f.n * sizeof(double));
    }
    delete S;
    return EGS_OK;
}

}  // extern "C"
