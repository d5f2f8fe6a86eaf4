// tll_server.cu -- continuous-batching server over the batched likelihood.
//
// Lens-modelling jobs (one observed lens each, its data resident on the
// device) are admitted against a device-memory budget; each job then
// submits parameter batches (a sampler's proposals) from host memory.  A
// launcher thread coalesces every pending batch -- of any admitted job --
// into one multi-lens launch (tll_batcher_run) per slot; several slots are in
// flight on their own streams, so a new launch fills the SMs as the previous
// one drains, and batches that arrive while others run join the next
// launch.  A completer thread retires launches in order and hands results
// back.  Only the public C ABI (tll.h) and the CUDA runtime are used here.
#include <cuda_runtime.h>

#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tll.h"

namespace {

thread_local char s_err[512] = "";

int sfail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s_err, sizeof s_err, fmt, ap);
    va_end(ap);
    return code;
}

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

constexpr int kMaxSlots = 4;
constexpr size_t kLatencyWindow = 1 << 16;

struct Request {
    long long id = 0;
    int job = 0, B = 0;
    int nparam = TLL_NPARAM;     // entries per vector of the job's lens
    const float *hp = nullptr;   // caller's host params [B][nparam]
    double *ho = nullptr;        // caller's host out [B]
    int state = 0;               // 0 pending, 1 in flight, 2 done, 3 failed
    double t_submit = 0, t_done = 0;
};

struct Job {
    tll_lens *L = nullptr;
    size_t bytes = 0;
    bool open = false;
    int outstanding = 0;         // requests not yet completed
};

struct Slot {
    cudaStream_t stream = nullptr;
    tll_batcher *bat = nullptr;
    float *d_params = nullptr, *h_params = nullptr;
    double *d_out = nullptr, *h_out = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
};

struct Flight {
    int slot = 0;
    std::vector<Request *> reqs;
    std::vector<int> offsets;        // first vector of each request
    std::vector<size_t> poffsets;    // first float of each request's parameters
};

}  // namespace

struct tll_server {
    tll_server_config_t cfg{};
    int dev = 0;
    size_t hbm_used = 0;
    std::vector<Job> jobs;
    Slot slots[kMaxSlots];
    int nslots = 0;
    std::unordered_map<long long, Request *> reqs;
    long long next_id = 1;
    std::deque<Request *> pending;
    std::deque<Flight> inflight;
    std::mutex mu;
    std::condition_variable cv_launch, cv_complete, cv_done;
    std::thread launcher, completer;
    bool stop = false;
    int error = TLL_OK;
    char error_msg[256] = "";
    // statistics
    long long n_launches = 0, n_vectors = 0, n_requests = 0, n_admit_refused = 0;
    std::vector<double> lat;     // ring of request latencies (ms)
    size_t lat_next = 0;
};

namespace {

void set_error(tll_server *S, int code, const char *msg)
{
    if (S->error == TLL_OK) {
        S->error = code;
        snprintf(S->error_msg, sizeof S->error_msg, "%s", msg);
    }
}

void fail_requests(tll_server *S, std::vector<Request *> &rs)
{
    for (Request *r : rs) {
        r->state = 3;
        r->t_done = now_ms();
        S->jobs[r->job].outstanding--;
    }
}

// Launcher: take all pending requests that fit (or one, when coalescing is
// off) into a free slot, stage their params, launch, copy results back.
void launcher_loop(tll_server *S)
{
    cudaSetDevice(S->dev);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_launch.wait(lk, [&] {
            if (S->stop) return true;
            if (S->pending.empty()) return false;
            for (int k = 0; k < S->nslots; ++k)
                if (!S->slots[k].busy) return true;
            return false;
        });
        if (S->stop) break;
        int slot = -1;
        for (int k = 0; k < S->nslots; ++k)
            if (!S->slots[k].busy) { slot = k; break; }
        Flight f;
        f.slot = slot;
        int total = 0;
        size_t ptotal = 0;
        while (!S->pending.empty()) {
            Request *r = S->pending.front();
            if (!f.reqs.empty() && (!S->cfg.coalesce ||
                                    total + r->B > S->cfg.max_vectors_per_launch))
                break;
            S->pending.pop_front();
            f.offsets.push_back(total);
            f.poffsets.push_back(ptotal);
            f.reqs.push_back(r);
            r->state = 1;
            total += r->B;
            ptotal += (size_t)r->B * r->nparam;
            if (!S->cfg.coalesce) break;
        }
        Slot &sl = S->slots[slot];
        sl.busy = true;
        std::vector<tll_lens *> lenses(f.reqs.size());
        for (size_t k = 0; k < f.reqs.size(); ++k) lenses[k] = S->jobs[f.reqs[k]->job].L;
        lk.unlock();

        // stage: host params -> pinned -> device, one copy per launch
        for (size_t k = 0; k < f.reqs.size(); ++k)
            memcpy(sl.h_params + f.poffsets[k], f.reqs[k]->hp,
                   (size_t)f.reqs[k]->B * f.reqs[k]->nparam * sizeof(float));
        std::vector<const float *> pp(f.reqs.size());
        std::vector<double *> oo(f.reqs.size());
        std::vector<int> cnt(f.reqs.size());
        for (size_t k = 0; k < f.reqs.size(); ++k) {
            pp[k] = sl.d_params + f.poffsets[k];
            oo[k] = sl.d_out + f.offsets[k];
            cnt[k] = f.reqs[k]->B;
        }
        int rc = TLL_OK;
        char msg[256] = "";
        cudaError_t e = cudaMemcpyAsync(sl.d_params, sl.h_params, ptotal * sizeof(float),
                                        cudaMemcpyHostToDevice, sl.stream);
        if (e != cudaSuccess) {
            rc = TLL_ECUDA;
            snprintf(msg, sizeof msg, "H2D: %s", cudaGetErrorString(e));
        }
        if (rc == TLL_OK) {
            rc = tll_batcher_run(sl.bat, lenses.data(), pp.data(), cnt.data(), oo.data(),
                                 (int)f.reqs.size(), sl.stream);
            if (rc) snprintf(msg, sizeof msg, "%s", tll_last_error());
        }
        if (rc == TLL_OK) {
            e = cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)total * sizeof(double),
                                cudaMemcpyDeviceToHost, sl.stream);
            if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
            if (e != cudaSuccess) {
                rc = TLL_ECUDA;
                snprintf(msg, sizeof msg, "D2H: %s", cudaGetErrorString(e));
            }
        }
        lk.lock();
        if (rc != TLL_OK) {
            set_error(S, rc, msg);
            fail_requests(S, f.reqs);
            sl.busy = false;
            S->cv_done.notify_all();
            continue;
        }
        S->n_launches++;
        S->inflight.push_back(std::move(f));
        S->cv_complete.notify_one();
    }
}

// Completer: wait for the oldest launch, copy each request's results to
// its caller buffer, free the slot.
void completer_loop(tll_server *S)
{
    cudaSetDevice(S->dev);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_complete.wait(lk, [&] { return S->stop || !S->inflight.empty(); });
        if (S->inflight.empty()) {
            if (S->stop) break;
            continue;
        }
        Flight f = S->inflight.front();
        Slot &sl = S->slots[f.slot];
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(sl.done);
        if (e == cudaSuccess)
            for (size_t k = 0; k < f.reqs.size(); ++k)
                memcpy(f.reqs[k]->ho, sl.h_out + f.offsets[k], (size_t)f.reqs[k]->B * sizeof(double));
        lk.lock();
        S->inflight.pop_front();
        if (e != cudaSuccess) {
            set_error(S, TLL_ECUDA, cudaGetErrorString(e));
            fail_requests(S, f.reqs);
        } else {
            const double t = now_ms();
            for (Request *r : f.reqs) {
                r->state = 2;
                r->t_done = t;
                S->jobs[r->job].outstanding--;
                S->n_vectors += r->B;
                S->n_requests++;
                const double l = t - r->t_submit;
                if (S->lat.size() < kLatencyWindow) S->lat.push_back(l);
                else S->lat[S->lat_next] = l;
                S->lat_next = (S->lat_next + 1) % kLatencyWindow;
            }
        }
        sl.busy = false;
        S->cv_launch.notify_one();
        S->cv_done.notify_all();
    }
}

void destroy_slots(tll_server *S)
{
    for (int k = 0; k < kMaxSlots; ++k) {
        Slot &sl = S->slots[k];
        if (sl.bat) tll_batcher_destroy(sl.bat);
        if (sl.d_params) cudaFree(sl.d_params);
        if (sl.d_out) cudaFree(sl.d_out);
        if (sl.h_params) cudaFreeHost(sl.h_params);
        if (sl.h_out) cudaFreeHost(sl.h_out);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        sl = Slot();
    }
}

}  // namespace

extern "C" {

const char *tll_server_last_error(void) { return s_err; }

int tll_server_create(const tll_server_config_t *cfg, tll_server **out)
{
    if (!out || !cfg) return sfail(TLL_EINVAL, "NULL argument");
    *out = nullptr;
    tll_server_config_t c = *cfg;
    if (c.max_jobs < 1 || c.max_jobs > 1 << 20) return sfail(TLL_EINVAL, "max_jobs out of range");
    if (c.max_vectors_per_launch < 1 || c.max_vectors_per_launch > 1 << 24)
        return sfail(TLL_EINVAL, "max_vectors_per_launch out of range");
    if (c.max_inflight < 1 || c.max_inflight > kMaxSlots)
        return sfail(TLL_EINVAL, "max_inflight must be 1..%d", kMaxSlots);
    tll_server *S = new (std::nothrow) tll_server;
    if (!S) return sfail(TLL_ENOMEM, "host allocation failed");
    S->cfg = c;
    if (cudaGetDevice(&S->dev) != cudaSuccess) {
        delete S;
        return sfail(TLL_ECUDA, "no CUDA device");
    }
    S->jobs.resize(c.max_jobs);
    S->nslots = c.max_inflight;
    const size_t nv = (size_t)c.max_vectors_per_launch;
    for (int k = 0; k < S->nslots; ++k) {
        Slot &sl = S->slots[k];
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_params, nv * TLL_NPARAM_EPL * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_out, nv * sizeof(double));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_params, nv * TLL_NPARAM_EPL * sizeof(float));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_out, nv * sizeof(double));
        int rc = e == cudaSuccess ? tll_batcher_create(c.use_graph, &sl.bat) : TLL_ECUDA;
        if (rc != TLL_OK) {
            destroy_slots(S);
            delete S;
            return rc == TLL_ECUDA && e != cudaSuccess
                       ? sfail(e == cudaErrorMemoryAllocation ? TLL_ENOMEM : TLL_ECUDA,
                               "server buffers: %s", cudaGetErrorString(e))
                       : sfail(rc, "batcher: %s", tll_last_error());
        }
    }
    S->launcher = std::thread(launcher_loop, S);
    S->completer = std::thread(completer_loop, S);
    *out = S;
    return TLL_OK;
}

void tll_server_destroy(tll_server *S)
{
    if (!S) return;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        // let queued and in-flight work finish, then stop the threads
        S->cv_done.wait(lk, [&] { return S->pending.empty() && S->inflight.empty(); });
        S->stop = true;
    }
    S->cv_launch.notify_all();
    S->cv_complete.notify_all();
    S->launcher.join();
    S->completer.join();
    cudaSetDevice(S->dev);
    for (Job &j : S->jobs)
        if (j.L) tll_destroy_lens(j.L);
    for (auto &kv : S->reqs) delete kv.second;
    destroy_slots(S);
    delete S;
}

int tll_server_open_job(tll_server *S, const float *image, const float *noise,
                        const float *psf, int psf_size, const tll_grid_t *grid, int flags,
                        int *job_id)
{
    if (!S || !job_id) return sfail(TLL_EINVAL, "NULL argument");
    *job_id = -1;
    int slot = -1;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->error) return sfail(S->error, "server failed: %s", S->error_msg);
        for (int k = 0; k < (int)S->jobs.size(); ++k)
            if (!S->jobs[k].open && !S->jobs[k].L) { slot = k; break; }
        if (slot < 0) {
            S->n_admit_refused++;
            return sfail(TLL_EBUSY, "all %d job slots in use", (int)S->jobs.size());
        }
        S->jobs[slot].open = true;   // reserve the slot
    }
    tll_lens *L = nullptr;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != S->dev) cudaSetDevice(S->dev);
    int rc = tll_create_lens(image, noise, psf, psf_size, grid, flags | TLL_FLAG_BATCH_ONLY, &L);
    if (rc == TLL_OK && S->cfg.autotune) {
        // first job of its signature: time the launch shapes (later jobs
        // of the same signature start with the result)
        tll_shape_t sh;
        if (tll_lens_shape(L, &sh) == TLL_OK && !sh.tuned) {
            cudaStream_t ts = nullptr;
            if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) {
                rc = TLL_ECUDA;
            } else {
                rc = tll_autotune(L, nullptr, 0, ts, nullptr, nullptr, 0, nullptr);
                cudaStreamDestroy(ts);
            }
            if (rc != TLL_OK) {
                tll_destroy_lens(L);
                L = nullptr;
            }
        }
    }
    if (prev >= 0 && prev != S->dev) cudaSetDevice(prev);
    size_t bytes = 0;
    if (rc == TLL_OK) rc = tll_lens_footprint(L, &bytes);
    std::lock_guard<std::mutex> lk(S->mu);
    if (rc != TLL_OK) {
        S->jobs[slot].open = false;
        return sfail(rc, "lens: %s", tll_last_error());
    }
    if (S->cfg.hbm_budget_bytes > 0 && S->hbm_used + bytes > S->cfg.hbm_budget_bytes) {
        S->jobs[slot].open = false;
        S->n_admit_refused++;
        tll_destroy_lens(L);
        return sfail(TLL_EBUSY, "job needs %zu bytes, %zu of %zu in use", bytes, S->hbm_used,
                     (size_t)S->cfg.hbm_budget_bytes);
    }
    Job &j = S->jobs[slot];
    j.L = L;
    j.bytes = bytes;
    j.outstanding = 0;
    S->hbm_used += bytes;
    *job_id = slot;
    return TLL_OK;
}

int tll_server_set_light(tll_server *S, int job_id, const tll_comp_t *comps, int ncomp)
{
    if (!S) return sfail(TLL_EINVAL, "NULL server");
    tll_lens *L = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (job_id < 0 || job_id >= (int)S->jobs.size() || !S->jobs[job_id].L)
            return sfail(TLL_EINVAL, "no open job %d", job_id);
        Job &j = S->jobs[job_id];
        if (j.outstanding > 0)
            return sfail(TLL_EBUSY, "job %d has %d requests outstanding", job_id, j.outstanding);
        L = j.L;
        j.outstanding++;   // keeps the job from being closed or used meanwhile
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != S->dev) cudaSetDevice(S->dev);
    int rc = tll_set_light(L, comps, ncomp);
    size_t bytes = 0;
    if (rc == TLL_OK) rc = tll_lens_footprint(L, &bytes);
    if (prev >= 0 && prev != S->dev) cudaSetDevice(prev);
    std::lock_guard<std::mutex> lk(S->mu);
    Job &j = S->jobs[job_id];
    j.outstanding--;
    if (rc != TLL_OK) return sfail(rc, "set_light: %s", tll_last_error());
    S->hbm_used = S->hbm_used - j.bytes + bytes;
    j.bytes = bytes;
    return TLL_OK;
}

int tll_server_close_job(tll_server *S, int job_id)
{
    if (!S) return sfail(TLL_EINVAL, "NULL server");
    tll_lens *L = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (job_id < 0 || job_id >= (int)S->jobs.size() || !S->jobs[job_id].L)
            return sfail(TLL_EINVAL, "no open job %d", job_id);
        Job &j = S->jobs[job_id];
        if (j.outstanding > 0)
            return sfail(TLL_EBUSY, "job %d has %d requests outstanding", job_id, j.outstanding);
        L = j.L;
        S->hbm_used -= j.bytes;
        j = Job();
    }
    tll_destroy_lens(L);
    return TLL_OK;
}

int tll_server_submit(tll_server *S, int job_id, const float *params, int B, double *out,
                      long long *request_id)
{
    if (!S || !request_id) return sfail(TLL_EINVAL, "NULL argument");
    *request_id = 0;
    if (B < 1 || B > S->cfg.max_vectors_per_launch)
        return sfail(TLL_EINVAL, "batch size %d outside 1..%d", B, S->cfg.max_vectors_per_launch);
    if (!params || !out) return sfail(TLL_EINVAL, "NULL params or out");
    Request *r = new (std::nothrow) Request;
    if (!r) return sfail(TLL_ENOMEM, "host allocation failed");
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error) {
        delete r;
        return sfail(S->error, "server failed: %s", S->error_msg);
    }
    if (job_id < 0 || job_id >= (int)S->jobs.size() || !S->jobs[job_id].L) {
        delete r;
        return sfail(TLL_EINVAL, "no open job %d", job_id);
    }
    r->id = S->next_id++;
    r->job = job_id;
    r->B = B;
    r->nparam = tll_lens_nparam(S->jobs[job_id].L);
    r->hp = params;
    r->ho = out;
    r->t_submit = now_ms();
    S->jobs[job_id].outstanding++;
    S->reqs[r->id] = r;
    S->pending.push_back(r);
    *request_id = r->id;
    S->cv_launch.notify_one();
    return TLL_OK;
}

int tll_server_poll(tll_server *S, long long request_id, int *done)
{
    if (!S || !done) return sfail(TLL_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return sfail(TLL_EINVAL, "unknown request %lld", request_id);
    *done = it->second->state >= 2;
    if (it->second->state == 3) return sfail(S->error ? S->error : TLL_ECUDA, "request failed");
    return TLL_OK;
}

int tll_server_wait(tll_server *S, long long request_id, int timeout_ms, double *latency_ms)
{
    if (!S) return sfail(TLL_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return sfail(TLL_EINVAL, "unknown request %lld", request_id);
    Request *r = it->second;
    auto ready = [&] { return r->state >= 2; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return sfail(TLL_ETIMEOUT, "request %lld not done after %d ms", request_id, timeout_ms);
    const int state = r->state;
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    S->reqs.erase(it);
    delete r;
    if (state == 3) return sfail(S->error ? S->error : TLL_ECUDA, "request failed: %s", S->error_msg);
    return TLL_OK;
}

int tll_server_stats(tll_server *S, tll_server_stats_t *st)
{
    if (!S || !st) return sfail(TLL_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(st, 0, sizeof *st);
    st->launches = S->n_launches;
    st->vectors = S->n_vectors;
    st->requests = S->n_requests;
    st->admissions_refused = S->n_admit_refused;
    st->pending = (long long)S->pending.size();
    st->inflight = (long long)S->inflight.size();
    st->hbm_used_bytes = S->hbm_used;
    int open = 0;
    for (const Job &j : S->jobs) open += j.L != nullptr;
    st->open_jobs = open;
    if (!S->lat.empty()) {
        std::vector<double> v = S->lat;
        std::sort(v.begin(), v.end());
        auto q = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        st->latency_p50_ms = q(0.50);
        st->latency_p99_ms = q(0.99);
        st->latency_max_ms = v.back();
    }
    return TLL_OK;
}

}  // extern "C"
