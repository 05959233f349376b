// Continuous-batching solve server.
//
// A long-running process answers requests "solve A x = b for these values of
// a known pattern" (the linear solve of one Newton iteration of one
// simulation).  The paper's solver handles one matrix at a time; this server
// keeps one handle resident per pattern and batches concurrent requests of
// the same pattern through the batched checked re-factorization and solve
// (same kernels and arithmetic as the single-matrix path, so every result
// equals the result of running that request alone on the same handle).
//
// Per pattern: a handle (symbolic structure, schedule, factors), a CUDA
// stream, device batch buffers for `slots` value sets, and a worker thread.
// The worker takes whatever requests are queued, up to `slots`, runs them as
// one batch, and answers them; requests that arrive meanwhile wait for the
// next batch, so slots are refilled as soon as they free up.  Patterns run on
// separate streams and overlap on the device.  A set whose pivot check fails
// is redone through gblu_refactorize (restart with pivoting, Section IV-C of
// the paper), which moves the pattern's handle to the new pivot sequence for
// later requests.
//
// Admission is by device-memory footprint: a pattern is admitted only if its
// handle plus its batch buffers fit in what remains of the server's budget;
// the slot count is the largest that fits (up to max_batch).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gblu.h"

namespace {

using Clock = std::chrono::steady_clock;

// patterns of more than this many unknowns share the device with small ones
// (max_sms = 3/4 of the SMs, low stream priority)
constexpr int32_t kSmallPatternMax = 100000;

thread_local std::string s_err = "no error";

int sfail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s_err = buf;
    return code;
}

struct Request {
    int64_t id = 0;
    int32_t pattern = 0;
    const double *Ax = nullptr;
    const double *b = nullptr;
    double *x = nullptr;
    int32_t mode = 0;   // 0: double precision; 1: single-precision factors + refinement
    Clock::time_point t_submit, t_start;
    gblu_request_result res{};
    bool done = false;
};

struct Pattern {
    int32_t id = 0;
    gblu_handle h = nullptr;
    int32_t n = 0;
    int64_t nnz_a = 0, lu_stride = 0;
    int32_t slots = 0;
    int64_t footprint = 0;
    cudaStream_t st = nullptr;
    double *Ax_d = nullptr, *LU_d = nullptr, *b_d = nullptr, *x_d = nullptr, *res_d = nullptr;
    double *res_h = nullptr;   // pinned, 4 per slot
    // pinned staging of every slot's values, right-hand side and solution:
    // a copy between the device and pageable host memory goes through the
    // driver's own staging, shared by every stream, and waits behind the
    // copies of other streams (one of them behind a pattern's seconds-long
    // launches); requests are copied into and out of these on the host
    double *in_h = nullptr, *out_h = nullptr;
    std::vector<int32_t> failed;
    std::deque<Request *> queue;
    std::condition_variable cv;
    std::thread worker;
    int64_t batches = 0, requests = 0, repivots = 0;
    int32_t max_batch_seen = 0;
};

}  // namespace

struct gblu_server_s {
    int device = 0;
    gblu_opts opts{};
    int64_t budget = 0, reserved = 0;
    int32_t max_batch = 1;
    std::mutex mu;                 // queues, requests, counters, reserved
    std::condition_variable cv_done;
    std::vector<std::unique_ptr<Pattern>> patterns;
    std::unordered_map<int64_t, std::unique_ptr<Request>> requests;
    int64_t next_id = 1, submitted = 0, completed = 0;
    bool stop = false;
};

namespace {

void free_pattern(Pattern *p)
{
    if (p->h) gblu_destroy(p->h);
    p->h = nullptr;
    cudaFree(p->Ax_d);
    cudaFree(p->LU_d);
    cudaFree(p->b_d);
    cudaFree(p->x_d);
    cudaFree(p->res_d);
    if (p->res_h) cudaFreeHost(p->res_h);
    if (p->in_h) cudaFreeHost(p->in_h);
    if (p->out_h) cudaFreeHost(p->out_h);
    if (p->st) cudaStreamDestroy(p->st);
    p->Ax_d = p->LU_d = p->b_d = p->x_d = p->res_d = p->res_h = nullptr;
    p->st = nullptr;
}

int64_t server_buffer_bytes(const Pattern *p)
{
    return 8 * (int64_t)p->slots * (p->nnz_a + p->lu_stride + 2 * (int64_t)p->n + 4);
}

int alloc_buffers(Pattern *p)
{
    const size_t S = (size_t)p->slots;
    if (cudaMalloc(&p->Ax_d, S * p->nnz_a * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&p->LU_d, S * p->lu_stride * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&p->b_d, S * p->n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&p->x_d, S * p->n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&p->res_d, S * 4 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&p->res_h, S * 4 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&p->in_h, S * (p->nnz_a + p->n) * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&p->out_h, S * p->n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return sfail(GBLU_ERR_NOMEM, "server: batch buffers for %d sets do not fit on the device", p->slots);
    }
    p->failed.assign(S, 0);
    return GBLU_OK;
}

// slot i's inputs through the pinned staging (host copies, then one
// asynchronous copy each) and its solution back the same way
int stage_in(Pattern *p, const Request *r, int i, cudaStream_t st)
{
    const int64_t n = p->n, na = p->nnz_a;
    double *hx = p->in_h + (size_t)i * (na + n);
    std::memcpy(hx, r->Ax, na * sizeof(double));
    std::memcpy(hx + na, r->b, n * sizeof(double));
    if (cudaMemcpyAsync(p->Ax_d + (size_t)i * na, hx, na * sizeof(double), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(p->b_d + (size_t)i * n, hx + na, n * sizeof(double), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return sfail(GBLU_ERR_CUDA, "server: copy of request inputs failed");
    return GBLU_OK;
}

int stage_out(Pattern *p, int i, cudaStream_t st)
{
    const int64_t n = p->n;
    if (cudaMemcpyAsync(p->out_h + (size_t)i * n, p->x_d + (size_t)i * n, n * sizeof(double),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return sfail(GBLU_ERR_CUDA, "server: copy of the solution failed");
    return GBLU_OK;
}

// A single-precision request (mode 1): gblu_refactorize_f32 and
// gblu_solve_refined on the pattern's handle (which falls back to double
// precision itself when refinement cannot reach 1e-12).
void run_refined(gblu_server_s *s, Pattern *p, Request *r)
{
    const Clock::time_point t0 = Clock::now();
    cudaStream_t st = p->st;
    const int64_t n = p->n, na = p->nnz_a;
    int rc = stage_in(p, r, 0, st);
    int32_t it = 0;
    double berr = -1.0;
    if (rc == GBLU_OK) rc = gblu_refactorize_f32(p->h, p->Ax_d, st, nullptr);
    if (rc == GBLU_OK) rc = gblu_solve_refined(p->h, p->Ax_d, p->b_d, p->x_d, 1e-12, 10, st, &it, &berr);
    if (rc == GBLU_OK) rc = stage_out(p, 0, st);
    if (rc == GBLU_OK && cudaStreamSynchronize(st) != cudaSuccess)
        rc = sfail(GBLU_ERR_CUDA, "server: copy of the solution failed");
    if (rc == GBLU_OK) std::memcpy(r->x, p->out_h, n * sizeof(double));
    const Clock::time_point t1 = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->t_start = t0;
    r->res.status = rc;
    r->res.repivoted = 0;
    r->res.batch_size = 1;
    r->res.pattern = p->id;
    r->res.berr = rc >= 0 ? berr : -1.0;
    r->res.refine_iters = it;
    r->res.queue_s = std::chrono::duration<double>(t0 - r->t_submit).count();
    r->res.latency_s = std::chrono::duration<double>(t1 - r->t_submit).count();
    r->done = true;
    p->batches++;
    p->requests++;
    s->completed++;
}

// One batch: copy in, batched refactor + solve, single-path redo of failed
// sets, residuals, copy out.  Fills every request's result.
void run_batch(gblu_server_s *s, Pattern *p, std::vector<Request *> &batch)
{
    const int k = (int)batch.size();
    const Clock::time_point t0 = Clock::now();
    cudaStream_t st = p->st;
    const int64_t n = p->n, na = p->nnz_a;
    int rc = GBLU_OK;
    for (int i = 0; i < k && rc == GBLU_OK; i++) {
        batch[i]->t_start = t0;
        rc = stage_in(p, batch[i], i, st);
    }
    int32_t nf = 0;
    if (rc == GBLU_OK)
        rc = gblu_refactorize_batch(p->h, k, p->Ax_d, na, p->LU_d, p->lu_stride, p->failed.data(), &nf, st);
    if (rc == GBLU_OK) rc = gblu_solve_batch(p->h, k, p->LU_d, p->lu_stride, p->b_d, n, p->x_d, n, st);
    std::vector<int> status(k, rc);
    bool restructured = false;
    if (rc == GBLU_OK && nf > 0) {
        // a failed set takes the single-matrix path: check, restart with
        // pivoting, solve (the handle keeps the new pivot sequence)
        for (int i = 0; i < k; i++) {
            if (!p->failed[i]) continue;
            int32_t rep = 0;
            int r = gblu_refactorize(p->h, p->Ax_d + i * na, st, &rep);
            if (r >= 0) {
                const int r2 = gblu_solve(p->h, p->b_d + i * n, p->x_d + i * n, st);
                if (r2 != GBLU_OK) r = r2;
            }
            status[i] = r;
            restructured |= (rep != 0);
        }
    }
    if (rc == GBLU_OK) {
        for (int i = 0; i < k; i++) {
            if (status[i] < 0) continue;
            const int r = gblu_residual(p->h, p->Ax_d + i * na, p->b_d + i * n, p->x_d + i * n, p->res_d + 4 * i, st);
            const int c = r != GBLU_OK ? r : stage_out(p, i, st);
            if (c != GBLU_OK) status[i] = c;   // keep GBLU_REPIVOTED
        }
        if (cudaMemcpyAsync(p->res_h, p->res_d, 4 * k * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            const int e = sfail(GBLU_ERR_CUDA, "server: stream failed");
            for (int i = 0; i < k; i++) status[i] = e;
        }
        for (int i = 0; i < k; i++)
            if (status[i] >= 0) std::memcpy(batch[i]->x, p->out_h + (size_t)i * n, n * sizeof(double));
    } else {
        cudaStreamSynchronize(st);
    }
    const Clock::time_point t1 = Clock::now();
    if (restructured) {
        // the restart may have grown the factor: widen the set stride
        gblu_stats hs{};
        if (gblu_get_stats(p->h, &hs) == GBLU_OK && hs.nnz_l + hs.nnz_u > p->lu_stride) {
            cudaFree(p->LU_d);
            p->LU_d = nullptr;
            const int64_t old = p->footprint;
            p->lu_stride = hs.nnz_l + hs.nnz_u;
            std::lock_guard<std::mutex> lk(s->mu);
            // keep within the budget by dropping slots if needed (at least one)
            while (p->slots > 1 &&
                   s->reserved - old + hs.device_bytes + server_buffer_bytes(p) > s->budget)
                p->slots--;
            if (cudaMalloc(&p->LU_d, (size_t)p->slots * p->lu_stride * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                p->slots = 0;   // the pattern cannot serve further requests
            }
            p->footprint = hs.device_bytes + server_buffer_bytes(p);
            s->reserved += p->footprint - old;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    for (int i = 0; i < k; i++) {
        Request *r = batch[i];
        r->res.status = status[i];
        r->res.repivoted = (p->failed[i] && status[i] == GBLU_REPIVOTED) ? 1 : 0;
        r->res.batch_size = k;
        r->res.pattern = p->id;
        r->res.berr = status[i] >= 0 ? p->res_h[4 * i] : -1.0;
        r->res.refine_iters = 0;
        r->res.queue_s = std::chrono::duration<double>(r->t_start - r->t_submit).count();
        r->res.latency_s = std::chrono::duration<double>(t1 - r->t_submit).count();
        r->done = true;
        p->repivots += r->res.repivoted;
    }
    p->batches++;
    p->requests += k;
    p->max_batch_seen = std::max(p->max_batch_seen, k);
    s->completed += k;
}

void worker_loop(gblu_server_s *s, Pattern *p)
{
    cudaSetDevice(s->device);
    std::vector<Request *> batch;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            p->cv.wait(lk, [&] { return s->stop || !p->queue.empty(); });
            if (p->queue.empty()) return;   // stopping and drained
            batch.clear();
            const size_t cap = (size_t)std::max(p->slots, 0);
            while (!p->queue.empty() && batch.size() < cap) {
                batch.push_back(p->queue.front());
                p->queue.pop_front();
            }
            if (batch.empty()) {   // no slots left: answer with an error
                while (!p->queue.empty()) {
                    Request *r = p->queue.front();
                    p->queue.pop_front();
                    r->res.status = GBLU_ERR_NOMEM;
                    r->res.pattern = p->id;
                    r->done = true;
                    s->completed++;
                }
                s->cv_done.notify_all();
                continue;
            }
        }
        // double-precision requests go into one batch; single-precision
        // ones run one by one after it
        std::vector<Request *> refined;
        size_t w = 0;
        for (Request *r : batch) {
            if (r->mode == 1) refined.push_back(r);
            else batch[w++] = r;
        }
        batch.resize(w);
        if (!batch.empty()) {
            run_batch(s, p, batch);
            s->cv_done.notify_all();
        }
        for (Request *r : refined) {
            run_refined(s, p, r);
            s->cv_done.notify_all();
        }
    }
}

}  // namespace

extern "C" {

const char *gblu_server_last_error(void) { return s_err.c_str(); }

int gblu_server_create(gblu_server *out, int device, int64_t hbm_budget_bytes, int32_t max_batch,
                       const gblu_opts *o)
{
    if (!out) return sfail(GBLU_ERR_INVALID_INPUT, "server: null output pointer");
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || max_batch < 1)
        return sfail(GBLU_ERR_INVALID_INPUT, "server: budget must be > 0 and max_batch >= 1");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return sfail(GBLU_ERR_CUDA, "server: CUDA device %d is not available", device);
    }
    auto s = new gblu_server_s;
    s->device = device;
    if (o) s->opts = *o;
    else gblu_default_opts(&s->opts);
    s->budget = hbm_budget_bytes;
    s->max_batch = max_batch;
    *out = s;
    return GBLU_OK;
}

int gblu_server_add_pattern(gblu_server s, int32_t n, const int32_t *Ap, const int32_t *Ai, const int32_t *Q,
                            const double *Ax0_host, int32_t *pattern, int32_t *slots)
{
    if (!s || !Ap || !Ai || !Ax0_host || !pattern) return sfail(GBLU_ERR_INVALID_INPUT, "server: null argument");
    if (cudaSetDevice(s->device) != cudaSuccess) return sfail(GBLU_ERR_CUDA, "server: cudaSetDevice failed");
    auto p = std::make_unique<Pattern>();
    int rc = gblu_create(&p->h, s->device, &s->opts);
    if (rc != GBLU_OK) return sfail(rc, "server: %s", gblu_last_error());
    // errors of the handle calls carry the handle's message; the server's
    // own errors were set by sfail
    auto bail = [&](int code) {
        free_pattern(p.get());
        return code;
    };
    auto bail_h = [&](int code) {
        s_err = std::string("server: ") + gblu_last_error();
        return bail(code);
    };
    rc = gblu_analyze(p->h, n, Ap, Ai, Q);
    if (rc != GBLU_OK) return bail_h(rc);
    // a large pattern's persistent launches hold a quarter of the SMs back
    // and run on a low-priority stream, so that the CTAs of small requests
    // queued meanwhile start on free SMs instead of waiting for its launch
    // to end (kernels are not preempted)
    const bool big = n > kSmallPatternMax;
    if (big) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        gblu_opts ho{};
        gblu_get_opts(p->h, &ho);
        if (ho.max_sms == 0 || ho.max_sms > sms * 3 / 4) {
            ho.max_sms = std::max(1, sms * 3 / 4);
            rc = gblu_set_opts(p->h, &ho, nullptr);
            if (rc != GBLU_OK) return bail_h(rc);
        }
    }
    int pr_least = 0, pr_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&pr_least, &pr_greatest);
    if (cudaStreamCreateWithPriority(&p->st, cudaStreamNonBlocking, big ? pr_least : pr_greatest) != cudaSuccess)
        return bail(sfail(GBLU_ERR_CUDA, "server: stream creation failed"));
    p->n = n;
    p->nnz_a = Ap[n];
    double *Ax0 = nullptr;
    if (cudaMalloc(&Ax0, (size_t)p->nnz_a * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return bail(sfail(GBLU_ERR_NOMEM, "server: no device memory for the first values"));
    }
    cudaMemcpy(Ax0, Ax0_host, (size_t)p->nnz_a * sizeof(double), cudaMemcpyHostToDevice);
    rc = gblu_factorize(p->h, Ax0, p->st);
    if (rc < 0) {
        cudaFree(Ax0);
        return bail_h(rc);
    }
    gblu_stats hs{};
    gblu_get_stats(p->h, &hs);
    p->lu_stride = hs.nnz_l + hs.nnz_u;
    // handle growth per batch set: ready flags, control block and arguments
    // of the batched refactor; intermediate vectors and sums of the solve
    const int64_t per_set = 8 * (p->nnz_a + p->lu_stride + 2 * (int64_t)n + 4) + 44 * (int64_t)n + 1024;
    int64_t avail;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // the handle, plus the single-precision workspace (float factors,
        // widened copy, refinement vectors) grown below
        avail = s->budget - s->reserved - hs.device_bytes - (12 * p->lu_stride + 32 * (int64_t)n);
    }
    p->slots = (int32_t)std::min<int64_t>(s->max_batch, avail > 0 ? avail / per_set : 0);
    if (p->slots < 1) {
        cudaFree(Ax0);
        return bail(sfail(GBLU_ERR_NOMEM, "server: pattern needs %lld + %lld bytes per set, %lld left in the budget",
                          (long long)hs.device_bytes, (long long)per_set, (long long)std::max<int64_t>(avail, 0)));
    }
    rc = alloc_buffers(p.get());
    if (rc != GBLU_OK) {
        cudaFree(Ax0);
        return bail(rc);
    }
    // grow the handle's batch workspace to `slots` sets once, so the
    // footprint is known and no request allocates
    for (int32_t i = 0; i < p->slots; i++)
        cudaMemcpyAsync(p->Ax_d + (size_t)i * p->nnz_a, Ax0, (size_t)p->nnz_a * sizeof(double),
                        cudaMemcpyDeviceToDevice, p->st);
    cudaMemsetAsync(p->b_d, 0, (size_t)p->slots * n * sizeof(double), p->st);
    rc = gblu_refactorize_batch(p->h, p->slots, p->Ax_d, p->nnz_a, p->LU_d, p->lu_stride, nullptr, nullptr, p->st);
    if (rc == GBLU_OK) rc = gblu_solve_batch(p->h, p->slots, p->LU_d, p->lu_stride, p->b_d, n, p->x_d, n, p->st);
    // and the workspace of single-precision requests (the first n values
    // serve as a right-hand side)
    if (rc == GBLU_OK) rc = gblu_refactorize_f32(p->h, p->Ax_d, p->st, nullptr);
    if (rc == GBLU_OK) rc = gblu_solve_refined(p->h, p->Ax_d, p->Ax_d, p->x_d, 1e-12, 2, p->st, nullptr, nullptr);
    cudaStreamSynchronize(p->st);
    cudaFree(Ax0);
    if (rc != GBLU_OK) return bail_h(rc);
    gblu_get_stats(p->h, &hs);
    p->footprint = hs.device_bytes + server_buffer_bytes(p.get());
    Pattern *pp = p.get();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->reserved + p->footprint > s->budget) {
            const long long need = (long long)p->footprint, left = (long long)(s->budget - s->reserved);
            free_pattern(pp);
            return sfail(GBLU_ERR_NOMEM, "server: pattern footprint %lld bytes exceeds the %lld left", need, left);
        }
        s->reserved += p->footprint;
        p->id = (int32_t)s->patterns.size();
        s->patterns.push_back(std::move(p));
    }
    *pattern = pp->id;
    if (slots) *slots = pp->slots;
    pp->worker = std::thread(worker_loop, s, pp);
    return GBLU_OK;
}

int gblu_server_pattern_info(gblu_server s, int32_t pattern, int32_t *slots, int64_t *footprint_bytes,
                             int64_t *nnz_lu)
{
    if (!s) return sfail(GBLU_ERR_INVALID_INPUT, "server: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (pattern < 0 || pattern >= (int32_t)s->patterns.size())
        return sfail(GBLU_ERR_INVALID_INPUT, "server: unknown pattern %d", pattern);
    if (slots) *slots = s->patterns[pattern]->slots;
    if (footprint_bytes) *footprint_bytes = s->patterns[pattern]->footprint;
    if (nnz_lu) *nnz_lu = s->patterns[pattern]->lu_stride;
    return GBLU_OK;
}

int gblu_server_submit(gblu_server s, int32_t pattern, const double *Ax_host, const double *b_host, double *x_host,
                       int32_t mode, int64_t *request)
{
    if (!s || !Ax_host || !b_host || !x_host || !request) return sfail(GBLU_ERR_INVALID_INPUT, "server: null argument");
    if (mode != 0 && mode != 1) return sfail(GBLU_ERR_INVALID_INPUT, "server: mode must be 0 or 1");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop) return sfail(GBLU_ERR_INVALID_INPUT, "server: shutting down");
    if (pattern < 0 || pattern >= (int32_t)s->patterns.size())
        return sfail(GBLU_ERR_INVALID_INPUT, "server: unknown pattern %d", pattern);
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->pattern = pattern;
    r->Ax = Ax_host;
    r->b = b_host;
    r->x = x_host;
    r->mode = mode;
    r->t_submit = Clock::now();
    Pattern *p = s->patterns[pattern].get();
    p->queue.push_back(r.get());
    *request = r->id;
    s->requests.emplace(r->id, std::move(r));
    s->submitted++;
    lk.unlock();
    p->cv.notify_one();
    return GBLU_OK;
}

int gblu_server_wait(gblu_server s, int64_t request, double timeout_s, gblu_request_result *res)
{
    if (!s || !res) return sfail(GBLU_ERR_INVALID_INPUT, "server: null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(request);
    if (it == s->requests.end()) return sfail(GBLU_ERR_INVALID_INPUT, "server: unknown request %lld", (long long)request);
    Request *r = it->second.get();
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(std::max(timeout_s, 0.0)));
    if (!s->cv_done.wait_until(lk, until, [&] { return r->done; }))
        return sfail(GBLU_ERR_BUSY, "server: request %lld not finished", (long long)request);
    *res = r->res;
    s->requests.erase(it);
    return GBLU_OK;
}

int gblu_server_get_stats(gblu_server s, gblu_server_stats *st)
{
    if (!s || !st) return sfail(GBLU_ERR_INVALID_INPUT, "server: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = gblu_server_stats{};
    st->budget_bytes = s->budget;
    st->reserved_bytes = s->reserved;
    st->n_patterns = (int32_t)s->patterns.size();
    st->submitted = s->submitted;
    st->completed = s->completed;
    for (auto &p : s->patterns) {
        st->batches += p->batches;
        st->repivots += p->repivots;
        st->max_batch_seen = std::max(st->max_batch_seen, p->max_batch_seen);
    }
    return GBLU_OK;
}

void gblu_server_destroy(gblu_server s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    for (auto &p : s->patterns) p->cv.notify_all();
    for (auto &p : s->patterns)
        if (p->worker.joinable()) p->worker.join();
    cudaSetDevice(s->device);
    for (auto &p : s->patterns) free_pattern(p.get());
    delete s;
}

}  // extern "C"
