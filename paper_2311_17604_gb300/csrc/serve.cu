// serve.cu -- the request loop of pd_serve.h: a FIFO queue, admission by
// free slot and device-memory budget, one host thread and CUDA stream per
// slot.  Host code only; every step of a scan runs through the public C ABI.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pd.h"
#include "../../include/pd_normals.h"
#include "../../include/pd_serve.h"
#include "pd_kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket;
    const int32_t* xyz;
    const uint8_t* rgb;
    uint8_t* keep;
    int64_t n, m;
    int64_t bytes;  // admission estimate
    int state;      // 0 queued, 1 running, 2 done
    pd_serve_result res;
};

}  // namespace

struct pd_server {
    pd_ctx* ctx;
    pd_serve_params p;
    int64_t budget;
    int64_t reserved = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work;  // workers: a request arrived / memory freed / closing
    std::condition_variable cv_done;  // pollers
    std::deque<Request*> queue;
    std::unordered_map<int64_t, Request*> all;
    int64_t next_ticket = 0;
    int64_t running = 0, done = 0;
    bool closing = false;
    std::vector<std::thread> workers;
};

namespace {

double ms_since(const pd_server* s) {
    return std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
}

int64_t estimate(const pd_server* s, int64_t n) {
    int64_t per = s->p.normals ? PD_SERVE_BYTES_PER_POINT_NORMALS : PD_SERVE_BYTES_PER_POINT;
    return per * n + (1 << 20);
}

// One scan on the worker's stream.  Device buffers are stream-ordered
// allocations of the context's allocator.
int run_scan(pd_server* s, Request* r, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    pd_ctx* ctx = s->ctx;
    const int64_t n = r->n;
    int rc = PD_OK;
    int32_t* xyz = nullptr;
    uint8_t *rgb = nullptr, *keep = nullptr, *valid = nullptr;
    uint16_t* feat = nullptr;
    float *pca = nullptr, *nrm = nullptr;
    pd_grid* g = nullptr;
    pd_cost_params cp = s->p.cost;
    cp.normals_dev = nullptr;
    cudaEventRecord(e0, st);
#define SCK(x)                                                              \
    do {                                                                    \
        cudaError_t e_ = (x);                                               \
        if (e_ != cudaSuccess) {                                            \
            rc = e_ == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA;    \
            goto out;                                                       \
        }                                                                   \
    } while (0)
#define SALLOC(ptr, type, count)                                                    \
    do {                                                                            \
        ptr = (type*)pd::api_alloc(ctx, sizeof(type) * (size_t)(count), st);        \
        if (!ptr) {                                                                 \
            rc = PD_ENOMEM;                                                         \
            goto out;                                                               \
        }                                                                           \
    } while (0)
#define SRC(x)            \
    do {                  \
        rc = (x);         \
        if (rc) goto out; \
    } while (0)
    SALLOC(xyz, int32_t, n * 3);
    SALLOC(keep, uint8_t, n);
    SCK(cudaMemcpyAsync(xyz, r->xyz, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, st));
    if (r->rgb) {
        SALLOC(rgb, uint8_t, n * 3);
        SCK(cudaMemcpyAsync(rgb, r->rgb, 3 * n, cudaMemcpyHostToDevice, st));
    }
    SRC(pd_build_grid(ctx, xyz, rgb, n, nullptr, st, &g));
    if (s->p.normals && cp.term == PD_TERM_ORIENT) {
        SALLOC(feat, uint16_t, n * PD_MLP_IN);
        SALLOC(pca, float, n * 3);
        SALLOC(valid, uint8_t, n);
        SALLOC(nrm, float, n * 3);
        SRC(pd_normals_pca(g, feat, pca, valid, st));
        SRC(pd_normals_mlp(ctx, s->p.mlp_params_dev, feat, pca, n, 0.f, nrm, st));
        pd::api_free(ctx, feat, st);
        feat = nullptr;
        cp.normals_dev = nrm;
    }
    SRC(pd_decimate_count(g, &cp, r->m, keep, st));
    pd_grid_stats(g, &r->res.stats);
    SCK(cudaMemcpyAsync(r->keep, keep, n, cudaMemcpyDeviceToHost, st));
    cudaEventRecord(e1, st);
    SCK(cudaStreamSynchronize(st));
    {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        r->res.gpu_ms = ms;
    }
out:
    if (g) pd_grid_free(g);
    void* bufs[] = {xyz, rgb, keep, valid, feat, pca, nrm};
    for (void* b : bufs) pd::api_free(ctx, b, st);
    cudaStreamSynchronize(st);
    return rc;
#undef SCK
#undef SALLOC
#undef SRC
}

void worker(pd_server* s, int device) {
    cudaSetDevice(device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // admit the queue head when its estimate fits (a scan alone always fits:
            // submit rejects estimates above the whole budget)
            s->cv_work.wait(lk, [&] {
                if (s->queue.empty()) return s->closing;
                return s->reserved + s->queue.front()->bytes <= s->budget;
            });
            if (s->queue.empty()) break;
            r = s->queue.front();
            s->queue.pop_front();
            s->reserved += r->bytes;
            s->running++;
            r->state = 1;
            r->res.t_admit_ms = ms_since(s);
        }
        int rc = run_scan(s, r, st, e0, e1);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            r->res.status = rc;
            r->res.t_done_ms = ms_since(s);
            r->state = 2;
            s->reserved -= r->bytes;
            s->running--;
            s->done++;
        }
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" int pd_serve_open(pd_ctx* ctx, const pd_serve_params* params, pd_server** out) {
    if (!ctx || !params || !out) return PD_EINVAL;
    const pd_cost_params& c = params->cost;
    if (c.k < 1 || c.k > PD_KMAX || c.term < 0 || c.term > 2 || params->slots < 0 ||
        params->mem_budget < 0)
        return PD_EINVAL;
    if (c.term == PD_TERM_ORIENT && !params->normals) return PD_EINVAL;  // nothing supplies normals
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return PD_ECUDA;
    // keep freed scan buffers cached in the default pool (stream-ordered
    // allocations of contexts without their own allocator)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    pd_server* s = new pd_server();
    s->ctx = ctx;
    s->p = *params;
    s->budget = params->mem_budget;
    if (s->budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete s;
            return PD_ECUDA;
        }
        s->budget = (int64_t)(0.8 * (double)fr);
    }
    s->t0 = Clock::now();
    int slots = params->slots ? params->slots : 4;
    for (int i = 0; i < slots; i++) s->workers.emplace_back(worker, s, device);
    *out = s;
    return PD_OK;
}

extern "C" int64_t pd_serve_submit(pd_server* s, const int32_t* xyz_host, const uint8_t* rgb_host,
                                   int64_t n, int64_t m, double ratio, uint8_t* keep_host) {
    if (!s || !xyz_host || !keep_host || n < 1 || n >= (1ll << 31) - 64) return -PD_EINVAL;
    if (m < 0) {
        if (!(ratio >= 0.0 && ratio <= 1.0)) return -PD_EINVAL;
        m = (int64_t)((double)n * ratio);
    }
    if (m > n) return -PD_EINVAL;
    if (s->p.cost.term == PD_TERM_COLOR && !rgb_host) return -PD_EINVAL;
    Request* r = new Request();
    memset(&r->res, 0, sizeof(r->res));
    r->xyz = xyz_host;
    r->rgb = rgb_host;
    r->keep = keep_host;
    r->n = n;
    r->m = m;
    r->bytes = estimate(s, n);
    r->res.n = n;
    r->res.m = m;
    if (r->bytes > s->budget) {
        delete r;
        return -PD_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->closing) {
            delete r;
            return -PD_EINTERNAL;
        }
        r->ticket = s->next_ticket++;
        r->state = 0;
        r->res.t_submit_ms = ms_since(s);
        s->all[r->ticket] = r;
        s->queue.push_back(r);
    }
    s->cv_work.notify_all();
    return r->ticket;
}

extern "C" int pd_serve_poll(pd_server* s, int64_t ticket, int wait_ms, pd_serve_result* out) {
    if (!s) return PD_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return PD_EINVAL;
    Request* r = it->second;
    auto ready = [&] { return r->state == 2; };
    if (wait_ms < 0) s->cv_done.wait(lk, ready);
    else s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    if (r->state != 2) return PD_ETIMEOUT;
    if (out) *out = r->res;
    return PD_OK;
}

extern "C" int pd_serve_counts(pd_server* s, int64_t* queued, int64_t* running, int64_t* done) {
    if (!s) return PD_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int64_t)s->queue.size();
    if (running) *running = s->running;
    if (done) *done = s->done;
    return PD_OK;
}

extern "C" int pd_serve_close(pd_server* s) {
    if (!s) return PD_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->closing = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->all) delete kv.second;
    delete s;
    return PD_OK;
}
