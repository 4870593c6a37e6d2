// capi.cu -- the C ABI of libpd (pd.h): contexts, grids, decimation driver.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pd.h"
#include "../../include/pd_normals.h"
#include "../../include/pd_quality.h"
#include "pd_internal.cuh"
#include "pd_kernels.h"

using namespace pd;

namespace pd {
long long g_launch_count = 0;

int device_sms() {
    static int cached[64];  // 0 = not queried yet
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = __atomic_load_n(&cached[dev], __ATOMIC_RELAXED);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
        return 152;
    __atomic_store_n(&cached[dev], v, __ATOMIC_RELAXED);
    return v;
}
}

namespace pd {
// launchers defined in rounds.cu
cudaError_t launch_dup_flag(const u64*, const int4*, int64_t, uint8_t*, unsigned long long*,
                            cudaStream_t);
cudaError_t launch_dup_remove(const uint8_t*, const int4*, int64_t, int, uint8_t*, cudaStream_t);
cudaError_t launch_sel_hist(const u64*, const uint8_t*, int64_t, const u64*, const int*, int64_t,
                            int, const uint32_t*, uint32_t*, cudaStream_t);
cudaError_t launch_sel_compact(const u64*, const int4*, const uint8_t*, int64_t, const u64*,
                               const int*, int64_t, int, const uint32_t*, u64*, int*, int*,
                               cudaStream_t);
cudaError_t launch_k1_fix(const int*, const int*, int, const int4*, const int*, const uint8_t*,
                          int, const uint8_t*, uint8_t*, int*, cudaStream_t);
cudaError_t launch_accept_above(const u64*, const int4*, const uint8_t*, int64_t, u64, int,
                                uint8_t*, int*, int*, cudaStream_t);
cudaError_t launch_pair_fix(const int2*, const int*, int, int, const uint8_t*, uint8_t*, int*,
                            cudaStream_t);
cudaError_t launch_remove(const int*, const int*, int, uint8_t*, uint8_t*, uint8_t*,
                          unsigned long long*, cudaStream_t);
cudaError_t launch_keep(const int4*, const uint8_t*, int64_t, uint8_t*, cudaStream_t);
cudaError_t launch_knn_out(const int4*, const double*, const int*, int64_t, int, int, double*,
                           int32_t*, cudaStream_t);
cudaError_t launch_newpos(const int*, int64_t, int*, cudaStream_t);
cudaError_t launch_remap(const int*, int64_t, const int*, int*, const int*, int64_t, int,
                         cudaStream_t);
cudaError_t launch_take_u64(const int*, int64_t, const u64*, u64*, cudaStream_t);
cudaError_t launch_take_i4(const int*, int64_t, const int4*, int4*, cudaStream_t);
cudaError_t launch_take_u8(const int*, int64_t, const uint8_t*, uint8_t*, cudaStream_t);
cudaError_t launch_take_uc4(const int*, int64_t, const uchar4*, uchar4*, cudaStream_t);
cudaError_t launch_take_f4(const int*, int64_t, const float4*, float4*, cudaStream_t);
}  // namespace pd

// ============================================================ context
struct pd_ctx {
    pd_allocator alloc;
    int has_alloc;
    int tuned_leaf;  // leaf capacity chosen by pd_autotune (0: none yet)
    char err[512];
    std::mutex mu;  // guards err (batch slots report errors concurrently)
    // device-memory budget (0: none).  Under a budget every block is tracked;
    // large blocks beyond it (and large cold ones) live in pinned host memory
    // that the kernels address in place.
    std::mutex mem_mu;
    std::atomic<bool> tracked{false};  // set once a budget was ever given
    uint64_t dev_budget = 0, spill_min = 0;
    uint64_t dev_used = 0, dev_peak = 0, host_used = 0, host_peak = 0;
    std::unordered_map<void*, std::pair<size_t, bool>> blocks;  // bytes, in host memory
};

static void set_err(pd_ctx* c, const char* fmt, const char* a = "", long long b = 0) {
    if (!c) return;
    std::lock_guard<std::mutex> lk(c->mu);
    snprintf(c->err, sizeof(c->err), fmt, a, b);
}

static void* dev_alloc(pd_ctx* c, size_t bytes, cudaStream_t st) {
    if (c->has_alloc) return c->alloc.alloc(c->alloc.user, bytes, (void*)st);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
static void dev_free(pd_ctx* c, void* p, cudaStream_t st) {
    if (c->has_alloc) c->alloc.free(c->alloc.user, p, (void*)st);
    else cudaFreeAsync(p, st);
}

// Blocks below this size always stay in device memory: the small control
// blocks, counters and histograms take device atomics.
#define PD_SPILL_FLOOR ((size_t)1 << 20)

// cold: a block the kernels touch about once (input copies, write-mostly
// state); under a budget such blocks go to host memory first.
static void* ctx_alloc(pd_ctx* c, size_t bytes, cudaStream_t st, bool cold = false) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (!c->tracked.load()) return dev_alloc(c, bytes, st);
    bool host;
    {
        std::lock_guard<std::mutex> lk(c->mem_mu);
        host = c->dev_budget > 0 && bytes >= PD_SPILL_FLOOR && bytes >= c->spill_min &&
               (cold || c->dev_used + bytes > c->dev_budget);
        if (!host) c->dev_used += bytes;  // reserved before the call
    }
    void* p = nullptr;
    if (host) {
        // pinned and mapped: with unified addressing the kernels use the
        // host address itself (over NVLink-C2C on Grace systems)
        void* d = nullptr;
        if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess || d != p) {
            cudaGetLastError();
            cudaFreeHost(p);
            return nullptr;
        }
    } else {
        p = dev_alloc(c, bytes, st);
    }
    std::lock_guard<std::mutex> lk(c->mem_mu);
    if (!p) {
        if (!host) c->dev_used -= bytes;
        return nullptr;
    }
    if (host) {
        c->host_used += bytes;
        c->host_peak = std::max(c->host_peak, c->host_used);
    } else {
        c->dev_peak = std::max(c->dev_peak, c->dev_used);
    }
    c->blocks[p] = std::make_pair(bytes, host);
    return p;
}
static void ctx_free(pd_ctx* c, void* p, cudaStream_t st) {
    if (!p) return;
    if (!c->tracked.load()) {
        dev_free(c, p, st);
        return;
    }
    bool host = false, known = false;
    {
        std::lock_guard<std::mutex> lk(c->mem_mu);
        auto it = c->blocks.find(p);
        if (it != c->blocks.end()) {
            known = true;
            host = it->second.second;
            if (host) c->host_used -= it->second.first;
            else c->dev_used -= it->second.first;
            c->blocks.erase(it);
        }
    }
    if (known && host) {
        // not stream-ordered: wait for the work that may still address it
        cudaStreamSynchronize(st);
        cudaFreeHost(p);
    } else {
        dev_free(c, p, st);
    }
}

// ============================================================ grid
struct pd_grid {
    pd_ctx* ctx;
    cudaStream_t st;
    int64_t n;   // input points
    int64_t ng;  // points held by the grid arrays
    int B, shift, T;
    int3 origin, umax;
    int4* pos;
    u64* code;
    uint8_t* leaf;
    uint8_t* alive;
    uchar4* rgb;
    float4* nrm;
    HashSlot* hash;
    u64 hmask;
    int4* groups;
    int ngroups;
    // neighbour state
    int S, k, density_k1;
    u64* prim;
    int* nbr;
    int* nbr0;  // k = 1 density: nbr[s * S], stored apart so that it reads coalesced
    u64* rk2;
    uint8_t* flg;
    u64* hz;  // k+b buffer horizon
    int* glist;  // flagged searches: groups holding a flagged query, and their count
    int* gcount;
    u64* cmin;   // during a decimation: least live key of every 32-position chunk
    // small device scalars
    int* d_int;                  // [0] ngroups, [1..7] counters
    unsigned long long* d_u64;   // [0] counts
    std::vector<void*> owned;
    pd_stats stats;
    double ms_grid;  // device time of the pd_build_grid call
    int k1_exact;    // k = 1 density searches: nearest entries that must be exact (0: all 8;
                     //   the rest of the 8 stored are kept below the reported horizon)
    int k1_exact_rq; // ... in the re-searches of the rounds
    int sparse_rq;   // k = 1 density re-searches over a list of the flagged points, 2 lanes
                     //   each (else a warp per flagged leaf group)
    double compact_at;  // the rounds compact the grid once live < compact_at * built
                        //   (0: the cost's default)
    int* rq_list;    // during a decimation: flagged Morton positions and their count
    int* rq_count;
    char* arena;     // during a decimation: scratch of the per-round compactions
    size_t arena_cap;
    int trace;       // PD_TRACE set: one line per removal round on stderr
    int max_rounds;  // PD_MAX_ROUNDS: diagnostic stop (0 = none)
    // packed batch (pd_decimate_batch): nseg scans in tiles of edge
    // 2^seg_shift mm; per-scan targets and grid ranges in seg (device)
    int nseg = 0, seg_shift = 0;
    SegDev* seg = nullptr;
    int* seg_chunk0 = nullptr;
    int* seg_items = nullptr;  // the scan of every selection work item
    std::vector<long long> seg_n, seg_m;  // host copies: points and targets per scan
};

namespace {

void* scratch_alloc(void* self, size_t bytes) {
    pd_grid* g = (pd_grid*)self;
    return ctx_alloc(g->ctx, bytes, g->st);
}
void scratch_free(void* self, void* p) {
    pd_grid* g = (pd_grid*)self;
    ctx_free(g->ctx, p, g->st);
}
Scratch scratch_of(pd_grid* g) {
    Scratch s;
    s.alloc = scratch_alloc;
    s.free = scratch_free;
    s.self = g;
    return s;
}

// Bump allocation from the grid's round arena (no allocator call per round:
// the batch runs many small decimations from several host threads).  The
// blocks of one compaction are released together by resetting the arena.
struct ArenaUse {
    pd_grid* g;
    size_t used;
};
void* arena_alloc(void* self, size_t bytes) {
    ArenaUse* a = (ArenaUse*)self;
    size_t b = (bytes + 255) & ~(size_t)255;
    if (!a->g->arena || a->used + b > a->g->arena_cap) return nullptr;
    void* p = a->g->arena + a->used;
    a->used += b;
    return p;
}
void arena_free(void*, void*) {}
// Scratch over the round arena when the decimation has one, else the allocator.
Scratch round_scratch(pd_grid* g, ArenaUse* a) {
    if (!g->arena) return scratch_of(g);
    a->g = g;
    a->used = 0;
    Scratch s;
    s.alloc = arena_alloc;
    s.free = arena_free;
    s.self = a;
    return s;
}

GridView view_of(const pd_grid* g) {
    GridView v;
    v.pos = g->pos;
    v.code = g->code;
    v.leaf = g->leaf;
    v.hash = g->hash;
    v.hmask = g->hmask;
    v.B = g->B;
    v.shift = g->shift;
    v.T = g->T;
    v.origin = g->origin;
    v.umax = g->umax;
    return v;
}

#define CK(x)                                                                  \
    do {                                                                       \
        cudaError_t e_ = (x);                                                  \
        if (e_ != cudaSuccess) {                                               \
            if (e_ == cudaErrorMemoryAllocation) {                             \
                set_err(g->ctx, "out of device memory at %s (line %lld)", #x,  \
                        (long long)__LINE__);                                  \
                return PD_ENOMEM;                                              \
            }                                                                  \
            set_err(g->ctx, "CUDA error at %s: %lld", #x, (long long)e_);      \
            return PD_ECUDA;                                                   \
        }                                                                      \
    } while (0)

#define ALLOC(ptr, type, count)                                                \
    do {                                                                       \
        ptr = (type*)ctx_alloc(g->ctx, sizeof(type) * (size_t)(count), g->st); \
        if (!ptr) {                                                            \
            set_err(g->ctx, "allocation of %s failed (%lld bytes)", #ptr,      \
                    (long long)(sizeof(type) * (size_t)(count)));              \
            return PD_ENOMEM;                                                  \
        }                                                                      \
    } while (0)

#define ALLOC_COLD(ptr, type, count)                                                \
    do {                                                                             \
        ptr = (type*)ctx_alloc(g->ctx, sizeof(type) * (size_t)(count), g->st, true); \
        if (!ptr) {                                                                  \
            set_err(g->ctx, "allocation of %s failed (%lld bytes)", #ptr,            \
                    (long long)(sizeof(type) * (size_t)(count)));                    \
            return PD_ENOMEM;                                                        \
        }                                                                            \
    } while (0)

void gfree(pd_grid* g, void* p) { ctx_free(g->ctx, p, g->st); }

// Temporary device blocks of one function: released (stream-ordered) when the
// function returns, on error paths too; done() releases one early.
struct Temps {
    pd_grid* g;
    std::vector<void*> p;
    explicit Temps(pd_grid* gg) : g(gg) {}
    ~Temps() {
        for (void* x : p) gfree(g, x);
    }
    void done(void* x) {
        for (auto& y : p)
            if (y == x) {
                gfree(g, y);
                y = nullptr;
            }
    }
};
#define TALLOC(t, ptr, type, count)           \
    do {                                      \
        ALLOC(ptr, type, count);              \
        (t).p.push_back((void*)(ptr));        \
    } while (0)

// S = stored neighbours per point for a cost with k neighbours
int width_for(int k, int density_k1) {
    if (density_k1) return 8;  // the 8 nearest: the shell plus spares (k+b buffer)
    if (k <= 6) return 8;      // k nearest + at least 2 spare (k+b buffer)
    return 17;
}
int filt_width(int k) { return k <= 4 ? 4 : (k <= 8 ? 8 : 17); }

// Octree leaf levels, cell hash and full-mode groups over pos/code[0, ng).
int build_cells(pd_grid* g) {
    Scratch s = scratch_of(g);
    CK(launch_leaf_levels(g->code, g->ng, g->T, g->B, g->leaf, g->st));
    CK(launch_node_count(g->code, g->leaf, g->ng, g->B, g->d_u64, g->st));
    unsigned long long nodes = 0;
    CK(cudaMemcpyAsync(&nodes, g->d_u64, sizeof(nodes), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    u64 cap = 1024;
    while (cap < 2 * nodes) cap <<= 1;
    if (g->hash && g->hmask + 1 < cap) {
        gfree(g, g->hash);
        g->hash = nullptr;
    }
    if (!g->hash) {
        ALLOC(g->hash, HashSlot, cap);
        g->hmask = cap - 1;
    }
    CK(launch_node_insert(g->code, g->leaf, g->ng, g->B, g->hash, g->hmask, g->st));
    GridView v = view_of(g);
    CK(launch_leaf_groups(v, g->ng, g->groups, g->d_int, g->st));
    int ng = 0;
    CK(cudaMemcpyAsync(&ng, g->d_int, sizeof(int), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    g->ngroups = ng;
    (void)s;
    return PD_OK;
}

}  // namespace

// ============================================================ API: context
extern "C" int pd_ctx_create(const pd_allocator* alloc, pd_ctx** out) {
    if (!out) return PD_EINVAL;
    pd_ctx* c = new (std::nothrow) pd_ctx();
    if (!c) return PD_ENOMEM;
    c->has_alloc = 0;
    c->tuned_leaf = 0;
    c->err[0] = 0;
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->has_alloc = 1;
    }
    *out = c;
    return PD_OK;
}

extern "C" void pd_ctx_destroy(pd_ctx* ctx) { delete ctx; }

extern "C" int pd_ctx_set_device_budget(pd_ctx* ctx, uint64_t bytes, uint64_t spill_min) {
    if (!ctx) return PD_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mem_mu);
    ctx->dev_budget = bytes;
    ctx->spill_min = spill_min;
    ctx->tracked.store(true);
    return PD_OK;
}

extern "C" int pd_ctx_memory(pd_ctx* ctx, pd_memory* out) {
    if (!ctx || !out) return PD_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mem_mu);
    memset(out, 0, sizeof(*out));
    out->budget = ctx->dev_budget;
    out->device_bytes = ctx->dev_used;
    out->device_peak = ctx->dev_peak;
    out->host_bytes = ctx->host_used;
    out->host_peak = ctx->host_peak;
    out->tracked = ctx->tracked.load() ? 1 : 0;
    return PD_OK;
}

extern "C" int pd_ctx_reset_peaks(pd_ctx* ctx) {
    if (!ctx) return PD_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mem_mu);
    ctx->dev_peak = ctx->dev_used;
    ctx->host_peak = ctx->host_used;
    return PD_OK;
}

extern "C" const char* pd_strerror(int code) {
    switch (code) {
        case PD_OK: return "ok";
        case PD_EINVAL: return "invalid argument";
        case PD_ERANGE: return "coordinate spread too large (>= 2^25 mm)";
        case PD_ENOMEM: return "out of device memory";
        case PD_ECUDA: return "CUDA runtime error";
        case PD_ETIMEOUT: return "device wait timed out";
        case PD_EINTERNAL: return "internal error";
        default: return "unknown error";
    }
}

extern "C" const char* pd_last_error(const pd_ctx* ctx) { return ctx ? ctx->err : ""; }

// ============================================================ API: grid
static int grid_release(pd_grid* g) {
    void* ptrs[] = {g->pos, g->code, g->leaf, g->alive, g->rgb, g->nrm, g->hash, g->groups,
                    g->prim, g->nbr, g->rk2, g->flg, g->hz, g->d_int, g->d_u64, g->glist,
                    g->gcount, g->cmin, g->nbr0, g->seg, g->seg_chunk0, g->seg_items};
    for (void* p : ptrs) gfree(g, p);
    return PD_OK;
}

extern "C" int pd_grid_free(pd_grid* g) {
    if (!g) return PD_EINVAL;
    grid_release(g);
    cudaStreamSynchronize(g->st);
    delete g;
    return PD_OK;
}

extern "C" int pd_build_grid(pd_ctx* ctx, const int32_t* xyz_dev, const uint8_t* rgb_dev,
                             int64_t n, const pd_grid_params* params, void* stream,
                             pd_grid** out) {
    if (!ctx || !out || !xyz_dev || n < 1 || n >= (1ll << 31) - 64) {
        if (ctx) set_err(ctx, "pd_build_grid: invalid argument%s (n = %lld)", "", (long long)n);
        return PD_EINVAL;
    }
    int T = params && params->leaf_max ? params->leaf_max : (ctx->tuned_leaf ? ctx->tuned_leaf : 32);
    if (T < 4 || T > 32) {
        set_err(ctx, "pd_build_grid: leaf_max must be in [4, 32]%s (got %lld)", "", T);
        return PD_EINVAL;
    }
    pd_grid* g = new pd_grid();
    memset(&g->stats, 0, sizeof(g->stats));
    g->stats.leaf_max = g->T;
    g->ctx = ctx;
    g->st = (cudaStream_t)stream;
    g->trace = getenv("PD_TRACE") != nullptr;
    g->max_rounds = getenv("PD_MAX_ROUNDS") ? atoi(getenv("PD_MAX_ROUNDS")) : 0;
    // diagnostic: exact depth of the k = 1 searches (any depth gives the same
    // result; the stored list is complete below the reported horizon)
    g->k1_exact = getenv("PD_K1_EXACT") ? atoi(getenv("PD_K1_EXACT")) : 2;
    g->k1_exact_rq = getenv("PD_K1_EXACT_RQ") ? atoi(getenv("PD_K1_EXACT_RQ")) : 3;
    // diagnostic: 0 runs the re-searches per leaf group (same results)
    g->sparse_rq = getenv("PD_SPARSE_REQUERY") ? atoi(getenv("PD_SPARSE_REQUERY")) : 1;
    // 0: by cost (decimate_impl); PD_COMPACT_AT overrides
    g->compact_at = getenv("PD_COMPACT_AT") ? atof(getenv("PD_COMPACT_AT")) : 0.0;
    if (!(g->compact_at > 0.0 && g->compact_at < 1.0)) g->compact_at = 0.0;
    g->n = n;
    g->ng = n;
    g->T = T;
    g->stats.leaf_max = T;
    int rc = PD_OK;
    auto fail = [&](int code) {
        grid_release(g);
        delete g;
        return code;
    };
#define TRY(x)                  \
    do {                        \
        rc = (x);               \
        if (rc) return fail(rc); \
    } while (0)
    cudaEvent_t be0 = nullptr, be1 = nullptr;
    cudaEventCreate(&be0);
    cudaEventCreate(&be1);
    cudaEventRecord(be0, g->st);
    auto body = [&]() -> int {
        ALLOC(g->d_int, int, 8);
        ALLOC(g->d_u64, unsigned long long, 4);
        int* d6 = (int*)g->d_int;
        CK(launch_bbox(xyz_dev, n, d6, g->st));
        int h6[6];
        CK(cudaMemcpyAsync(h6, d6, sizeof(h6), cudaMemcpyDeviceToHost, g->st));
        CK(cudaStreamSynchronize(g->st));
        long long span = 0;
        for (int a = 0; a < 3; a++) span = std::max(span, (long long)h6[3 + a] - h6[a]);
        if (span >= (1ll << 25)) {
            set_err(ctx, "pd_build_grid: coordinate spread %s%lld mm >= 2^25", "", span);
            return PD_ERANGE;
        }
        g->origin = make_int3(h6[0], h6[1], h6[2]);
        g->umax = make_int3(h6[3] - h6[0], h6[4] - h6[1], h6[5] - h6[2]);
        int bits = 1;
        while ((1ll << bits) <= span) bits++;
        g->shift = bits > PD_MAXLEVEL ? bits - PD_MAXLEVEL : 0;
        g->B = bits - g->shift;
        if (g->B < 1) g->B = 1;
        ALLOC_COLD(g->code, u64, n);
        uint32_t* perm;
        Temps tmp(g);
        TALLOC(tmp, perm, uint32_t, n);
        Scratch s = scratch_of(g);
        CK(launch_morton(xyz_dev, n, g->origin, g->shift, g->code, perm, g->st));
        CK(radix_sort_pairs(g->code, perm, n, 3 * g->B, s, g->st));
        ALLOC(g->pos, int4, n);
        if (rgb_dev) ALLOC(g->rgb, uchar4, n);
        CK(launch_gather(xyz_dev, rgb_dev, nullptr, perm, n, g->pos, g->rgb, nullptr, g->st));
        tmp.done(perm);
        ALLOC(g->leaf, uint8_t, n);
        ALLOC(g->alive, uint8_t, n);
        CK(cudaMemsetAsync(g->alive, 1, n, g->st));
        ALLOC(g->groups, int4, n);
        return build_cells(g);
    };
    rc = body();
    cudaEventRecord(be1, g->st);
    float bms = 0.f;
    if (!rc && cudaEventSynchronize(be1) == cudaSuccess) cudaEventElapsedTime(&bms, be0, be1);
    cudaEventDestroy(be0);
    cudaEventDestroy(be1);
    if (rc) return fail(rc);
#undef TRY
    g->ms_grid = bms;
    g->stats.ms_grid = bms;
    *out = g;
    return PD_OK;
}

extern "C" int pd_grid_stats(const pd_grid* g, pd_stats* out) {
    if (!g || !out) return PD_EINVAL;
    *out = g->stats;
    return PD_OK;
}

// ============================================================ neighbour state
namespace {

int check_cost(pd_grid* g, const pd_cost_params* cp) {
    if (!cp || cp->k < 1 || cp->k > PD_KMAX || cp->term < 0 || cp->term > 2) {
        set_err(g->ctx, "invalid cost parameters%s (k = %lld)", "", cp ? cp->k : -1);
        return PD_EINVAL;
    }
    if (cp->term == PD_TERM_COLOR && !g->rgb) {
        set_err(g->ctx, "colour term needs rgb at pd_build_grid%s", "", 0);
        return PD_EINVAL;
    }
    if (cp->term == PD_TERM_ORIENT && !cp->normals_dev) {
        set_err(g->ctx, "orientation term needs normals_dev%s", "", 0);
        return PD_EINVAL;
    }
    return PD_OK;
}

// (Re)allocate the neighbour state for a cost and gather normals.
int prepare_state(pd_grid* g, const pd_cost_params* cp) {
    int dk1 = cp->k == 1 && cp->term == PD_TERM_NONE;
    int S = width_for(cp->k, dk1);
    if (g->nbr && g->S != S) {
        gfree(g, g->nbr);
        g->nbr = nullptr;
    }
    g->S = S;
    g->k = cp->k;
    g->density_k1 = dk1;
    if (!g->prim) ALLOC(g->prim, u64, g->n);
    if (!g->nbr) ALLOC(g->nbr, int, (size_t)g->n * S);
    if (dk1 && !g->nbr0) ALLOC(g->nbr0, int, g->n);
    if (!g->rk2) ALLOC_COLD(g->rk2, u64, g->n);
    if (!g->flg) ALLOC(g->flg, uint8_t, g->n);
    if (!g->hz) ALLOC_COLD(g->hz, u64, g->n);
    if (cp->term == PD_TERM_ORIENT) {
        if (!g->nrm) ALLOC(g->nrm, float4, g->n);
        // normals are given in input order: gather through pos[].w
        CK(launch_gather_nrm(cp->normals_dev, g->pos, g->ng, g->nrm, g->st));
    }
    return PD_OK;
}

KnnArgs base_args(pd_grid* g, const pd_cost_params* cp) {
    KnnArgs a;
    memset(&a, 0, sizeof(a));
    a.groups = g->groups;
    a.ngroups = g->ngroups;
    a.alive = g->alive;
    a.prim = g->prim;
    a.k = cp->k;
    a.S = g->S;
    a.density_k1 = g->density_k1;
    a.term = cp->term;
    a.weight = cp->weight;
    a.rgb = g->rgb;
    a.nrm = g->nrm;
    a.nbr = g->nbr;
    a.nbr0_out = g->density_k1 ? g->nbr0 : nullptr;
    a.prim_out = g->prim;
    a.rk2_out = g->rk2;
    a.flg_out = g->flg;
    a.hz_out = g->hz;
    a.cmin = g->cmin;
    if (g->density_k1 && g->k1_exact > 0) a.r_exact = g->k1_exact;
    return a;
}

// Deferred event timing: pairs of events recorded on the launching stream,
// resolved once at the end of a call (no synchronisation per launch).
struct Timers {
    struct Span {
        cudaEvent_t a, b;
        double* acc;
    };
    std::vector<Span> spans;
    cudaStream_t st;
    bool off = false;  // set while a round is captured into a graph
    explicit Timers(cudaStream_t s) : st(s) {}
    Span* open(double* acc) {
        Span sp;
        cudaEventCreate(&sp.a);
        cudaEventCreate(&sp.b);
        sp.acc = acc;
        cudaEventRecord(sp.a, st);
        spans.push_back(sp);
        return &spans.back();
    }
    void close() { cudaEventRecord(spans.back().b, st); }
    void resolve() {
        for (auto& sp : spans) {
            cudaEventSynchronize(sp.b);
            float ms = 0;
            cudaEventElapsedTime(&ms, sp.a, sp.b);
            *sp.acc += ms;
            cudaEventDestroy(sp.a);
            cudaEventDestroy(sp.b);
        }
        spans.clear();
    }
    ~Timers() { resolve(); }
};
struct Span {
    Timers& t;
    bool on;
    Span(Timers& tt, double* acc) : t(tt), on(!tt.off) {
        if (on) t.open(acc);
    }
    ~Span() {
        if (on) t.close();
    }
};

// kNN over every grid point (full mode)
int knn_all(pd_grid* g, const pd_cost_params* cp, double* cost_s) {
    KnnArgs a = base_args(g, cp);
    a.cost_out = cost_s;
    CK(launch_knn(view_of(g), a, g->st));
    return PD_OK;
}

// Compact the live points into a fresh grid order (keeps Morton order) and
// rebuild the cell table; stored neighbours are remapped (A7).
int compact_rebuild(pd_grid* g, bool remap_state) {
    Scratch s = scratch_of(g);
    Temps tmp(g);
    int* list;
    TALLOC(tmp, list, int, g->ng);
    int* d_cnt = g->d_int + 2;
    CK(stable_compact(g->alive, g->ng, list, d_cnt, s, g->st));
    int nl = 0;
    CK(cudaMemcpyAsync(&nl, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    // the compacted arrays hold the live points only
    const int64_t cn = nl > 0 ? nl : 1;
    int* newpos;
    TALLOC(tmp, newpos, int, g->ng);
    CK(cudaMemsetAsync(newpos, 0xff, g->ng * sizeof(int), g->st));  // -1: not kept
    CK(launch_newpos(list, nl, newpos, g->st));
    int4* pos2;
    ALLOC(pos2, int4, cn);
    CK(launch_take_i4(list, nl, g->pos, pos2, g->st));
    gfree(g, g->pos);
    g->pos = pos2;
    u64* code2;
    ALLOC_COLD(code2, u64, cn);
    CK(launch_take_u64(list, nl, g->code, code2, g->st));
    gfree(g, g->code);
    g->code = code2;
    if (g->rgb) {
        uchar4* r2;
        ALLOC(r2, uchar4, cn);
        CK(launch_take_uc4(list, nl, g->rgb, r2, g->st));
        gfree(g, g->rgb);
        g->rgb = r2;
    }
    if (g->nrm) {
        float4* n2;
        ALLOC(n2, float4, cn);
        CK(launch_take_f4(list, nl, g->nrm, n2, g->st));
        gfree(g, g->nrm);
        g->nrm = n2;
    }
    if (remap_state) {
        u64* p2;
        ALLOC(p2, u64, cn);
        CK(launch_take_u64(list, nl, g->prim, p2, g->st));
        gfree(g, g->prim);
        g->prim = p2;
        u64* r2;
        ALLOC_COLD(r2, u64, cn);
        CK(launch_take_u64(list, nl, g->rk2, r2, g->st));
        gfree(g, g->rk2);
        g->rk2 = r2;
        uint8_t* f2;
        ALLOC(f2, uint8_t, cn);
        CK(launch_take_u8(list, nl, g->flg, f2, g->st));
        gfree(g, g->flg);
        g->flg = f2;
        u64* h2;
        ALLOC_COLD(h2, u64, cn);
        CK(launch_take_u64(list, nl, g->hz, h2, g->st));
        gfree(g, g->hz);
        g->hz = h2;
        int* nb2;
        ALLOC(nb2, int, (size_t)cn * g->S);
        CK(launch_remap(list, nl, g->nbr, nb2, newpos, g->ng, g->S, g->st));
        gfree(g, g->nbr);
        g->nbr = nb2;
        if (g->nbr0) {
            int* n02;
            ALLOC(n02, int, cn);
            CK(launch_remap(list, nl, g->nbr0, n02, newpos, g->ng, 1, g->st));
            gfree(g, g->nbr0);
            g->nbr0 = n02;
        }
    }
    tmp.done(newpos);
    tmp.done(list);
    g->ng = nl;
    CK(cudaMemsetAsync(g->alive, 1, nl, g->st));
    g->stats.grid_builds++;
    return build_cells(g);
}

// r-th largest live key (1-based).  With band_rank > 0 also returns the
// lower boundary of the first-digit bin holding the band_rank-th largest key.
struct Sel {
    u64 prim;
    int idx;
};

Sel key_from_digits(const uint32_t* d, int npass) {
    // 96-bit value with digits 0..npass-1 set and the rest zero
    unsigned __int128 v = 0;
    for (int p = 0; p < 8; p++) {
        v <<= 12;
        if (p < npass) v |= d[p];
    }
    Sel s;
    s.prim = (u64)(v >> 32);
    s.idx = (int)(uint32_t)v;
    return s;
}

int select_rank(pd_grid* g, const u64* prim, const uint8_t* alive, int64_t r, int64_t band_rank,
                Sel* out, Sel* band_out) {
    Temps tmp(g);
    uint32_t* hist;
    TALLOC(tmp, hist, uint32_t, 4096);
    std::vector<uint32_t> h(4096);
    uint32_t pre[8] = {0};
    u64* bufA = nullptr;
    int* idA = nullptr;
    int64_t len = 0;
    int* d_cnt = g->d_int + 3;
    int rc = PD_OK;
    bool done = false;
    for (int pass = 0; pass < 8 && !done; pass++) {
        CK(launch_sel_hist(prim, alive, g->ng, pass ? bufA : nullptr, idA, len, pass, pre, hist,
                           g->st));
        CK(cudaMemcpyAsync(h.data(), hist, 4096 * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                           g->st));
        CK(cudaStreamSynchronize(g->st));
        int64_t cum = 0;
        int b = 4095;
        for (; b >= 0; b--) {
            if (cum + h[b] >= r) break;
            cum += h[b];
        }
        if (b < 0) {
            set_err(g->ctx, "select_rank: rank beyond live count%s (r = %lld)", "", r);
            rc = PD_EINTERNAL;
            break;
        }
        if (pass == 0 && band_out) {
            int64_t c2 = 0;
            int bb = 4095;
            for (; bb > 0; bb--) {
                if (c2 + h[bb] >= band_rank) break;
                c2 += h[bb];
            }
            uint32_t d0[8] = {(uint32_t)bb};
            *band_out = key_from_digits(d0, 1);
        }
        pre[pass] = (uint32_t)b;
        if (cum + h[b] == r || pass == 7) {
            *out = key_from_digits(pre, pass + 1);
            done = true;
            break;
        }
        r -= cum;
        int64_t nlen = h[b];
        u64* nb;
        int* ni;
        TALLOC(tmp, nb, u64, nlen);
        TALLOC(tmp, ni, int, nlen);
        CK(launch_sel_compact(prim, g->pos, alive, g->ng, pass ? bufA : nullptr, idA, len, pass,
                              pre, nb, ni, d_cnt, g->st));
        if (bufA) {
            tmp.done(bufA);
            tmp.done(idA);
        }
        bufA = nb;
        idA = ni;
        len = nlen;
    }
    return rc;
}


BufView bufview(pd_grid* g, const pd_cost_params* cp) {
    BufView b;
    b.pos = g->pos;
    b.prim = g->prim;
    b.nbr = g->nbr;
    b.nbr0 = g->density_k1 ? g->nbr0 : nullptr;
    b.rk2 = g->rk2;
    b.flg = g->flg;
    b.hz = g->hz;
    b.rgb = g->rgb;
    b.nrm = g->nrm;
    b.term = cp->term;
    b.weight = cp->weight;
    return b;
}

// kNN over the leaf groups, querying only the points whose flag is set.
int knn_flag(pd_grid* g, const pd_cost_params* cp, int filter, int S, const uint8_t* qflag,
             u64* fout, const RoundDev* rd) {
    KnnArgs a = base_args(g, cp);
    a.filter = filter;
    a.S = S;
    a.qflag = qflag;
    a.rd = rd;
    if (filter == FILT_BELOW_SELF) a.fprim_out = fout;
    if (filter == FILT_BELOW_TAU) a.lam_out = fout;
    if (filter == FILT_NONE && g->sparse_rq && g->rq_list) {
        // k = 1 density re-searches: the flagged points, listed, 2 lanes each
        // over their own cells (the weighted and k >= 2 rounds re-search few
        // points per round, where a warp per flagged group measured faster)
        ArenaUse au;
        if (g->k1_exact_rq > 0) a.r_exact = g->k1_exact_rq;
        CK(stable_compact(qflag, g->ng, g->rq_list, g->rq_count, round_scratch(g, &au), g->st));
        CK(launch_knn_sparse(view_of(g), a, g->rq_list, g->rq_count, g->ng, g->st));
        return PD_OK;
    }
    if (!g->glist) {  // groups never outnumber the points of the first build
        ALLOC(g->glist, int, g->n);
        ALLOC(g->gcount, int, 1);
    }
    CK(launch_knn_flagged(view_of(g), a, g->glist, g->gcount, g->st));
    return PD_OK;
}

// A round the device could not settle: the danger analysis overflowed (or
// fewer than k low points exist), or the fixpoint needed more sweeps.
int settle_round(pd_grid* g, RoundDev* rd, const RoundDev& h, uint8_t* inP, uint8_t* rej,
                 int* dep, int* cand, int2* pairs, int pair_cap, SelBuffers* sel,
                 uint32_t* seg_hist, int64_t* removed) {
    int* d = g->d_int;
    if (h.overflow) {
        // drop this round's candidates and remove the global maximum only
        CK(launch_remove(cand, &rd->ncand, 0, inP, rej, g->alive, g->d_u64, g->st));
        CK(cudaMemsetAsync(inP, 0, g->ng, g->st));
        CK(cudaMemsetAsync(rej, 0, g->ng, g->st));
        CK(cudaMemsetAsync(d + 4, 0, sizeof(int), g->st));
        if (g->nseg) {
            // packed batch: the largest key of every scan still above its
            // target (each is its scan's next sequential pop)
            int one = 1, zero = 0;
            CK(cudaMemcpyAsync(&rd->seg_rank_one, &one, sizeof(int), cudaMemcpyHostToDevice,
                               g->st));
            CK(seg_launch_select(g->prim, g->pos, g->alive, g->ng, *sel, seg_hist, rd, g->seg,
                                 g->seg_chunk0, g->seg_items, g->nseg, g->st));
            CK(cudaMemcpyAsync(&rd->seg_rank_one, &zero, sizeof(int), cudaMemcpyHostToDevice,
                               g->st));
            CK(seg_launch_accept(g->prim, g->pos, g->alive, g->ng, rd, inP, cand, d + 4, g->st));
            CK(launch_remove(cand, d + 4, g->nseg, inP, rej, g->alive, g->d_u64, g->st));
        } else {
            Sel top;
            int rc = select_rank(g, g->prim, g->alive, 1, 0, &top, nullptr);
            if (rc) return rc;
            CK(launch_accept_above(g->prim, g->pos, g->alive, g->ng, top.prim, top.idx, inP, cand,
                                   d + 4, g->st));
            CK(launch_remove(cand, d + 4, 1, inP, rej, g->alive, g->d_u64, g->st));
        }
    } else {
        // keep sweeping the fixpoint until nothing changes
        for (int it = 0; it < 1000000; it++) {
            CK(cudaMemsetAsync(d + 6, 0, sizeof(int), g->st));
            if (g->density_k1)
                CK(launch_k1_fix(dep, &rd->ndep, h.ndep, g->pos, g->nbr, g->flg, g->S, inP,
                                 rej, d + 6, g->st));
            else
                CK(launch_pair_fix(pairs, &rd->npairs, std::min(h.npairs, pair_cap), pair_cap,
                                   inP, rej, d + 6, g->st));
            int ch = 0;
            CK(cudaMemcpyAsync(&ch, d + 6, sizeof(int), cudaMemcpyDeviceToHost, g->st));
            CK(cudaStreamSynchronize(g->st));
            if (!ch) break;
        }
        CK(launch_remove(cand, &rd->ncand, h.ncand, inP, rej, g->alive, g->d_u64, g->st));
    }
    unsigned long long r = 0;
    CK(cudaMemcpyAsync(&r, g->d_u64, sizeof(r), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    *removed = (int64_t)r;
    return PD_OK;
}

static_assert(PD_BATCH_MAX_SCANS == PD_SEG_MAX, "packed batch scan limit");

// A packed batch one of whose scans has more coincident points than it must
// lose: the batch runs its scans one grid each instead.
#define PD_SEG_FALLBACK 100

// Duplicate phase: coincident points beyond the smallest index of their
// class are the first pops of the sequential greedy (their cost is +inf).
int remove_duplicates(pd_grid* g, int64_t need, int64_t* removed,
                      const std::vector<long long>* seg_need = nullptr) {
    *removed = 0;
    Temps tmp(g);
    uint8_t* dup;
    TALLOC(tmp, dup, uint8_t, g->ng);
    CK(launch_dup_flag(g->code, g->pos, g->ng, dup, g->d_u64, g->st));
    unsigned long long nd = 0;
    CK(cudaMemcpyAsync(&nd, g->d_u64, sizeof(nd), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    if (g->nseg && nd > 0) {
        // packed batch: every scan must be able to lose all its duplicates
        unsigned long long* cnt;
        TALLOC(tmp, cnt, unsigned long long, g->nseg);
        CK(cudaMemsetAsync(cnt, 0, g->nseg * sizeof(*cnt), g->st));
        CK(seg_launch_count(dup, g->pos, g->ng, g->seg_shift, cnt, g->st));
        std::vector<unsigned long long> hc(g->nseg);
        CK(cudaMemcpyAsync(hc.data(), cnt, g->nseg * sizeof(*cnt), cudaMemcpyDeviceToHost,
                           g->st));
        CK(cudaStreamSynchronize(g->st));
        for (int i = 0; i < g->nseg; i++)
            if ((long long)hc[i] > (*seg_need)[i]) return PD_SEG_FALLBACK;
        *removed = (int64_t)nd;
        CK(launch_dup_remove(dup, g->pos, g->ng, 0, g->alive, g->st));
        return PD_OK;
    }
    int idx_min = 0;
    if (nd > 0 && need > 0) {
        if ((int64_t)nd > need) {
            // the need largest input indices among the duplicates
            u64* zeros;
            TALLOC(tmp, zeros, u64, g->ng);
            CK(cudaMemsetAsync(zeros, 0, g->ng * sizeof(u64), g->st));
            Sel s;
            int rc = select_rank(g, zeros, dup, need, 0, &s, nullptr);
            tmp.done(zeros);
            if (rc) return rc;
            idx_min = s.idx;
            *removed = need;
        } else {
            *removed = (int64_t)nd;
        }
        CK(launch_dup_remove(dup, g->pos, g->ng, idx_min, g->alive, g->st));
    }
    return PD_OK;
}

// Scratch and events of one decimation, released (stream-ordered) on every
// exit path, errors included.
struct RoundScratch {
    pd_grid* g;
    std::vector<void*> ptrs;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // replayed rounds: the instantiated graph, its stream and fork/join events
    cudaGraphExec_t gx = nullptr;
    cudaStream_t gs = nullptr;
    cudaEvent_t gfork = nullptr, gjoin = nullptr;
    cudaEvent_t tq0 = nullptr, tq1 = nullptr;  // trace only: a round's re-search time
    explicit RoundScratch(pd_grid* gg) : g(gg) {}
    ~RoundScratch() {
        if (tq0) cudaEventDestroy(tq0);
        if (tq1) cudaEventDestroy(tq1);
        if (gx) cudaGraphExecDestroy(gx);
        if (gs) {
            cudaStreamSynchronize(gs);
            cudaStreamDestroy(gs);
        }
        if (gfork) cudaEventDestroy(gfork);
        if (gjoin) cudaEventDestroy(gjoin);
        for (void* p : ptrs) gfree(g, p);
        gfree(g, g->cmin);
        g->cmin = nullptr;
        g->rq_list = nullptr;  // released with ptrs
        g->rq_count = nullptr;
        g->arena = nullptr;
        g->arena_cap = 0;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};
#define RALLOC(ptr, type, count)              \
    do {                                      \
        ALLOC(ptr, type, count);              \
        rs.ptrs.push_back((void*)(ptr));      \
    } while (0)

// kernel nodes of a captured graph (launch accounting of replayed rounds)
long long count_kernel_nodes(cudaGraph_t graph) {
    size_t nn = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) != cudaSuccess || nn == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(graph, nodes.data(), &nn) != cudaSuccess) return 0;
    long long c = 0;
    for (size_t i = 0; i < nn; i++) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) c++;
    }
    return c;
}

int decimate_impl(pd_grid* g, const pd_cost_params* cp, int64_t m, uint8_t* keep_dev) {
    int rc = check_cost(g, cp);
    if (rc) return rc;
    if (m < 0 || m > g->n || !keep_dev) {
        set_err(g->ctx, "pd_decimate: m must be in [0, n] and keep_dev set%s (m = %lld)", "", m);
        return PD_EINVAL;
    }
    if (g->ng != g->n) {
        set_err(g->ctx, "pd_decimate: grid already decimated; build a new one%s", "", 0);
        return PD_EINVAL;
    }
    memset(&g->stats, 0, sizeof(g->stats));
    g->stats.leaf_max = g->T;
    g->stats.n = g->n;
    g->stats.m = m;
    g->stats.ms_grid = g->ms_grid;
    long long launches0 = g_launch_count;
    RoundScratch rs(g);
    Timers T(g->st);
    cudaEventCreate(&rs.e0);
    cudaEventCreate(&rs.e1);
    cudaEvent_t e0 = rs.e0, e1 = rs.e1;
    cudaEventRecord(e0, g->st);
    rc = prepare_state(g, cp);
    if (rc) return rc;
    int k = cp->k;
    // k >= 2 candidate band: fraction of the live points examined per round.
    // It adapts to the cloud: halved when a round's danger analysis overflows
    // or its yield is poor (the band then covers whole dense regions with no
    // lower keys inside), grown again while yields stay high.  Any band gives
    // the same result; only the number of rounds changes.
    double band_max = cp->band > 0 ? cp->band : 0.02;
    // small clouds: examine at least ~4096 keys per round
    if (cp->band <= 0 && g->n > 0) band_max = std::max(band_max, std::min(0.5, 4096.0 / g->n));
    // colour / orientation weights make costs non-monotone (a removal can
    // raise a neighbour's cost), so the rounds are no longer provably the
    // sequential order: a narrow band keeps them close to it
    if (cp->band <= 0 && cp->term != PD_TERM_NONE) band_max = 0.01;
    int64_t live = g->n;
    // ---- duplicate phase
    int64_t nd = 0;
    std::vector<long long> seg_need;
    for (int i = 0; i < g->nseg; i++) seg_need.push_back(g->seg_n[i] - g->seg_m[i]);
    rc = remove_duplicates(g, live - m, &nd, g->nseg ? &seg_need : nullptr);
    if (rc) return rc;
    g->stats.dup_removed = nd;
    live -= nd;
    if (nd > 0) {
        rc = compact_rebuild(g, false);
        if (rc) return rc;
    }
    // packed batch: every scan's grid range and its selection work items
    if (g->nseg)
        CK(seg_launch_ranges(g->pos, g->ng, g->seg, g->seg_chunk0, g->seg_items, g->nseg,
                             g->seg_shift, g->st));
    // ---- first neighbour pass
    {
        unsigned long long* dpairs;
        RALLOC(dpairs, unsigned long long, PD_PAIR_SLOTS);
        CK(cudaMemsetAsync(dpairs, 0, PD_PAIR_SLOTS * sizeof(*dpairs), g->st));
        {
            Span t(T, &g->stats.ms_knn_first);
            KnnArgs a = base_args(g, cp);
            a.pairs_out = dpairs;
            CK(launch_knn(view_of(g), a, g->st));
        }
        unsigned long long hp[PD_PAIR_SLOTS];
        CK(cudaMemcpyAsync(hp, dpairs, sizeof(hp), cudaMemcpyDeviceToHost, g->st));
        CK(cudaStreamSynchronize(g->st));
        unsigned long long pairs = 0;
        for (int i = 0; i < PD_PAIR_SLOTS; i++) pairs += hp[i];
        g->stats.pairs_first = (int64_t)pairs;
    }
    g->stats.q_first = g->ng;
    int S = g->S;
    int Sf = filt_width(k);
    int kchk = g->density_k1 ? S : k;
    bool use_buf = !g->density_k1 && S <= 8;
    uint8_t *inP, *rej, *dirty, *fqf = nullptr, *dgf = nullptr;  // dgf: lambda search flags
    int *cand, *slow, *src = nullptr, *csort = nullptr, *dep = nullptr;
    u64 *fprim = nullptr, *lam = nullptr;
    int2* pairs = nullptr;
    int64_t cap = g->n;
    RALLOC(inP, uint8_t, cap);
    RALLOC(rej, uint8_t, cap);
    RALLOC(dirty, uint8_t, cap);
    if (g->sparse_rq && g->density_k1) {
        RALLOC(g->rq_list, int, cap);
        RALLOC(g->rq_count, int, 1);
    }
    {
        // offsets of one compaction (a word per 1024 points) and the sums of
        // its scan (a word per 1024 offsets, recursively), 256-byte aligned
        size_t nb = (size_t)(cap + 1023) / 1024;
        size_t words = nb + nb / 512 + 64;
        g->arena_cap = words * 4 + 8 * 256;
        RALLOC(g->arena, char, g->arena_cap);
    }
    RALLOC(cand, int, cap);
    RALLOC(slow, int, cap);
    if (g->density_k1) RALLOC(dep, int, cap);
    CK(cudaMemsetAsync(inP, 0, cap, g->st));
    CK(cudaMemsetAsync(rej, 0, cap, g->st));
    int pair_cap = 0;
    if (!g->density_k1) {
        RALLOC(fqf, uint8_t, cap);
        RALLOC(dgf, uint8_t, cap);
        RALLOC(src, int, cap);
        RALLOC(csort, int, cap);
        RALLOC(fprim, u64, cap);
        RALLOC(lam, u64, cap);
        pair_cap = (int)std::min<int64_t>(std::max<int64_t>(cap * 4, 1 << 16), 1 << 30);
        // diagnostic: a smaller danger-pair capacity forces the host settle of
        // overflowing rounds (the result does not change, only the rounds)
        if (getenv("PD_PAIR_CAP")) {
            int v = atoi(getenv("PD_PAIR_CAP"));
            if (v >= 1 && v < pair_cap) pair_cap = v;
        }
        RALLOC(pairs, int2, pair_cap);
        ALLOC(g->cmin, u64, (cap + 31) / 32 + 1);
    }
    SelBuffers sb;
    RALLOC(sb.p[0], u64, cap);
    RALLOC(sb.p[1], u64, cap);
    RALLOC(sb.i[0], int, cap);
    RALLOC(sb.i[1], int, cap);
    RALLOC(sb.hist, uint32_t, 4096);
    CK(cudaMemsetAsync(sb.hist, 0, 4096 * sizeof(uint32_t), g->st));
    RoundDev* rd;
    RALLOC(rd, RoundDev, 1);
    uint32_t* seg_hist = nullptr;  // packed batch: a 4096-bin histogram per scan
    if (g->nseg) {
        RALLOC(seg_hist, uint32_t, (size_t)g->nseg * 4096);
        CK(cudaMemsetAsync(seg_hist, 0, (size_t)g->nseg * 4096 * sizeof(uint32_t), g->st));
    }
    RoundDev h;
    memset(&h, 0, sizeof(h));
    if (g->nseg) {
        h.seg = g->seg;
        h.seg_chunk0 = g->seg_chunk0;
        h.nseg = g->nseg;
        h.seg_shift = g->seg_shift;
    }
    h.live = live;
    h.m = m;
    h.band = band_max;
    h.band_max = band_max;
    h.density_k1 = g->density_k1;
    h.band_mode = getenv("PD_BAND_MODE") ? atoi(getenv("PD_BAND_MODE")) : 1;
    h.fix_iters = g->density_k1 ? PD_FIX_ITERS : PD_FIX_ITERS_KK;
    if (g->density_k1 && getenv("PD_FIX_SWEEPS"))  // fewer sweeps: more rounds settled on the host
        h.fix_iters = std::max(1, std::min(PD_FIX_ITERS, atoi(getenv("PD_FIX_SWEEPS"))));
    CK(cudaMemcpyAsync(rd, &h, sizeof(h), cudaMemcpyHostToDevice, g->st));
    int64_t built = live;
    // small clouds are bound by launches: from the third round on, a round's
    // launches are captured into a CUDA graph and replayed (PD_ROUND_GRAPH:
    // 1 always, 0 never; default for grids up to 8M points and packed batches)
    bool round_graph = g->n <= ((int64_t)8 << 20) || g->nseg > 0;
    if (getenv("PD_ROUND_GRAPH")) round_graph = atoi(getenv("PD_ROUND_GRAPH")) != 0;
    void* graph_pos = nullptr;
    long long graph_kernels = 0;
    if (g->trace) {
        cudaEventCreate(&rs.tq0);
        cudaEventCreate(&rs.tq1);
    }
    cudaEvent_t tq0 = rs.tq0, tq1 = rs.tq1;
    auto issue_round = [&]() -> int {
            GridView v = view_of(g);
            CK(round_launch_setup(rd, g->st));
            {
                Span t(T, &g->stats.ms_select);
                if (g->nseg)
                    CK(seg_launch_select(g->prim, g->pos, g->alive, g->ng, sb, seg_hist, rd,
                                         g->seg, g->seg_chunk0, g->seg_items, g->nseg, g->st));
                else
                    CK(round_launch_select(g->prim, g->pos, g->alive, g->ng, sb, rd, g->st));
            }
            if (g->density_k1) {
                CK(round_launch_k1(v, g->prim, g->alive, g->nbr, g->nbr0, g->flg, g->rk2, g->ng, S,
                                   rd, inP, rej, cand, slow, dep, h.fix_iters, g->st));
            } else {
                BufView bv = bufview(g, cp);
                CK(round_launch_kk_cand2(bv, g->alive, g->ng, S, k, rd, inP, cand, fqf, dgf, lam, src,
                                         g->st));
                CK(launch_chunk_min(g->prim, g->alive, g->ng, g->cmin, g->st));
                {
                    Span t(T, &g->stats.ms_knn);
                    rc = knn_flag(g, cp, FILT_BELOW_SELF, Sf, fqf, fprim, rd);
                    if (rc) return rc;
                }
                CK(round_launch_kk_accept(fqf, g->prim, fprim, g->ng, rd, inP, cand, g->st));
                {
                    Span t(T, &g->stats.ms_knn);
                    rc = knn_flag(g, cp, FILT_BELOW_TAU, Sf, dgf, lam, rd);
                    if (rc) return rc;
                }
                {
                    Span t(T, &g->stats.ms_danger);
                    // candidates in Morton order, so each source finds its own by search
                    ArenaUse au;
                    CK(stable_compact(inP, g->ng, csort, &rd->ncs, round_scratch(g, &au), g->st));
                    CK(round_launch_danger(v, src, g->prim, g->alive, inP, rej, lam, g->nbr, S, k,
                                           pairs, pair_cap, csort, rd, g->st));
                }
                CK(round_launch_pairs_fix(pairs, pair_cap, inP, rej, rd, g->st));
            }
            CK(round_launch_remove(cand, inP, rej, g->alive, rd, g->st));
            if (g->density_k1) {
                // absorb removals in the stored 8 nearest; search where the new
                // nearest shell may be incomplete
                CK(round_launch_k1_update(bufview(g, cp), g->alive, g->ng, S, dirty, rd, g->st));
            } else if (use_buf) {
                // absorb removals in the k+b buffers; search only where < k remain
                CK(round_launch_kk_update(bufview(g, cp), g->alive, g->ng, S, k, dirty, rd, g->st));
            } else {
                CK(round_launch_dirty(g->alive, g->nbr, g->ng, S, kchk, dirty, rd, g->st));
            }
            if (g->trace) cudaEventRecord(tq0, g->st);
            {
                Span t(T, &g->stats.ms_knn_requery);
                rc = knn_flag(g, cp, FILT_NONE, S, dirty, nullptr, rd);
                if (rc) return rc;
            }
            if (g->trace) cudaEventRecord(tq1, g->st);
            CK(round_launch_finish(rd, g->st));
            return PD_OK;
    };
    while (live > m) {
        g->stats.rounds++;
        g->stats.live_rounds += live;
        if (g->max_rounds && g->stats.rounds > g->max_rounds) {
            set_err(g->ctx, "pd_decimate: stopped after %s%lld rounds (PD_MAX_ROUNDS)", "",
                    (long long)g->max_rounds);
            return PD_EINTERNAL;
        }
        if (g->stats.rounds > 1000000) {
            set_err(g->ctx, "pd_decimate: round limit reached%s (live = %lld)", "", live);
            return PD_EINTERNAL;
        }
        int rr = PD_OK;
        const bool replay = round_graph && g->stats.rounds >= 3 && !g->trace;
        if (replay && (!rs.gx || graph_pos != (void*)g->pos)) {
            // capture this round's launches once per grid layout (compaction
            // replaces the arrays) on a private stream, then replay the graph
            if (rs.gx) {
                cudaGraphExecDestroy(rs.gx);
                rs.gx = nullptr;
            }
            if (!rs.gs) {
                cudaStreamCreateWithFlags(&rs.gs, cudaStreamNonBlocking);
                cudaEventCreateWithFlags(&rs.gfork, cudaEventDisableTiming);
                cudaEventCreateWithFlags(&rs.gjoin, cudaEventDisableTiming);
            }
            cudaStream_t caller = g->st;
            g->st = rs.gs;
            T.off = true;
            cudaGraph_t graph = nullptr;
            cudaError_t eb = cudaStreamBeginCapture(rs.gs, cudaStreamCaptureModeThreadLocal);
            int rc_cap = eb ? PD_ECUDA : issue_round();
            cudaError_t ee = eb ? cudaSuccess : cudaStreamEndCapture(rs.gs, &graph);
            g->st = caller;
            T.off = false;
            if (!eb && !rc_cap && !ee && graph &&
                cudaGraphInstantiate(&rs.gx, graph, 0) == cudaSuccess) {
                graph_pos = (void*)g->pos;
                // the captured launches ran nothing; each replay runs its kernel nodes
                graph_kernels = count_kernel_nodes(graph);
                __atomic_fetch_sub(&g_launch_count, graph_kernels, __ATOMIC_RELAXED);
            } else {
                rs.gx = nullptr;
                round_graph = false;  // capture refused: launch the rounds directly
                cudaGetLastError();
            }
            if (graph) cudaGraphDestroy(graph);
        }
        if (replay && rs.gx) {
            CK(cudaEventRecord(rs.gfork, g->st));
            CK(cudaStreamWaitEvent(rs.gs, rs.gfork, 0));
            CK(cudaGraphLaunch(rs.gx, rs.gs));
            CK(cudaEventRecord(rs.gjoin, rs.gs));
            CK(cudaStreamWaitEvent(g->st, rs.gjoin, 0));
            g->stats.graph_rounds++;
            __atomic_fetch_add(&g_launch_count, graph_kernels, __ATOMIC_RELAXED);
        } else {
            rr = issue_round();
            if (rr) return rr;
        }
        CK(cudaMemcpyAsync(&h, rd, sizeof(h), cudaMemcpyDeviceToHost, g->st));
        CK(cudaStreamSynchronize(g->st));
        if (h.overflow || h.fix_unconverged) {
            // settle on the host: finish the fixpoint, or (danger overflow / too
            // few low points) take only the global maximum, always removable
            int64_t removed = 0;
            rc = settle_round(g, rd, h, inP, rej, dep, cand, pairs, pair_cap, &sb, seg_hist,
                              &removed);
            if (rc) return rc;
            if (g->density_k1)
                CK(round_launch_k1_update(bufview(g, cp), g->alive, g->ng, S, dirty, rd, g->st));
            else if (use_buf)
                CK(round_launch_kk_update(bufview(g, cp), g->alive, g->ng, S, k, dirty, rd, g->st));
            else
                CK(round_launch_dirty(g->alive, g->nbr, g->ng, S, kchk, dirty, rd, g->st));
            {
                Span t(T, &g->stats.ms_knn_requery);
                rc = knn_flag(g, cp, FILT_NONE, S, dirty, nullptr, rd);
                if (rc) return rc;
            }
            h.live -= removed;
            h.removed = (unsigned long long)removed;
            if (!g->density_k1) {
                // an overflowing round always narrows the band, as before
                h.band = host_next_band(h.band, h.band_max, h.band_mode,
                                        h.cap_over + (h.overflow ? 1 : 0), h.ncand, h.removed);
                CK(cudaMemcpyAsync(&rd->band, &h.band, sizeof(h.band), cudaMemcpyHostToDevice,
                                   g->st));
            }
            CK(cudaMemcpyAsync(&rd->live, &h.live, sizeof(h.live), cudaMemcpyHostToDevice,
                               g->st));
            CK(cudaMemcpyAsync(&rd->tot_requery, &h.tot_requery, sizeof(u64),
                               cudaMemcpyHostToDevice, g->st));
        }
        if (g->trace) {
            float rq_ms = 0.f;
            cudaEventSynchronize(tq1);
            cudaEventElapsedTime(&rq_ms, tq0, tq1);
            fprintf(stderr, "pd round %d live %lld need %lld cand %d removed %llu band %.3g "
                    "sources %d pairs %d cap-over %llu requeries %llu (%.2f ms)%s\n",
                    g->stats.rounds, (long long)live, (long long)(live - m), h.ncand, h.removed,
                    h.band, h.nsrc, h.npairs, h.cap_over, h.tot_requery, rq_ms,
                    h.overflow ? " overflow" : (h.fix_unconverged ? " unconverged" : ""));
        }
        if (h.removed == 0 || (int64_t)h.removed > live - m) {
            set_err(g->ctx, "pd_decimate: round removed %s%lld points", "", (long long)h.removed);
            return PD_EINTERNAL;
        }
        live = h.live;
        if (live <= m) break;
        // every live point now stores live neighbours only: safe to compact
        // k = 1 re-searches are cheap next to a rebuild (measured best at
        // 0.6 on the billion-point scan); the k >= 2 rounds are many and
        // scan their dead points every round (0.7)
        const double at = g->compact_at > 0.0 ? g->compact_at : (g->density_k1 ? 0.6 : 0.7);
        if ((double)live < at * (double)built) {
            Span t(T, &g->stats.ms_build);
            rc = compact_rebuild(g, true);
            if (rc) return rc;
            if (g->nseg)
                CK(seg_launch_ranges(g->pos, g->ng, g->seg, g->seg_chunk0, g->seg_items,
                                     g->nseg, g->seg_shift, g->st));
            built = live;
        }
    }
    g->stats.requeries = (int64_t)h.tot_requery;
    g->stats.filtered_queries = (int64_t)h.tot_filtered;
    g->stats.danger_queries = (int64_t)h.tot_lambda;
    CK(cudaMemsetAsync(keep_dev, 0, g->n, g->st));
    CK(launch_keep(g->pos, g->alive, g->ng, keep_dev, g->st));
    cudaEventRecord(e1, g->st);
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    g->stats.ms_total = ms;
    T.resolve();
    g->stats.ms_knn += g->stats.ms_knn_first + g->stats.ms_knn_requery;
    g->stats.ms_rules = ms - g->stats.ms_knn - g->stats.ms_build;
    g->stats.launches = g_launch_count - launches0;
    g->ng = 0;  // consumed
    return PD_OK;
}

}  // namespace

// The paper's iterative w_up scheme with parallel removal rounds (wup.cu).
static int wup_impl(pd_grid* g, const pd_cost_params* cp, int64_t m, uint8_t* keep_dev) {
    if (!cp || cp->k < 1 || cp->k > 6 || cp->term != PD_TERM_NONE) {
        set_err(g->ctx, "pd_decimate_wup: density cost with k in [1, 6] only%s (k = %lld)", "",
                cp ? cp->k : -1);
        return PD_EINVAL;
    }
    if (m < 0 || m > g->n || !keep_dev) {
        set_err(g->ctx, "pd_decimate_wup: m must be in [0, n] and keep_dev set%s (m = %lld)", "",
                m);
        return PD_EINVAL;
    }
    if (g->ng != g->n) {
        set_err(g->ctx, "pd_decimate_wup: grid already decimated; build a new one%s", "", 0);
        return PD_EINVAL;
    }
    memset(&g->stats, 0, sizeof(g->stats));
    g->stats.leaf_max = g->T;
    g->stats.n = g->n;
    g->stats.m = m;
    g->stats.ms_grid = g->ms_grid;
    long long launches0 = g_launch_count;
    RoundScratch rs(g);
    Timers T(g->st);
    cudaEventCreate(&rs.e0);
    cudaEventCreate(&rs.e1);
    cudaEventRecord(rs.e0, g->st);
    // equal distances ordered by input index, so that the stored lists (and
    // the adjacency of the removal rule) do not depend on the Morton order
    pd_cost_params c2 = *cp;
    c2.term = PD_TERM_INDEX_TIE;
    int rc = prepare_state(g, &c2);
    if (rc) return rc;
    const int k = cp->k, S = g->S;
    const int64_t cap = g->n;
    uint8_t *wdirty, *pick;
    u64* mark_p;
    int* mark_i;
    RALLOC(wdirty, uint8_t, cap);
    RALLOC(pick, uint8_t, cap);
    RALLOC(mark_p, u64, cap);
    RALLOC(mark_i, int, cap);
    SelBuffers sb;
    RALLOC(sb.p[0], u64, cap);
    RALLOC(sb.p[1], u64, cap);
    RALLOC(sb.i[0], int, cap);
    RALLOC(sb.i[1], int, cap);
    RALLOC(sb.hist, uint32_t, 4096);
    CK(cudaMemsetAsync(sb.hist, 0, 4096 * sizeof(uint32_t), g->st));
    RoundDev* rd;
    RALLOC(rd, RoundDev, 1);
    u64* tmin;
    int* imin;
    RALLOC(tmin, u64, 1);
    RALLOC(imin, int, 1);
    int64_t live = g->n, built = g->n;
    int iters = 0;
    while (live > m) {
        if (++iters > 100000) {
            set_err(g->ctx, "pd_decimate_wup: iteration limit reached%s (live = %lld)", "", live);
            return PD_EINTERNAL;
        }
        if (live * 2 < built) {
            Span t(T, &g->stats.ms_build);
            rc = compact_rebuild(g, false);
            if (rc) return rc;
            built = live;
        }
        // 1. every live point's S nearest and cost
        {
            Span t(T, &g->stats.ms_knn);
            KnnArgs a = base_args(g, &c2);
            a.qflag = g->alive;
            CK(launch_knn(view_of(g), a, g->st));
        }
        CK(cudaMemsetAsync(wdirty, 0, g->ng, g->st));
        // 2. w_up: the (live - m)-th largest key is the smallest one above it
        RoundDev h;
        memset(&h, 0, sizeof(h));
        h.live = live;
        h.m = m;
        CK(cudaMemcpyAsync(rd, &h, sizeof(h), cudaMemcpyHostToDevice, g->st));
        CK(wup_launch_setup(rd, g->st));
        {
            Span t(T, &g->stats.ms_select);
            CK(round_launch_select(g->prim, g->pos, g->alive, g->ng, sb, rd, g->st));
            CK(wup_launch_exact_tau(g->prim, g->pos, g->alive, g->ng, rd, tmin, imin, g->st));
        }
        // 3. removal rounds above w_up
        for (int r = 0;; r++) {
            CK(wup_launch_round(bufview(g, &c2), g->alive, wdirty, g->ng, S, k, rd, mark_p,
                                mark_i, pick, g->st));
            unsigned long long removed = 0;
            CK(cudaMemcpyAsync(&removed, &rd->removed, sizeof(removed), cudaMemcpyDeviceToHost,
                               g->st));
            CK(cudaStreamSynchronize(g->st));
            g->stats.rounds++;
            g->stats.live_rounds += live;
            if ((int64_t)removed > live - m || (r == 0 && removed == 0)) {
                set_err(g->ctx, "pd_decimate_wup: a round removed %s%lld points", "",
                        (long long)removed);
                return PD_EINTERNAL;
            }
            live -= (int64_t)removed;
            if (g->trace)
                fprintf(stderr, "pd wup iteration %d round %d removed %llu live %lld\n", iters, r,
                        removed, (long long)live);
            if (removed == 0 || live <= m) break;
        }
    }
    g->stats.iterations = iters;
    CK(cudaMemsetAsync(keep_dev, 0, g->n, g->st));
    CK(launch_keep(g->pos, g->alive, g->ng, keep_dev, g->st));
    cudaEventRecord(rs.e1, g->st);
    CK(cudaEventSynchronize(rs.e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, rs.e0, rs.e1);
    g->stats.ms_total = ms;
    T.resolve();
    g->stats.ms_rules = ms - g->stats.ms_knn - g->stats.ms_build;
    g->stats.launches = g_launch_count - launches0;
    g->ng = 0;  // consumed
    return PD_OK;
}

extern "C" int pd_knn_cost(pd_grid* g, const pd_cost_params* cp, double* cost_dev,
                           int32_t* knn_dev, void* stream) {
    if (!g) return PD_EINVAL;
    g->st = (cudaStream_t)stream;
    int rc = check_cost(g, cp);
    if (rc) return rc;
    if (g->ng != g->n) {
        set_err(g->ctx, "pd_knn_cost: grid already decimated%s", "", 0);
        return PD_EINVAL;
    }
    rc = prepare_state(g, cp);
    if (rc) return rc;
    Temps tmp(g);
    double* cost_s;
    TALLOC(tmp, cost_s, double, g->n);
    rc = knn_all(g, cp, cost_s);
    if (rc) return rc;
    CK(launch_knn_out(g->pos, cost_s, g->nbr, g->ng, g->S, cp->k, cost_dev, knn_dev, g->st));
    tmp.done(cost_s);
    CK(cudaStreamSynchronize(g->st));
    return PD_OK;
}

extern "C" int pd_decimate_count(pd_grid* g, const pd_cost_params* cp, int64_t m,
                                 uint8_t* keep_dev, void* stream) {
    if (!g) return PD_EINVAL;
    g->st = (cudaStream_t)stream;
    int rc = decimate_impl(g, cp, m, keep_dev);
    cudaError_t e = cudaStreamSynchronize(g->st);
    if (!rc && e) {
        set_err(g->ctx, "pd_decimate: CUDA error %s%lld", "", (long long)e);
        rc = PD_ECUDA;
    }
    return rc;
}

extern "C" int pd_decimate_wup(pd_grid* g, const pd_cost_params* cp, int64_t m,
                               uint8_t* keep_dev, void* stream) {
    if (!g) return PD_EINVAL;
    g->st = (cudaStream_t)stream;
    int rc = wup_impl(g, cp, m, keep_dev);
    cudaError_t e = cudaStreamSynchronize(g->st);
    if (!rc && e) {
        set_err(g->ctx, "pd_decimate_wup: CUDA error %s%lld", "", (long long)e);
        rc = PD_ECUDA;
    }
    return rc;
}

extern "C" int pd_decimate_ratio(pd_grid* g, const pd_cost_params* cp, double ratio,
                                 uint8_t* keep_dev, void* stream) {
    if (!g || !(ratio >= 0.0 && ratio <= 1.0)) {
        if (g) set_err(g->ctx, "pd_decimate_ratio: ratio must be in [0, 1]%s", "", 0);
        return PD_EINVAL;
    }
    double v = ratio * (double)g->n;
    int64_t m = (int64_t)v;  // floor for non-negative values
    return pd_decimate_count(g, cp, m, keep_dev, stream);
}

extern "C" int pd_decimate_host(pd_ctx* ctx, const int32_t* xyz_host, const uint8_t* rgb_host,
                                const float* normals_host, int64_t n, const pd_cost_params* cp,
                                int64_t m, uint8_t* keep_host, void* stream, pd_stats* stats) {
    if (!ctx || !xyz_host || !keep_host || !cp || n < 1) return PD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t* xyz = (int32_t*)ctx_alloc(ctx, (size_t)n * 12, st, true);
    uint8_t* rgb = rgb_host ? (uint8_t*)ctx_alloc(ctx, (size_t)n * 3, st, true) : nullptr;
    float* nrm = normals_host && cp->term == PD_TERM_ORIENT
                     ? (float*)ctx_alloc(ctx, (size_t)n * 12, st, true)
                     : nullptr;
    uint8_t* keep = (uint8_t*)ctx_alloc(ctx, (size_t)n, st, true);
    int rc = PD_OK;
    if (!xyz || !keep || (rgb_host && !rgb) || (normals_host && cp->term == PD_TERM_ORIENT && !nrm)) {
        set_err(ctx, "pd_decimate_host: allocation failed%s", "", 0);
        rc = PD_ENOMEM;
    }
    pd_grid* g = nullptr;
    if (!rc && cudaMemcpyAsync(xyz, xyz_host, (size_t)n * 12, cudaMemcpyDefault, st))
        rc = PD_ECUDA;
    if (!rc && rgb && cudaMemcpyAsync(rgb, rgb_host, (size_t)n * 3, cudaMemcpyDefault, st))
        rc = PD_ECUDA;
    if (!rc && nrm && cudaMemcpyAsync(nrm, normals_host, (size_t)n * 12, cudaMemcpyDefault, st))
        rc = PD_ECUDA;
    if (!rc) rc = pd_build_grid(ctx, xyz, rgb, n, nullptr, stream, &g);
    if (!rc) {
        pd_cost_params c2 = *cp;
        if (nrm) c2.normals_dev = nrm;
        rc = pd_decimate_count(g, &c2, m, keep, stream);
        if (!rc && stats) pd_grid_stats(g, stats);
    }
    if (!rc && cudaMemcpyAsync(keep_host, keep, (size_t)n, cudaMemcpyDefault, st))
        rc = PD_ECUDA;
    if (g) pd_grid_free(g);
    ctx_free(ctx, xyz, st);
    ctx_free(ctx, rgb, st);
    ctx_free(ctx, nrm, st);
    ctx_free(ctx, keep, st);
    if (cudaStreamSynchronize(st) && !rc) rc = PD_ECUDA;
    return rc;
}

// ============================================================ API: autotune
extern "C" int pd_autotune(pd_ctx* ctx, const int32_t* xyz_dev, const uint8_t* rgb_dev, int64_t n,
                           const pd_cost_params* cp, double ratio, int64_t sample, void* stream,
                           int32_t* leaf_max_out) {
    if (!ctx || !xyz_dev || !cp || n < 1 || !(ratio >= 0.0 && ratio <= 1.0)) {
        if (ctx) set_err(ctx, "pd_autotune: invalid argument%s", "", 0);
        return PD_EINVAL;
    }
    static const int kLeaf[] = {12, 16, 24, 32};
    const int64_t ns = sample > 0 && sample < n ? sample : n;
    const int64_t m = (int64_t)((double)ns * ratio);
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t* keep = (uint8_t*)ctx_alloc(ctx, (size_t)ns, st);
    if (!keep) {
        set_err(ctx, "pd_autotune: allocation failed%s", "", 0);
        return PD_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = PD_OK, best = 32;
    float best_ms = 0.f;
    // the first (untimed) pass takes the first-call costs out of the comparison
    for (int t = -1; t < 4 && !rc; t++) {
        pd_grid_params gp;
        memset(&gp, 0, sizeof(gp));
        gp.leaf_max = t < 0 ? 32 : kLeaf[t];
        pd_grid* g = nullptr;
        cudaEventRecord(e0, st);
        rc = pd_build_grid(ctx, xyz_dev, rgb_dev, ns, &gp, stream, &g);
        if (!rc) rc = pd_decimate_count(g, cp, m, keep, stream);
        cudaEventRecord(e1, st);
        if (g) pd_grid_free(g);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = PD_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (t >= 0 && (t == 0 || ms < best_ms)) {
            best_ms = ms;
            best = kLeaf[t];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx_free(ctx, keep, st);
    cudaStreamSynchronize(st);
    if (rc) return rc;
    ctx->tuned_leaf = best;
    if (leaf_max_out) *leaf_max_out = best;
    return PD_OK;
}

// Internal diagnostics (not part of pd.h): copy one state array of the grid
// (in Morton order) to host memory.  what: 0 pos int4, 1 code u64, 2 leaf u8,
// 3 alive u8, 4 prim u64, 5 nbr int32 (S per point), 6 flg u8, 7 groups int4,
// 8 scalars int64[8] = {n, ng, ngroups, B, shift, S, hmask+1, T}.
extern "C" int pd__debug_dump(pd_grid* g, int what, void* host, int64_t bytes) {
    if (!g || !host) return PD_EINVAL;
    const void* src = nullptr;
    size_t sz = 0;
    switch (what) {
        case 0: src = g->pos; sz = sizeof(int4) * g->ng; break;
        case 1: src = g->code; sz = sizeof(u64) * g->ng; break;
        case 2: src = g->leaf; sz = g->ng; break;
        case 3: src = g->alive; sz = g->ng; break;
        case 4: src = g->prim; sz = sizeof(u64) * g->ng; break;
        case 5: src = g->nbr; sz = sizeof(int) * g->ng * g->S; break;
        case 6: src = g->flg; sz = g->ng; break;
        case 7: src = g->groups; sz = sizeof(int4) * g->ngroups; break;
        case 8: {
            int64_t v[8] = {g->n, g->ng, g->ngroups, g->B, g->shift, g->S,
                            (int64_t)(g->hmask + 1), g->T};
            memcpy(host, v, std::min<int64_t>(bytes, sizeof(v)));
            return PD_OK;
        }
        default: return PD_EINVAL;
    }
    if (!src) return PD_EINVAL;
    if ((int64_t)sz > bytes) sz = (size_t)bytes;
    cudaStreamSynchronize(g->st);
    return cudaMemcpy(host, src, sz, cudaMemcpyDeviceToHost) ? PD_ECUDA : PD_OK;
}

// Internal diagnostics: run the duplicate phase and the first neighbour pass
// of a decimation and stop (state left in the grid for pd__debug_dump).
extern "C" int pd__debug_first_pass(pd_grid* g, const pd_cost_params* cp, int64_t m) {
    if (!g) return PD_EINVAL;
    int rc = check_cost(g, cp);
    if (rc) return rc;
    rc = prepare_state(g, cp);
    if (rc) return rc;
    int64_t nd = 0;
    rc = remove_duplicates(g, g->n - m, &nd);
    if (rc) return rc;
    if (nd > 0) {
        rc = compact_rebuild(g, false);
        if (rc) return rc;
    }
    rc = knn_all(g, cp, nullptr);
    cudaStreamSynchronize(g->st);
    return rc;
}

// Internal: kernels launched by this library so far in the process.
extern "C" long long pd__launch_count(void) { return g_launch_count; }

// ============================================================ hooks for normals.cu
namespace pd {
void* api_alloc(pd_ctx* c, size_t bytes, cudaStream_t st) { return ctx_alloc(c, bytes, st); }
void api_free(pd_ctx* c, void* p, cudaStream_t st) { ctx_free(c, p, st); }
void api_error(pd_ctx* c, const char* what, long long v) { set_err(c, "%s (%lld)", what, v); }

// The 16 nearest neighbours of every grid point, ascending (d^2, input index),
// stored as Morton positions in the grid's neighbour array (width S = 17).
int grid_knn16(pd_grid* g, cudaStream_t st, GridNbrs* out) {
    g->st = st;
    if (g->ng != g->n) {
        set_err(g->ctx, "pd_normals_pca: grid already decimated%s", "", 0);
        return PD_EINVAL;
    }
    pd_cost_params cp;
    memset(&cp, 0, sizeof(cp));
    cp.k = PD_NORMAL_K;
    int rc = prepare_state(g, &cp);
    if (rc) return rc;
    KnnArgs a = base_args(g, &cp);
    a.term = PD_TERM_INDEX_TIE;
    CK(launch_knn(view_of(g), a, g->st));
    out->pos = g->pos;
    out->nbr = g->nbr;
    out->S = g->S;
    out->n = g->ng;
    out->ctx = g->ctx;
    return PD_OK;
}
}  // namespace pd

// ============================================================ API: quality report
namespace {
struct CtxScratch {
    pd_ctx* c;
    cudaStream_t st;
};
void* cs_alloc(void* self, size_t bytes) {
    CtxScratch* x = (CtxScratch*)self;
    return ctx_alloc(x->c, bytes, x->st);
}
void cs_free(void* self, void* p) {
    CtxScratch* x = (CtxScratch*)self;
    ctx_free(x->c, p, x->st);
}
}  // namespace

static_assert(PD_QUALITY_MAX_RADII == PD_QUALITY_MAXR, "radius limit");

extern "C" int pd_quality_report(pd_ctx* ctx, const int32_t* xyz_dev, const uint8_t* keep_dev,
                                 int64_t n, const int32_t* radii_mm, int nr, pd_quality* out,
                                 void* stream) {
    if (!ctx || !xyz_dev || !radii_mm || !out || n < 1 || n >= (1ll << 31) - 64 || nr < 1 ||
        nr > PD_QUALITY_MAX_RADII) {
        if (ctx) set_err(ctx, "pd_quality_report: invalid argument%s (nr = %lld)", "", nr);
        return PD_EINVAL;
    }
    for (int j = 0; j < nr; j++) {
        if (radii_mm[j] < 1 || radii_mm[j] > (1 << 24) || (j && radii_mm[j] <= radii_mm[j - 1])) {
            set_err(ctx, "pd_quality_report: radii must ascend strictly in [1, 2^24] mm%s (%lld)",
                    "", j);
            return PD_EINVAL;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    memset(out, 0, sizeof(*out));
    out->nr = nr;
    for (int j = 0; j < nr; j++) out->radius_mm[j] = radii_mm[j];
    CtxScratch cs = {ctx, st};
    Scratch sc;
    sc.alloc = cs_alloc;
    sc.free = cs_free;
    sc.self = &cs;
    std::vector<void*> owned;
    auto get = [&](size_t bytes) {
        void* p = ctx_alloc(ctx, bytes, st);
        if (p) owned.push_back(p);
        return p;
    };
    pd_grid* g = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, c0 = nullptr, c1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&c0);
    cudaEventCreate(&c1);
    auto body = [&]() -> int {
#define QCK(x)                                                                     \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) {                                                   \
            set_err(ctx, "pd_quality_report: CUDA error at %s (%lld)", #x, (long long)e_); \
            return e_ == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA;         \
        }                                                                          \
    } while (0)
#define QGET(ptr, type, count)                                                     \
    do {                                                                           \
        ptr = (type*)get(sizeof(type) * (size_t)(count));                          \
        if (!ptr) {                                                                \
            set_err(ctx, "pd_quality_report: allocation of %s failed (%lld)", #ptr, \
                    (long long)(count));                                   \
            return PD_ENOMEM;                                                      \
        }                                                                          \
    } while (0)
        QCK(cudaEventRecord(e0, st));
        // the retained points, in input order
        const int32_t* xyz = xyz_dev;
        int64_t P = n;
        if (keep_dev) {
            int* list;
            int* cnt;
            QGET(list, int, n);
            QGET(cnt, int, 1);
            QCK(stable_compact(keep_dev, n, list, cnt, sc, st));
            int hp = 0;
            QCK(cudaMemcpyAsync(&hp, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
            QCK(cudaStreamSynchronize(st));
            P = hp;
            if (P > 0) {
                int32_t* kx;
                QGET(kx, int32_t, 3 * P);
                QCK(launch_take_xyz(list, cnt, P, xyz_dev, kx, st));
                xyz = kx;
            }
        }
        out->points = P;
        out->min_spacing2_mm2 = -1;
        if (P == 0) return PD_OK;
        pd_grid_params gp;
        memset(&gp, 0, sizeof(gp));
        gp.leaf_max = 32;
        int rc = pd_build_grid(ctx, xyz, nullptr, P, &gp, stream, &g);
        if (rc) return rc;
        // Eq. 2: nearest-neighbour spacing of the retained points (k = 1 search)
        if (P >= 2) {
            pd_cost_params cp;
            memset(&cp, 0, sizeof(cp));
            cp.k = 1;
            rc = prepare_state(g, &cp);
            if (rc) return rc;
            rc = knn_all(g, &cp, nullptr);
            if (rc) return rc;
            const int64_t nb = (P + 255) / 256;
            u64* bmin;
            double* bsum;
            QGET(bmin, u64, nb);
            QGET(bsum, double, nb);
            QCK(launch_spacing(g->rk2, P, bmin, bsum, st));
            std::vector<u64> hmin(nb);
            std::vector<double> hsum(nb);
            QCK(cudaMemcpyAsync(hmin.data(), bmin, nb * sizeof(u64), cudaMemcpyDeviceToHost, st));
            QCK(cudaMemcpyAsync(hsum.data(), bsum, nb * sizeof(double), cudaMemcpyDeviceToHost,
                                st));
            QCK(cudaStreamSynchronize(st));
            u64 mn = ~0ull;
            double sum = 0.0;
            for (int64_t b = 0; b < nb; b++) {
                mn = std::min(mn, hmin[b]);
                sum = sum + hsum[b];
            }
            out->min_spacing2_mm2 = (int64_t)mn;
            out->mean_spacing_mm = sum / (double)P;
        }
        // neighbour counts within each radius: cells whose edge reaches r_max
        int L = 0;
        while (L < g->B && (1ll << (L + g->shift)) < (long long)radii_mm[nr - 1]) L++;
        const int H = PD_QUALITY_HIST;
        u64 *r2, *sn, *sn2;
        uint32_t* hist;
        QGET(r2, u64, nr);
        QGET(sn, u64, nr);
        QGET(sn2, u64, nr);
        QGET(hist, uint32_t, (size_t)nr * H);
        std::vector<u64> hr2(nr);
        for (int j = 0; j < nr; j++) hr2[j] = (u64)radii_mm[j] * (u64)radii_mm[j];
        QCK(cudaMemcpyAsync(r2, hr2.data(), nr * sizeof(u64), cudaMemcpyHostToDevice, st));
        QCK(cudaMemsetAsync(sn, 0, nr * sizeof(u64), st));
        QCK(cudaMemsetAsync(sn2, 0, nr * sizeof(u64), st));
        QCK(cudaMemsetAsync(hist, 0, (size_t)nr * H * sizeof(uint32_t), st));
        QCK(cudaEventRecord(c0, st));
        QCK(launch_radius_counts(view_of(g), P, L, r2, nr, sn, sn2, hist, H, st));
        QCK(cudaEventRecord(c1, st));
        std::vector<u64> T(nr), U(nr);
        std::vector<uint32_t> hh((size_t)nr * H);
        QCK(cudaMemcpyAsync(T.data(), sn, nr * sizeof(u64), cudaMemcpyDeviceToHost, st));
        QCK(cudaMemcpyAsync(U.data(), sn2, nr * sizeof(u64), cudaMemcpyDeviceToHost, st));
        QCK(cudaMemcpyAsync(hh.data(), hist, (size_t)nr * H * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, st));
        QCK(cudaEventRecord(e1, st));
        QCK(cudaStreamSynchronize(st));
        // fractiles: the smallest v with #{N <= v} >= ceil(f P)
        static const int kFrac[PD_QUALITY_NFRAC] = {1, 10, 25, 50, 75, 90, 99};
        for (int j = 0; j < nr; j++) {
            out->mean[j] = (double)T[j] / (double)P;
            const uint32_t* hj = &hh[(size_t)j * H];
            out->count_clipped += hj[H - 1];
            for (int f = 0; f < PD_QUALITY_NFRAC; f++) {
                int64_t rank = (kFrac[f] * P + 99) / 100;
                if (rank < 1) rank = 1;
                int64_t cum = 0;
                int v = 0;
                for (; v < H; v++) {
                    cum += hj[v];
                    if (cum >= rank) break;
                }
                out->fractile[j][f] = v < H ? v : H - 1;
            }
        }
        // least squares of y = N_j(p) on x = pi r_j^2 (m^2) over the P * nr samples
        std::vector<double> x(nr);
        double xs = 0.0;
        for (int j = 0; j < nr; j++) {
            double r = (double)radii_mm[j] / 1000.0;
            x[j] = 3.141592653589793 * r * r;
            xs = xs + x[j];
        }
        const double xbar = xs / (double)nr;
        double varx = 0.0, cov = 0.0;
        unsigned __int128 sy = 0, suu = 0;
        for (int j = 0; j < nr; j++) {
            double dx = x[j] - xbar;
            varx = varx + dx * dx;
            cov = cov + dx * (double)T[j];
            sy += T[j];
            suu += U[j];
        }
        varx = varx * (double)P;   // sum over all samples of (x - xbar)^2
        const unsigned __int128 N = (unsigned __int128)P * (unsigned __int128)nr;
        // N * sum (y - ybar)^2 = N * sum y^2 - (sum y)^2, exact in 128 bits
        const unsigned __int128 nss = N * suu - sy * sy;
        const double sstot = (double)nss / (double)N;
        if (nr >= 2 && varx > 0.0) {
            out->slope_per_m2 = cov / varx;
            out->intercept = (double)sy / (double)N - out->slope_per_m2 * xbar;
            double ssres = sstot - cov * cov / varx;
            if (ssres < 0.0) ssres = 0.0;
            out->r2 = sstot > 0.0 ? cov * cov / (varx * sstot) : 1.0;
            out->rmse = sqrt(ssres / (double)N);
        } else {
            out->slope_per_m2 = out->intercept = out->r2 = out->rmse = NAN;
        }
        float ms = 0.f, mc = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventElapsedTime(&mc, c0, c1);
        out->ms = ms;
        out->ms_counts = mc;
        return PD_OK;
#undef QCK
#undef QGET
    };
    int rc = body();
    if (g) pd_grid_free(g);
    for (void* p : owned) ctx_free(ctx, p, st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(c0);
    cudaEventDestroy(c1);
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = PD_ECUDA;
    return rc;
}

// ============================================================ API: batch
namespace {

// Every scan of a batch in one grid (the packed mode of pd_decimate_batch):
// scan i moves into the aligned tile of edge 2^T mm whose Morton index is i,
// the tiles are decimated together, and the keep masks are copied back.
// Returns PD_SEG_FALLBACK when the batch cannot be packed (then nothing was
// written): too many scans or points, a target of k points or fewer (a scan
// must keep more than k, so that every search stays inside it), a missing
// colour or normal array, a tile arrangement beyond the coordinate range, or
// a scan with more coincident points than it must lose.
int batch_packed(pd_ctx* ctx, pd_scan_desc* scans, int nscans, const pd_cost_params* cp,
                 cudaStream_t st) {
    if (nscans > PD_SEG_MAX || !cp || cp->k < 1 || cp->k > PD_KMAX) return PD_SEG_FALLBACK;
    const bool want_rgb = cp->term == PD_TERM_COLOR, want_nrm = cp->term == PD_TERM_ORIENT;
    std::vector<PackScan> hs(nscans);
    std::vector<long long> nv(nscans), mv(nscans);
    long long N = 0, M = 0;
    int nchunks = 0;
    for (int i = 0; i < nscans; i++) {
        const pd_scan_desc& d = scans[i];
        const long long m = d.m >= 0 ? d.m : (long long)(d.ratio * (double)d.n);
        if (m <= cp->k || (want_rgb && !d.rgb_dev) || (want_nrm && !d.normals_dev))
            return PD_SEG_FALLBACK;
        PackScan& p = hs[i];
        memset(&p, 0, sizeof(p));
        p.xyz = d.xyz_dev;
        p.rgb = want_rgb ? d.rgb_dev : nullptr;
        p.nrm = want_nrm ? d.normals_dev : nullptr;
        p.keep = d.keep_dev;
        p.n = d.n;
        p.off = N;
        p.chunk0 = nchunks;
        for (int a = 0; a < 3; a++) {
            p.bb[a] = 0x7fffffff;
            p.bb[3 + a] = (int)0x80000000;
        }
        nv[i] = d.n;
        mv[i] = m;
        N += d.n;
        M += m;
        nchunks += (int)((d.n + PD_SEG_CHUNK - 1) / PD_SEG_CHUNK);
        if (N >= (1ll << 31) - 64) return PD_SEG_FALLBACK;
    }
    struct Blocks {  // released in order on every exit path
        pd_ctx* c;
        cudaStream_t st;
        std::vector<void*> p;
        void* get(size_t b) {
            void* x = ctx_alloc(c, b, st);
            if (x) p.push_back(x);
            return x;
        }
        ~Blocks() {
            for (void* x : p) ctx_free(c, x, st);
        }
    } blk{ctx, st, {}};
    PackScan* ds = (PackScan*)blk.get(sizeof(PackScan) * nscans);
    if (!ds) return PD_ENOMEM;
    if (cudaMemcpyAsync(ds, hs.data(), sizeof(PackScan) * nscans, cudaMemcpyHostToDevice, st) ||
        pack_launch_bbox(ds, nscans, nchunks, st) ||
        cudaMemcpyAsync(hs.data(), ds, sizeof(PackScan) * nscans, cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st)) {
        set_err(ctx, "pd_decimate_batch: packing failed%s", "", 0);
        return PD_ECUDA;
    }
    // tile edge 2^T >= 3 E + 2, E the largest per-axis extent of any scan: two
    // points of different tiles are at least 2^T - E > sqrt(3) E apart, more
    // than any two points of one scan, so a scan that keeps more than k points
    // never finds a neighbour elsewhere
    long long E = 0;
    for (const PackScan& p : hs)
        for (int a = 0; a < 3; a++) E = std::max(E, (long long)p.bb[3 + a] - p.bb[a]);
    int T = 10;
    while ((1ll << T) < 3 * E + 2) T++;
    int td = 1;  // tiles per axis
    while ((long long)td * td * td < nscans) td *= 2;
    if ((long long)(td - 1) * (1ll << T) + E >= (1ll << 25)) return PD_SEG_FALLBACK;
    for (int i = 0; i < nscans; i++) {
        PackScan& p = hs[i];
        const long long tile[3] = {(long long)compact3((u64)i), (long long)compact3((u64)i >> 1),
                                   (long long)compact3((u64)i >> 2)};
        int* o[3] = {&p.ox, &p.oy, &p.oz};
        for (int a = 0; a < 3; a++) {
            const long long v = (tile[a] << T) - (long long)p.bb[a];
            if (v > 0x7fffffffll || v < -0x7fffffffll) return PD_SEG_FALLBACK;
            *o[a] = (int)v;
        }
    }
    int32_t* xyz = (int32_t*)blk.get((size_t)N * 12);
    uint8_t* rgb = want_rgb ? (uint8_t*)blk.get((size_t)N * 3) : nullptr;
    float* nrm = want_nrm ? (float*)blk.get((size_t)N * 12) : nullptr;
    uint8_t* keep = (uint8_t*)blk.get((size_t)N);
    if (!xyz || !keep || (want_rgb && !rgb) || (want_nrm && !nrm)) {
        set_err(ctx, "pd_decimate_batch: allocation of the packed batch failed%s (%lld points)",
                "", N);
        return PD_ENOMEM;
    }
    if (cudaMemcpyAsync(ds, hs.data(), sizeof(PackScan) * nscans, cudaMemcpyHostToDevice, st) ||
        pack_launch_copy(ds, nscans, nchunks, xyz, rgb, nrm, st)) {
        set_err(ctx, "pd_decimate_batch: packing failed%s", "", 0);
        return PD_ECUDA;
    }
    pd_grid* g = nullptr;
    int rc = pd_build_grid(ctx, xyz, rgb, N, nullptr, st, &g);
    if (rc) return rc;
    struct GridGuard {
        pd_grid* g;
        ~GridGuard() {
            if (g) pd_grid_free(g);
        }
    } gg{g};
    g->nseg = nscans;
    g->seg_shift = T;
    g->seg_n = nv;
    g->seg_m = mv;
    g->seg = (SegDev*)ctx_alloc(ctx, sizeof(SegDev) * nscans, st);
    g->seg_chunk0 = (int*)ctx_alloc(ctx, sizeof(int) * (nscans + 1), st);
    g->seg_items = (int*)ctx_alloc(ctx, sizeof(int) * (N / PD_SEG_CHUNK + nscans + 1), st);
    if (!g->seg || !g->seg_chunk0 || !g->seg_items) {
        set_err(ctx, "pd_decimate_batch: allocation of the scan table failed%s", "", 0);
        return PD_ENOMEM;
    }
    std::vector<SegDev> sd(nscans);
    memset(sd.data(), 0, sizeof(SegDev) * nscans);
    for (int i = 0; i < nscans; i++) {
        sd[i].m = mv[i];
        sd[i].done = 1;
    }
    if (cudaMemcpyAsync(g->seg, sd.data(), sizeof(SegDev) * nscans, cudaMemcpyHostToDevice, st))
        return PD_ECUDA;
    pd_cost_params c2 = *cp;
    c2.normals_dev = nrm;
    rc = pd_decimate_count(g, &c2, M, keep, st);
    if (rc) return rc;
    if (pack_launch_unpack(ds, nscans, nchunks, keep, st)) return PD_ECUDA;
    pd_stats gs;
    pd_grid_stats(g, &gs);
    for (int i = 0; i < nscans; i++) {
        scans[i].stats = gs;  // the whole batch's decimation
        scans[i].stats.n = nv[i];
        scans[i].stats.m = mv[i];
        scans[i].status = PD_OK;
    }
    if (cudaStreamSynchronize(st)) return PD_ECUDA;
    return PD_OK;
}

}  // namespace

// Many independent scans.  Packed mode (concurrency PD_BATCH_PACKED): all
// scans in one grid, decimated together (batch_packed).  Otherwise, or when
// a batch cannot be packed, a fixed number of concurrent slots: every
// slot owns a CUDA stream and a host thread that builds the scan's grid and
// runs its removal rounds; the slots' kernels overlap on the device.  The
// call orders all work after what is already queued on `stream` and makes
// `stream` wait for all of it before returning.
extern "C" int pd_decimate_batch(pd_ctx* ctx, pd_scan_desc* scans, int nscans,
                                 const pd_cost_params* cp, int concurrency, void* stream) {
    if (!ctx || !scans || nscans < 0 || !cp) return PD_EINVAL;
    if (nscans == 0) return PD_OK;
    for (int i = 0; i < nscans; i++) {
        const pd_scan_desc& d = scans[i];
        if (!d.xyz_dev || !d.keep_dev || d.n < 1 ||
            (d.m < 0 && !(d.ratio >= 0.0 && d.ratio <= 1.0)) || d.m > d.n) {
            set_err(ctx, "pd_decimate_batch: invalid scan descriptor %s%lld", "", i);
            return PD_EINVAL;
        }
    }
    cudaStream_t caller = (cudaStream_t)stream;
    if (concurrency == PD_BATCH_PACKED) {
        int rc = batch_packed(ctx, scans, nscans, cp, caller);
        if (rc != PD_SEG_FALLBACK) return rc;
        concurrency = 0;  // not packable: slots
    }
    int slots = concurrency > 0 ? concurrency : 8;
    if (slots > nscans) slots = nscans;
    int dev = 0;
    if (cudaGetDevice(&dev)) return PD_ECUDA;
    cudaEvent_t start;
    if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming)) return PD_ECUDA;
    cudaEventRecord(start, caller);
    std::vector<cudaStream_t> st(slots);
    std::vector<cudaEvent_t> fin(slots);
    for (int s = 0; s < slots; s++) {
        cudaStreamCreateWithFlags(&st[s], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&fin[s], cudaEventDisableTiming);
        cudaStreamWaitEvent(st[s], start, 0);
    }
    std::atomic<int> next(0);
    std::atomic<int> first_err(PD_OK);
    auto worker = [&](int slot) {
        cudaSetDevice(dev);
        for (;;) {
            int i = next.fetch_add(1);
            if (i >= nscans) break;
            pd_scan_desc& d = scans[i];
            pd_grid* g = nullptr;
            int rc = pd_build_grid(ctx, d.xyz_dev, d.rgb_dev, d.n, nullptr, st[slot], &g);
            if (!rc) {
                pd_cost_params c2 = *cp;
                if (d.normals_dev) c2.normals_dev = d.normals_dev;
                int64_t m = d.m >= 0 ? d.m : (int64_t)(d.ratio * (double)d.n);
                rc = pd_decimate_count(g, &c2, m, d.keep_dev, st[slot]);
                if (!rc) pd_grid_stats(g, &d.stats);
            }
            if (g) pd_grid_free(g);
            d.status = rc;
            if (rc) {
                int expect = PD_OK;
                first_err.compare_exchange_strong(expect, rc);
            }
        }
        cudaEventRecord(fin[slot], st[slot]);
    };
    std::vector<std::thread> th;
    for (int s = 0; s < slots; s++) th.emplace_back(worker, s);
    for (auto& t : th) t.join();
    for (int s = 0; s < slots; s++) {
        cudaStreamWaitEvent(caller, fin[s], 0);
        cudaEventDestroy(fin[s]);
        cudaStreamDestroy(st[s]);
    }
    cudaEventDestroy(start);
    return first_err.load();
}
