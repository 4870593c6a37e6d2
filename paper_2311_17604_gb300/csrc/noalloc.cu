// noalloc.cu -- pd_knn_cost_static: the neighbour/cost pass of pd_knn_cost for
// small clouds, using a fixed device array instead of any device allocation.
//
// Some callers cannot allocate device memory when they call us: a real-time
// ingest loop that fixes its memory budget at start-up, a host process whose
// memory-pool policy forbids new device allocations after initialisation, or a
// plug-in that must not touch the host application's allocator.  This entry
// point runs the same kernels as pd_build_grid + pd_knn_cost, but every
// temporary lives in g_static_scratch below, a file-scope __device__ array of
// PD_STATIC_SCRATCH_BYTES bytes that each GPU loading the library holds until
// the process exits.  It calls no cudaMalloc, cudaFree, cudaMallocAsync or any
// allocating library routine.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/pd.h"
#include "pd_internal.cuh"
#include "pd_kernels.h"

using namespace pd;

namespace pd {
cudaError_t launch_knn_out(const int4*, const double*, const int*, int64_t, int, int, double*,
                           int32_t*, cudaStream_t);
}

// hash-table slots per point of the fixed cell table (power-of-two capacity
// at least twice the number of octree cells)
#define PD_STATIC_HASH_SLOTS_PER_POINT 4

namespace {

// The scratch array.  Its name is only a host-side handle: host code must use
// the address that cudaGetSymbolAddress returns for the current device.
__device__ __align__(256) unsigned char g_static_scratch[PD_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_dev_addr[128];
bool g_have[128];

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_have[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e) return e;
        g_dev_addr[dev] = p;
        g_have[dev] = true;
    }
    *out = g_dev_addr[dev];
    return cudaSuccess;
}

// Bump allocator over the scratch array; everything is released at once when
// the call returns (put() is a no-op).
struct Arena {
    char* base;
    size_t cap, used;
    void* get(size_t bytes) {
        size_t b = (bytes + 255) & ~(size_t)255;
        if (used + b > cap) return nullptr;
        void* p = base + used;
        used += b;
        return p;
    }
};
void* arena_get(void* self, size_t bytes) { return ((Arena*)self)->get(bytes); }
void arena_put(void*, void*) {}

}  // namespace

#define SCK(x)                                       \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ == cudaErrorMemoryAllocation)         \
            return PD_ENOMEM;                        \
        if (e_ != cudaSuccess) return PD_ECUDA;      \
    } while (0)
#define SGET(ptr, type, count)                                        \
    do {                                                              \
        ptr = (type*)ar.get(sizeof(type) * (size_t)(count));          \
        if (!ptr) return PD_ENOMEM;                                   \
    } while (0)

extern "C" int pd_knn_cost_static(const int32_t* xyz_dev, int64_t n, int k, double* cost_dev,
                                  int32_t* knn_dev, void* stream) {
    if (!xyz_dev || n < 1 || k < 1 || k > PD_KMAX) return PD_EINVAL;
    if (n > PD_STATIC_MAX_POINTS) return PD_ERANGE;
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    SCK(scratch_address(&base));
    Arena ar = {(char*)base, (size_t)PD_STATIC_SCRATCH_BYTES, 0};
    Scratch s;
    s.alloc = arena_get;
    s.free = arena_put;
    s.self = &ar;

    // extent (one host read, as in pd_build_grid)
    int* d6;
    SGET(d6, int, 8);
    SCK(launch_bbox(xyz_dev, n, d6, st));
    int h6[6];
    SCK(cudaMemcpyAsync(h6, d6, sizeof(h6), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    long long span = 0;
    for (int a = 0; a < 3; a++) {
        long long w = (long long)h6[3 + a] - h6[a];
        if (w > span) span = w;
    }
    if (span >= (1ll << 25)) return PD_ERANGE;
    GridView g;
    memset(&g, 0, sizeof(g));
    g.origin = make_int3(h6[0], h6[1], h6[2]);
    g.umax = make_int3(h6[3] - h6[0], h6[4] - h6[1], h6[5] - h6[2]);
    int bits = 1;
    while ((1ll << bits) <= span) bits++;
    g.shift = bits > PD_MAXLEVEL ? bits - PD_MAXLEVEL : 0;
    g.B = bits - g.shift;
    if (g.B < 1) g.B = 1;
    g.T = 32;

    // Morton order
    u64* code;
    uint32_t* perm;
    SGET(code, u64, n);
    SGET(perm, uint32_t, n);
    SCK(launch_morton(xyz_dev, n, g.origin, g.shift, code, perm, st));
    SCK(radix_sort_pairs(code, perm, n, 3 * g.B, s, st));
    int4* pos;
    SGET(pos, int4, n);
    SCK(launch_gather(xyz_dev, nullptr, nullptr, perm, n, pos, nullptr, nullptr, st));
    uint8_t* leaf;
    SGET(leaf, uint8_t, n);
    SCK(launch_leaf_levels(code, n, g.T, g.B, leaf, st));

    // cell table: fixed capacity of PD_STATIC_HASH_SLOTS_PER_POINT slots per point
    unsigned long long* dcount;
    SGET(dcount, unsigned long long, 1);
    SCK(launch_node_count(code, leaf, n, g.B, dcount, st));
    unsigned long long nodes = 0;
    SCK(cudaMemcpyAsync(&nodes, dcount, sizeof(nodes), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    u64 cap = 1024;
    while (cap < 2 * nodes) cap <<= 1;
    if (cap > (u64)PD_STATIC_HASH_SLOTS_PER_POINT * (u64)PD_STATIC_MAX_POINTS) return PD_ENOMEM;
    HashSlot* hash;
    SGET(hash, HashSlot, cap);
    SCK(launch_node_insert(code, leaf, n, g.B, hash, cap - 1, st));
    g.pos = pos;
    g.code = code;
    g.leaf = leaf;
    g.hash = hash;
    g.hmask = cap - 1;
    int4* groups;
    int* dng;
    SGET(groups, int4, n);
    SGET(dng, int, 1);
    SCK(launch_leaf_groups(g, n, groups, dng, st));
    int ngroups = 0;
    SCK(cudaMemcpyAsync(&ngroups, dng, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));

    // one full neighbour / cost pass, as pd_knn_cost runs it
    int dk1 = k == 1;
    int S = dk1 ? 8 : (k <= 6 ? 8 : 17);
    u64 *prim, *rk2, *hz;
    int* nbr;
    uint8_t* flg;
    double* cost_s;
    SGET(prim, u64, n);
    SGET(rk2, u64, n);
    SGET(hz, u64, n);
    SGET(nbr, int, (size_t)n * S);
    SGET(flg, uint8_t, n);
    SGET(cost_s, double, n);
    KnnArgs a;
    memset(&a, 0, sizeof(a));
    a.groups = groups;
    a.ngroups = ngroups;
    a.k = k;
    a.S = S;
    a.density_k1 = dk1;
    a.nbr = nbr;
    a.prim_out = prim;
    a.rk2_out = rk2;
    a.flg_out = flg;
    a.hz_out = hz;
    a.cost_out = cost_s;
    SCK(launch_knn(g, a, st));
    SCK(launch_knn_out(pos, cost_s, nbr, n, S, k, cost_dev, knn_dev, st));
    SCK(cudaStreamSynchronize(st));
    return PD_OK;
}
