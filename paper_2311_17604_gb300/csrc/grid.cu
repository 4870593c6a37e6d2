// grid.cu -- voxel-grid build: extent, Morton codes, stable LSD radix sort,
// gather into Morton order, adaptive octree leaf levels and the hashed table
// of octree cells (the paper's voxelisation, section "Sub-sampling algorithm",
// rebuilt as one sort that serves every power-of-two cell size).
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_internal.cuh"
#include "pd_kernels.h"

namespace pd {

// ------------------------------------------------------------------ extent
__global__ void bbox_kernel(const int32_t* __restrict__ xyz, int64_t n, int* out6) {
    int mn[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, mx[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; a++) {
            int v = xyz[3 * i + a];
            mn[a] = min(mn[a], v);
            mx[a] = max(mx[a], v);
        }
    }
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o; o >>= 1) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; a++) {
            atomicMin(&out6[a], mn[a]);
            atomicMax(&out6[3 + a], mx[a]);
        }
    }
}

cudaError_t launch_bbox(const int32_t* xyz, int64_t n, int* out6, cudaStream_t st) {
    int init[6] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, INT32_MIN};
    cudaError_t e = cudaMemcpyAsync(out6, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e) return e;
    int blocks = (int)((n + 255) / 256);
    if (blocks > device_sms() * 8) blocks = device_sms() * 8;
    if (blocks < 1) blocks = 1;
    bbox_kernel<<<blocks, 256, 0, st>>>(xyz, n, out6); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Morton
__global__ void morton_kernel(const int32_t* __restrict__ xyz, int64_t n, int3 o, int shift,
                              u64* __restrict__ keys, uint32_t* __restrict__ vals) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t ux = (uint32_t)(xyz[3 * i] - o.x) >> shift;
    uint32_t uy = (uint32_t)(xyz[3 * i + 1] - o.y) >> shift;
    uint32_t uz = (uint32_t)(xyz[3 * i + 2] - o.z) >> shift;
    keys[i] = morton3(ux, uy, uz);
    vals[i] = (uint32_t)i;
}

cudaError_t launch_morton(const int32_t* xyz, int64_t n, int3 origin, int shift, u64* keys,
                          uint32_t* vals, cudaStream_t st) {
    morton_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xyz, n, origin, shift, keys, vals); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of uint32 (block = 256 threads x 4 items = 1024).
__global__ void scan_block_kernel(uint32_t* data, int64_t len, uint32_t* sums) {
    __shared__ uint32_t wsum[8];
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int64_t base = (int64_t)blockIdx.x * 1024 + t * 4;
    uint32_t v[4];
    uint32_t acc = 0;
    for (int j = 0; j < 4; j++) {
        v[j] = base + j < len ? data[base + j] : 0;
        acc += v[j];
    }
    uint32_t inc = acc;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < 8 ? wsum[lane] : 0;
        for (int o = 1; o < 8; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < 8) wsum[lane] = s;
    }
    __syncthreads();
    uint32_t off = (w ? wsum[w - 1] : 0) + inc - acc;
    for (int j = 0; j < 4; j++) {
        if (base + j < len) data[base + j] = off;
        off += v[j];
    }
    if (t == 255 && sums) sums[blockIdx.x] = wsum[7];
}

__global__ void scan_add_kernel(uint32_t* data, int64_t len, const uint32_t* sums) {
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    uint32_t add = sums[blockIdx.x];
    for (int j = 0; j < 4; j++, i += 256)
        if (i < len) data[i] += add;
}

cudaError_t exclusive_scan_u32(uint32_t* data, int64_t len, const Scratch& s, cudaStream_t st) {
    if (len <= 0) return cudaSuccess;
    int64_t nb = (len + 1023) / 1024;
    if (nb == 1) {
        scan_block_kernel<<<1, 256, 0, st>>>(data, len, nullptr); note_launch();
        return cudaGetLastError();
    }
    uint32_t* sums = (uint32_t*)s.get(nb * sizeof(uint32_t));
    if (!sums) return cudaErrorMemoryAllocation;
    scan_block_kernel<<<(unsigned)nb, 256, 0, st>>>(data, len, sums); note_launch();
    cudaError_t e = exclusive_scan_u32(sums, nb, s, st);
    if (!e) scan_add_kernel<<<(unsigned)nb, 256, 0, st>>>(data, len, sums); note_launch();
    s.put(sums);
    return e ? e : cudaGetLastError();
}

// ------------------------------------------------------------------ radix sort
// Tiles of 2048 keys: 256 threads x 8 sub-tiles of 256 consecutive keys.
#define RS_TILE 2048

__global__ void radix_hist_kernel(const u64* __restrict__ keys, int64_t n, int shift,
                                  uint32_t* counts, int nblk) {
    __shared__ uint32_t h[256];
    int t = threadIdx.x;
    h[t] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < 8; j++) {
        int64_t i = base + j * 256 + t;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    counts[(int64_t)t * nblk + blockIdx.x] = h[t];
}

// Scatter of one 8-bit digit.  The tile's keys are first placed in digit
// order in shared memory (stable: sub-tile by sub-tile, warp by warp, lane by
// lane), then written out in that order, so that consecutive threads write
// consecutive addresses of one digit's run.  offs is the exclusive scan of the
// digit-major [digit][tile] counts: the tile's own count of digit d is the gap
// to the next entry (n at the very end).
__global__ void radix_scatter_kernel(const u64* __restrict__ kin, const uint32_t* __restrict__ vin,
                                     u64* __restrict__ kout, uint32_t* __restrict__ vout,
                                     int64_t n, int shift, const uint32_t* __restrict__ offs,
                                     int nblk) {
    __shared__ u64 sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    __shared__ uint32_t goff[256];
    __shared__ uint32_t tpre[256];  // first slot of digit d in the tile's sorted order
    __shared__ uint32_t run[256];
    __shared__ uint32_t wsum[8];
    __shared__ uint16_t wcnt[8][257];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int64_t gi = (int64_t)t * nblk + blockIdx.x;
    const uint32_t go = offs[gi];
    const uint32_t next = gi + 1 < (int64_t)256 * nblk ? offs[gi + 1] : (uint32_t)n;
    goff[t] = go;
    run[t] = 0;
    // exclusive scan of the tile's per-digit counts over the 256 digits
    {
        const uint32_t c = next - go;
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int ww = 0; ww < w; ww++) before += wsum[ww];
        tpre[t] = before + x - c;
    }
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_TILE / 256; j++) {
        for (int x = t; x < 8 * 257; x += 256) (&wcnt[0][0])[x] = 0;
        __syncthreads();
        const int64_t i = base + j * 256 + t;
        const bool valid = i < n;
        const u64 k = valid ? kin[i] : 0ull;
        const uint32_t v = valid ? vin[i] : 0u;
        const int d = valid ? (int)((k >> shift) & 255) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int lrank = __popc(peers & ((1u << lane) - 1u));
        if (lane == __ffs(peers) - 1) wcnt[w][d] = (uint16_t)__popc(peers);
        __syncthreads();
        {
            uint32_t acc = run[t];
            for (int ww = 0; ww < 8; ww++) {
                uint32_t c = wcnt[ww][t];
                wcnt[ww][t] = (uint16_t)acc;
                acc += c;
            }
            run[t] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t lp = tpre[d] + wcnt[w][d] + (uint32_t)lrank;
            sk[lp] = k;
            sv[lp] = v;
        }
        __syncthreads();  // wcnt is cleared at the top of the next sub-tile
    }
    const int tn = (int)min((int64_t)RS_TILE, n - base);
    for (int x = t; x < tn; x += 256) {
        const u64 k = sk[x];
        const int d = (int)((k >> shift) & 255);
        const uint32_t p = goff[d] + ((uint32_t)x - tpre[d]);
        kout[p] = k;
        vout[p] = sv[x];
    }
}

cudaError_t radix_sort_pairs(u64* keys, uint32_t* vals, int64_t n, int bits, const Scratch& s,
                             cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    u64* k2 = (u64*)s.get(n * sizeof(u64));
    uint32_t* v2 = (uint32_t*)s.get(n * sizeof(uint32_t));
    uint32_t* counts = (uint32_t*)s.get((size_t)256 * nblk * sizeof(uint32_t));
    cudaError_t e = cudaSuccess;
    if (!k2 || !v2 || !counts) e = cudaErrorMemoryAllocation;
    u64 *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes && !e; p++) {
        radix_hist_kernel<<<nblk, 256, 0, st>>>(ka, n, 8 * p, counts, nblk); note_launch();
        e = cudaGetLastError();
        if (!e) e = exclusive_scan_u32(counts, (int64_t)256 * nblk, s, st);
        if (!e) {
            radix_scatter_kernel<<<nblk, 256, 0, st>>>(ka, va, kb, vb, n, 8 * p, counts, nblk); note_launch();
            e = cudaGetLastError();
        }
        u64* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    if (!e && ka != keys) {
        e = cudaMemcpyAsync(keys, ka, n * sizeof(u64), cudaMemcpyDefault, st);
        if (!e) e = cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDefault, st);
    }
    s.put(counts);
    s.put(v2);
    s.put(k2);
    return e;
}

// ------------------------------------------------------------------ gather
__global__ void gather_kernel(const int32_t* __restrict__ xyz, const uint8_t* __restrict__ rgb,
                              const float* __restrict__ nrm, const uint32_t* __restrict__ perm,
                              int64_t n, int4* __restrict__ pos, uchar4* __restrict__ rgb_s,
                              float4* __restrict__ nrm_s) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t i = perm[s];
    pos[s] = make_int4(xyz[3 * (int64_t)i], xyz[3 * (int64_t)i + 1], xyz[3 * (int64_t)i + 2],
                       (int)i);
    if (rgb_s) {
        rgb_s[s] = make_uchar4(rgb[3 * (int64_t)i], rgb[3 * (int64_t)i + 1],
                               rgb[3 * (int64_t)i + 2], 0);
    }
    if (nrm_s) {
        nrm_s[s] = make_float4(nrm[3 * (int64_t)i], nrm[3 * (int64_t)i + 1],
                               nrm[3 * (int64_t)i + 2], 0.f);
    }
}

cudaError_t launch_gather(const int32_t* xyz, const uint8_t* rgb, const float* nrm,
                          const uint32_t* perm, int64_t n, int4* pos, uchar4* rgb_s,
                          float4* nrm_s, cudaStream_t st) {
    gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        xyz, rgb_s ? rgb : nullptr, nrm_s ? nrm : nullptr, perm, n, pos, rgb_s, nrm_s); note_launch();
    return cudaGetLastError();
}

__global__ void gather_nrm_kernel(const float* __restrict__ nrm, const int4* __restrict__ pos,
                                  int64_t n, float4* __restrict__ out) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t i = pos[s].w;
    out[s] = make_float4(nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2], 0.f);
}

cudaError_t launch_gather_nrm(const float* nrm, const int4* pos, int64_t n, float4* out,
                              cudaStream_t st) {
    gather_nrm_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nrm, pos, n, out); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ leaf levels
// A level-L cell holding s has more than T points iff some window of T+1
// consecutive Morton positions around s shares the level-L prefix.  With
// Ls(j) = smallest level at which code[j] and code[j+T] share a cell, the
// leaf level of s is min over j in [s-T, s] of Ls(j), minus one.
__global__ void leaf_level_kernel(const u64* __restrict__ code, int64_t n, int T, int B,
                                  uint8_t* __restrict__ leaf) {
    extern __shared__ uint8_t ls[];
    int64_t b0 = (int64_t)blockIdx.x * 256;
    for (int x = threadIdx.x; x < 256 + T; x += 256) {
        int64_t j = b0 - T + x;
        uint8_t v = 255;
        if (j >= 0 && j + T < n) {
            u64 d = code[j] ^ code[j + T];
            v = d == 0 ? 0 : (uint8_t)((63 - __clzll((long long)d)) / 3 + 1);
        }
        ls[x] = v;
    }
    __syncthreads();
    int64_t i = b0 + threadIdx.x;
    if (i >= n) return;
    int mn = 255;
    for (int x = 0; x <= T; x++) mn = min(mn, (int)ls[threadIdx.x + x]);
    int L = mn == 255 ? B : (mn > 0 ? mn - 1 : 0);
    if (L > B) L = B;
    leaf[i] = (uint8_t)L;
}

cudaError_t launch_leaf_levels(const u64* code, int64_t n, int T, int B, uint8_t* leaf,
                               cudaStream_t st) {
    leaf_level_kernel<<<(unsigned)((n + 255) / 256), 256, 256 + T, st>>>(code, n, T, B, leaf); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ cell table
// Highest level at which the level prefixes (code >> 3L) of a and b differ;
// -1 for equal codes.  Position i opens a level-L cell (a run head) iff
// i == 0 or L <= diff_level(code[i-1], code[i]); it closes one (a run tail)
// iff i == n-1 or L <= diff_level(code[i], code[i+1]).
__device__ inline int diff_level(u64 a, u64 b) {
    u64 d = a ^ b;
    return d ? (63 - __clzll((long long)d)) / 3 : -1;
}
__device__ inline int head_level(const u64* code, int64_t i, int B) {
    return i == 0 ? B : diff_level(code[i - 1], code[i]);
}
__device__ inline int tail_level(const u64* code, int64_t i, int64_t n, int B) {
    return i == n - 1 ? B : diff_level(code[i], code[i + 1]);
}

// Octree nodes: one per (level L >= the point's leaf level, run head).
__global__ void node_count_kernel(const u64* __restrict__ code, const uint8_t* __restrict__ leaf,
                                  int64_t n, int B, unsigned long long* count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned c = 0;
    if (i < n) {
        int hi = min(head_level(code, i, B), B);
        int lo = leaf[i];
        c = hi >= lo ? (unsigned)(hi - lo + 1) : 0u;
    }
    block_add(count, c);
}

cudaError_t launch_node_count(const u64* code, const uint8_t* leaf, int64_t n, int B,
                              unsigned long long* count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e) return e;
    node_count_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(code, leaf, n, B, count); note_launch();
    return cudaGetLastError();
}

__device__ inline long long hash_insert(HashSlot* tab, u64 mask, u64 key) {
    u64 h = mix64(key) & mask;
    for (u64 it = 0; it <= mask; it++) {
        u64 prev = atomicCAS(&tab[h].key, PD_EMPTY_KEY, key);
        if (prev == PD_EMPTY_KEY || prev == key) return (long long)h;
        h = (h + 1) & mask;
    }
    return -1;
}

__global__ void node_insert_kernel(const u64* __restrict__ code, const uint8_t* __restrict__ leaf,
                                   int64_t n, int B, HashSlot* tab, u64 mask) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int hh = head_level(code, i, B), ht = tail_level(code, i, n, B);
    const int top = min(max(hh, ht), B);  // above it i neither opens nor closes a cell
    const u64 c = code[i];
    for (int L = leaf[i]; L <= top; L++) {
        bool h = L <= hh, t = L <= ht;
        u64 prefix = c >> (3 * L);
        long long slot = hash_insert(tab, mask, cell_key(prefix, L, B));
        if (slot < 0) continue;  // table sized at 2x the node count: cannot fill
        if (h) tab[slot].b = (uint32_t)i;
        if (t) tab[slot].e = (uint32_t)(i + 1);
    }
}

cudaError_t launch_node_insert(const u64* code, const uint8_t* leaf, int64_t n, int B,
                               HashSlot* tab, u64 mask, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(tab, 0, (mask + 1) * sizeof(HashSlot), st);
    if (e) return e;
    node_insert_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(code, leaf, n, B, tab, mask); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ groups
// Range [b, e) of the leaf that holds Morton position s.
__device__ inline bool leaf_range(const GridView& g, int64_t s, uint32_t& b, uint32_t& e) {
    int L = g.leaf[s];
    return hash_find(g.hash, g.hmask, cell_key(g.code[s] >> (3 * L), L, g.B), b, e);
}

// Groups of <= 32 consecutive points of one leaf.  Position s starts a group
// when it opens its leaf, or when the leaf holds 32 or more points before s
// (leaves above 32 points only occur at level 0) and s - b is a multiple of
// 32, b the leaf's first position (from the cell table).
__global__ void leaf_groups_kernel(GridView g, int64_t n, int4* groups, int* ngroups) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool start = false;
    int cnt = 0, L = 0;
    if (s < n) {
        L = g.leaf[s];
        const u64 p = g.code[s] >> (3 * L);
        if (s == 0 || (g.code[s - 1] >> (3 * L)) != p) {
            start = true;
        } else if (s >= 32 && (g.code[s - 32] >> (3 * L)) == p) {
            uint32_t b, e;
            start = leaf_range(g, s, b, e) && ((uint32_t)s - b) % 32 == 0;
        }
        if (start) {
            cnt = 1;
            while (cnt < 32 && s + cnt < n && (g.code[s + cnt] >> (3 * L)) == p) cnt++;
        }
    }
    const int slot = block_append(start, ngroups);
    if (start) groups[slot] = make_int4((int)s, cnt, L, 0);
}

cudaError_t launch_leaf_groups(const GridView& g, int64_t n, int4* groups, int* ngroups,
                               cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ngroups, 0, sizeof(int), st);
    if (e) return e;
    leaf_groups_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, n, groups, ngroups); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ compaction
__global__ void compact_count_kernel(const uint8_t* __restrict__ flag, int64_t n,
                                     uint32_t* counts) {
    __shared__ uint32_t ws[8];
    int64_t base = (int64_t)blockIdx.x * 1024;
    uint32_t c = 0;
    for (int j = 0; j < 4; j++) {
        int64_t i = base + j * 256 + threadIdx.x;
        c += (i < n && flag[i]) ? 1u : 0u;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < 8; w++) s += ws[w];
        counts[blockIdx.x] = s;
    }
}

__global__ void compact_write_kernel(const uint8_t* __restrict__ flag, int64_t n,
                                     const uint32_t* __restrict__ offs, int nblk, int* out,
                                     int* count) {
    __shared__ uint32_t ws[8];
    __shared__ uint32_t run;
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) run = offs[blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * 1024;
    for (int j = 0; j < 4; j++) {
        __syncthreads();
        int64_t i = base + j * 256 + t;
        bool f = i < n && flag[i];
        unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) ws[w] = __popc(bal);
        __syncthreads();
        uint32_t off = run;
        for (int ww = 0; ww < w; ww++) off += ws[ww];
        if (f) out[off + __popc(bal & ((1u << lane) - 1u))] = (int)i;
        __syncthreads();
        if (t == 0) {
            uint32_t s = 0;
            for (int ww = 0; ww < 8; ww++) s += ws[ww];
            run += s;
        }
    }
    __syncthreads();
    if (blockIdx.x == nblk - 1 && t == 0) *count = (int)run;
}

cudaError_t stable_compact(const uint8_t* flag, int64_t n, int* out, int* count,
                           const Scratch& s, cudaStream_t st) {
    if (n <= 0) return cudaMemsetAsync(count, 0, sizeof(int), st);
    int nblk = (int)((n + 1023) / 1024);
    uint32_t* offs = (uint32_t*)s.get((size_t)nblk * sizeof(uint32_t));
    if (!offs) return cudaErrorMemoryAllocation;
    compact_count_kernel<<<nblk, 256, 0, st>>>(flag, n, offs); note_launch();
    cudaError_t e = cudaGetLastError();
    if (!e) e = exclusive_scan_u32(offs, nblk, s, st);
    if (!e) {
        compact_write_kernel<<<nblk, 256, 0, st>>>(flag, n, offs, nblk, out, count); note_launch();
        e = cudaGetLastError();
    }
    s.put(offs);
    return e;
}

}  // namespace pd
