// pd_internal.cuh -- shared device definitions of libpd (sm_103a).
//
// Layout of one resident cloud (all arrays indexed by the point's position s
// in Morton order, 0 <= s < n):
//   pos[s]    int4 {x, y, z, input index}     16 B, read by every neighbour scan
//   code[s]   uint64 Morton code of (x,y,z) - origin, >> shift
//   leaf[s]   uint8 level of the octree leaf that holds s
//   alive[s]  uint8 1 while the point is retained
//   prim[s]   uint64 primary key, larger = higher cost (see key_prim_*)
//   nbr[s*S+i] int32 Morton positions of the S nearest live points
//   rk2[s]    uint64 squared distance of the k-th nearest (UINT64_MAX if none)
//   flg[s]    uint8 bit0: a further point ties the k-th distance
//                   bit1: (k = 1) the stored nearest-distance shell may be incomplete
// A cell of level L is the set of points whose codes share the prefix
// code >> 3L; it is a contiguous range of the Morton order.  The octree keeps
// splitting cells holding more than T points; its nodes (internal and leaf)
// are stored in an open-addressing hash keyed by (level, prefix).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define PD_WARPS 4                 // warps per block in warp-per-group kernels
#define PD_MAXLEVEL 21             // Morton bits per axis
#define PD_EMPTY_KEY 0ull

namespace pd {

struct HashSlot {
    unsigned long long key;        // marker-bit encoded (level, prefix); 0 = empty
    uint32_t b, e;                 // [b, e) in Morton order
};

struct GridView {
    const int4* pos;
    const unsigned long long* code;
    const uint8_t* leaf;
    const HashSlot* hash;
    unsigned long long hmask;
    int B;         // Morton bits per axis of the root cell
    int shift;     // coordinates are (x - origin) >> shift before interleaving
    int T;         // largest leaf
    int3 origin;
    int3 umax;     // largest (x - origin) per axis
};

// ---------------------------------------------------------------- Morton
__host__ __device__ inline unsigned long long spread3(uint32_t v) {
    unsigned long long x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
__host__ __device__ inline uint32_t compact3(unsigned long long x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}
__host__ __device__ inline unsigned long long morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// (level, prefix) -> hash key: a marker bit just above the prefix's 3(B-L) bits.
__device__ inline unsigned long long cell_key(unsigned long long prefix, int L, int B) {
    return (1ull << (3 * (B - L))) | prefix;
}
__device__ inline unsigned long long mix64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}
__device__ inline bool hash_find(const HashSlot* tab, unsigned long long mask,
                                 unsigned long long key, uint32_t& b, uint32_t& e) {
    unsigned long long h = mix64(key) & mask;
    for (unsigned long long i = 0; i <= mask; i++) {
        unsigned long long k = tab[h].key;
        if (k == key) {
            b = tab[h].b;
            e = tab[h].e;
            return true;
        }
        if (k == PD_EMPTY_KEY) return false;
        h = (h + 1) & mask;
    }
    return false;
}

// Range of the level-L cell (cx,cy,cz).  Returns 0 = empty, 1 = the cell is an
// octree node (its exact range), 2 = the cell lies inside a coarser leaf
// (the whole leaf's range is returned; *lvl_out = that leaf's level).
__device__ inline int resolve_cell(const GridView& g, int L, int cx, int cy, int cz,
                                   uint32_t& b, uint32_t& e, int* lvl_out) {
    int lim = 1 << (g.B - L);
    if (cx < 0 || cy < 0 || cz < 0 || cx >= lim || cy >= lim || cz >= lim) return 0;
    unsigned long long prefix = morton3((uint32_t)cx, (uint32_t)cy, (uint32_t)cz);
    if (hash_find(g.hash, g.hmask, cell_key(prefix, L, g.B), b, e)) {
        *lvl_out = L;
        return 1;
    }
    for (int L2 = L + 1; L2 <= g.B; L2++) {
        prefix >>= 3;
        if (hash_find(g.hash, g.hmask, cell_key(prefix, L2, g.B), b, e)) {
            if (e - b > (uint32_t)g.T) return 0;  // internal node: that child is empty
            *lvl_out = L2;
            return 2;
        }
    }
    return 0;
}

// ---------------------------------------------------------------- keys
// Larger key = removed first: (cost, input index) compared lexicographically.
// k = 1 density cost: order by d1^2 ascending, encoded as the complement of
// the IEEE bits of (double)d1^2 (exact: d^2 < 2^53).  Other costs: the IEEE
// bits of the non-negative binary64 cost (+inf for coincident points).
__device__ inline unsigned long long key_prim_d2(unsigned long long d2) {
    double v = d2 == ~0ull ? __longlong_as_double(0x7ff0000000000000ll) : (double)d2;
    return ~(unsigned long long)__double_as_longlong(v);
}
__device__ inline unsigned long long key_prim_cost(double c) {
    return (unsigned long long)__double_as_longlong(c);
}
__device__ inline bool key_gt(unsigned long long pa, int ia, unsigned long long pb, int ib) {
    return pa > pb || (pa == pb && ia > ib);
}

// Per-neighbour weight of the optional cost terms (section "Additional cost
// terms"): 1 - a * ||rgb_p - rgb_q|| / (255 sqrt 3) for colour, 1 - a * (1 -
// |n_p . n_q|) for orientation (Eq. 13), 1 otherwise.  Every operation is a
// separately rounded binary64 operation (no contraction).
__device__ inline double term_weight(int term, double a, const uchar4* rgb, const float4* nrm,
                                     int q, int j) {
    if (term == 1) {
        uchar4 p = rgb[q], r = rgb[j];
        double dr = (double)p.x - (double)r.x;
        double dg = (double)p.y - (double)r.y;
        double db = (double)p.z - (double)r.z;
        double s = __dmul_rn(dr, dr);
        s = __dadd_rn(s, __dmul_rn(dg, dg));
        s = __dadd_rn(s, __dmul_rn(db, db));
        double dist = __dsqrt_rn(s);
        double scale = __dmul_rn(255.0, __dsqrt_rn(3.0));
        return __dsub_rn(1.0, __dmul_rn(a, __ddiv_rn(dist, scale)));
    }
    if (term == 2) {
        float4 p = nrm[q], r = nrm[j];
        double d = __dmul_rn((double)p.x, (double)r.x);
        d = __dadd_rn(d, __dmul_rn((double)p.y, (double)r.y));
        d = __dadd_rn(d, __dmul_rn((double)p.z, (double)r.z));
        return __dsub_rn(1.0, __dmul_rn(a, __dsub_rn(1.0, fabs(d))));
    }
    return 1.0;
}

__device__ inline unsigned long long sqd(int4 a, int4 b) {
    long long dx = (long long)a.x - b.x, dy = (long long)a.y - b.y, dz = (long long)a.z - b.z;
    return (unsigned long long)(dx * dx + dy * dy + dz * dz);
}

// ---------------------------------------------------------------- launches
// Number of kernels this library has launched (process-wide, host counter).
extern long long g_launch_count;
inline void note_launch() { __atomic_fetch_add(&g_launch_count, 1, __ATOMIC_RELAXED); }

// Block-level aggregation of counters and list appends: one global atomic
// per block instead of one per warp (atomics on one address serialise in L2,
// and a full-grid kernel over a billion points has 31M warps).  Every thread
// of the block must make the call (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ void block_add(unsigned long long* dst, unsigned long long v) {
    __shared__ unsigned long long s_part[32];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // s_part may still be read by a previous call
    if (lane == 0) s_part[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += s_part[i];
        if (t) atomicAdd(dst, t);
    }
}
// Two counters at once (one reduction, two atomics per block).
__device__ __forceinline__ void block_add2(unsigned long long* d1, unsigned long long v1,
                                           unsigned long long* d2, unsigned long long v2) {
    __shared__ unsigned long long s_p1[32], s_p2[32];
    for (int o = 16; o; o >>= 1) {
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        s_p1[w] = v1;
        s_p2[w] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t1 = 0, t2 = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            t1 += s_p1[i];
            t2 += s_p2[i];
        }
        if (t1) atomicAdd(d1, t1);
        if (t2) atomicAdd(d2, t2);
    }
}
// Appends for every thread with want set; returns the thread's slot in the
// list (meaningful where want is set).
__device__ __forceinline__ int block_append(bool want, int* count) {
    __shared__ int s_w[33];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, want);
    __syncthreads();  // s_w may still be read by a previous call
    if (lane == 0) s_w[w] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            int c = s_w[i];
            s_w[i] = acc;
            acc += c;
        }
        s_w[32] = acc ? atomicAdd(count, acc) : 0;
    }
    __syncthreads();
    return s_w[32] + s_w[w] + __popc(m & ((1u << lane) - 1u));
}

// Streaming multiprocessors of the current device (queried once per device
// and cached); persistent and grid-stride launches size their grids from it.
int device_sms();

// ---------------------------------------------------------------- warp utils
__device__ inline int warp_lane() { return threadIdx.x & 31; }

// The 3x3x3 cells around a query cell in the order they are scanned: the
// cell itself, the 6 face neighbours, the 12 edge and the 8 corner neighbours
// (cell o = (dx+1) + 3 (dy+1) + 9 (dz+1)).  Nearer cells first tighten the
// k-th distance bound early, which prunes more of the farther cells.
static __device__ __constant__ const unsigned char kCellOrder[27] = {13, 4, 10, 12, 14, 16, 22, 1, 3, 5, 7, 9, 11, 15, 17, 19, 21, 23, 25, 0, 2, 6, 8, 18, 20, 24, 26};

}  // namespace pd
