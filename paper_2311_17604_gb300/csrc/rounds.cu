// rounds.cu -- device-side removal rounds that reproduce the sequential greedy.
//
// The sequential greedy (section "Computing per-sample costs"; section
// "Sub-sampling algorithm", step 2: removing a point never raises a cost)
// pops the live point of largest key (cost, input index).  A round removes a
// set P at once; P is chosen so that the sequential run pops exactly the
// points of P among its next `need` pops and, apart from them, behaves as the
// run on the cloud without P:
//   (R2) key(p) >= K*, the need-th largest live key, so p is popped within
//        the next `need` pops once its key cannot change;
//   (A)  key(p) does not change when every point of larger key is removed,
//        so it stays fixed until p is popped;
//   (B)  p can never change the key of a point x that is popped before p
//        while x is not itself in P.
// k = 1: (A) holds iff p has no neighbour or some point at distance d1(p)
//        (the "shell") has a smaller key; (B) holds iff every shell member
//        of larger input index is itself in P (a fixpoint over P).
// k >= 2: (A) is checked by a neighbour search restricted to smaller keys;
//        (B) by counting, for every larger-key point x near p, the points of
//        key below key(p) that are closer to x than p is: p can enter x's k
//        nearest only if fewer than k of them exist (again a fixpoint).
// Before the rounds, coincident points (infinite cost) are removed in one
// step: all but the smallest input index of each coincident class are the
// first pops of the sequential run, in decreasing index order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_internal.cuh"
#include "pd_kernels.h"

namespace pd {

#define FULLM 0xffffffffu

// ------------------------------------------------------------------ duplicates
__global__ void dup_flag_kernel(const u64* __restrict__ code, const int4* __restrict__ pos,
                                int64_t n, uint8_t* dup, unsigned long long* count) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned c = 0;
    if (s < n) {
        uint8_t f = 0;
        if (s > 0 && code[s] == code[s - 1]) {
            int4 a = pos[s], b = pos[s - 1];
            f = a.x == b.x && a.y == b.y && a.z == b.z;
        }
        dup[s] = f;
        c = f;
    }
    block_add(count, c);
}

// remove flagged duplicates whose input index is >= idx_min
__global__ void dup_remove_kernel(const uint8_t* __restrict__ dup, const int4* __restrict__ pos,
                                  int64_t n, int idx_min, uint8_t* alive) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    alive[s] = !(dup[s] && pos[s].w >= idx_min);
}

// ------------------------------------------------------------------ selection
// Digit `pass` (12 bits) of the 96-bit key (prim << 32 | input index),
// most significant first: passes 0-4 read prim, 5 straddles, 6-7 read idx.
__device__ inline uint32_t key_digit(u64 prim, int idx, int pass) {
    int lo = 84 - 12 * pass;  // lowest bit of the digit
    uint32_t ui = (uint32_t)idx;
    if (lo >= 32) return (uint32_t)(prim >> (lo - 32)) & 0xfffu;
    if (lo + 12 <= 32) return (ui >> lo) & 0xfffu;
    // straddle: bits [lo, 32) of idx and [0, lo + 12 - 32) of prim
    int nlow = 32 - lo;
    return ((uint32_t)(prim << nlow) | (ui >> lo)) & 0xfffu;
}
__device__ inline bool prefix_match(u64 prim, int idx, int npass, const uint32_t* pre) {
    for (int p = 0; p < npass; p++)
        if (key_digit(prim, idx, p) != pre[p]) return false;
    return true;
}

struct SelPrefix {
    uint32_t d[8];
};

// Histogram of digit `pass`.  Grid mode (lp == NULL, pass 0 only): every
// alive grid point.  List mode: compacted (prim, idx) pairs that match the
// digits chosen so far.
__global__ void sel_hist_kernel(const u64* __restrict__ prim, const uint8_t* __restrict__ alive,
                                int64_t n, const u64* __restrict__ lp, const int* __restrict__ li,
                                int64_t llen, int pass, SelPrefix pre, uint32_t* hist) {
    __shared__ uint32_t h[4096];
    for (int x = threadIdx.x; x < 4096; x += blockDim.x) h[x] = 0;
    __syncthreads();
    int64_t len = lp ? llen : n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (lp) {
            u64 p = lp[i];
            int id = li[i];
            if (!prefix_match(p, id, pass, pre.d)) continue;
            atomicAdd(&h[key_digit(p, id, pass)], 1u);
        } else {
            if (!alive[i]) continue;
            atomicAdd(&h[(uint32_t)(prim[i] >> 52)], 1u);
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < 4096; x += blockDim.x)
        if (h[x]) atomicAdd(&hist[x], h[x]);
}

// Keep the entries whose digits 0..pass equal pre[0..pass].
__global__ void sel_compact_kernel(const u64* __restrict__ prim, const int4* __restrict__ pos,
                                   const uint8_t* __restrict__ alive, int64_t n,
                                   const u64* __restrict__ lp, const int* __restrict__ li,
                                   int64_t llen, int pass, SelPrefix pre, u64* op, int* oi,
                                   int* ocount) {
    int64_t len = lp ? llen : n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        u64 p;
        int id;
        if (lp) {
            p = lp[i];
            id = li[i];
            if (!prefix_match(p, id, pass + 1, pre.d)) continue;
        } else {
            if (!alive[i]) continue;
            p = prim[i];
            if ((uint32_t)(p >> 52) != pre.d[0]) continue;
            id = pos[i].w;
        }
        int slot = atomicAdd(ocount, 1);
        op[slot] = p;
        oi[slot] = id;
    }
}

// (B) for k = 1: a shell member of larger input index must be in P.  The
// shell is the first flg >> 2 stored neighbours.
__global__ void k1_fix_kernel(const int* __restrict__ cand, const int* __restrict__ ncand,
                              const int4* __restrict__ pos, const int* __restrict__ nbr,
                              const uint8_t* __restrict__ flg, int S,
                              const uint8_t* __restrict__ inP, uint8_t* rej, int* changed) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *ncand) return;
    int s = cand[t];
    if (rej[s]) return;
    int is = pos[s].w;
    int shell = flg[s] >> 2;
    for (int i = 0; i < shell; i++) {
        int x = nbr[(int64_t)s * S + i];
        if (x < 0) continue;
        if (pos[x].w > is && (!inP[x] || rej[x])) {
            rej[s] = 1;
            *changed = 1;
            return;
        }
    }
}

// Danger pairs.  One warp per source x: collect every live point y with
// d^2(x,y) < lam(x) (lam = k-th squared distance from x to keys below tau),
// then for each candidate p among them with key(p) < key(x) count the points
// y != p of key below key(p) with d^2(x,y) <= d^2(x,p); fewer than k means p
// could enter x's k nearest before it is popped: record (x, p).
#define DG_CAP 512
#define DG_WARPS 2
#define DG_BLOCKS_PER_SM 14  // resident blocks per SM (registers capped to fit)
#define PD_DG_SMAX 8  // stored neighbours used as shields (S up to 8)

__device__ inline u64 box_d2x(int ux, int uy, int uz, int bx, int by, int bz, int sh) {
    long long q[3] = {ux, uy, uz};
    int c[3] = {bx, by, bz};
    u64 s = 0;
    for (int a = 0; a < 3; a++) {
        long long lo = (long long)c[a] << sh;
        long long hi = ((long long)(c[a] + 1) << sh) - 1;
        long long d = q[a] < lo ? lo - q[a] : (q[a] > hi ? q[a] - hi : 0);
        s += (u64)(d * d);
    }
    return s;
}

// Cells of the level-L cube around a point that hold every point closer than
// sqrt(lam); returns the level (the first whose cube covers that ball).
__device__ inline int cover_level(const GridView& g, int ux, int uy, int uz, u64 c0, int L0,
                                  u64 lam, int& cx, int& cy, int& cz) {
    for (int L = L0;; L++) {
        cx = cy = cz = 0;
        if (L >= g.B) return g.B;
        cx = (int)compact3(c0 >> (3 * L));
        cy = (int)compact3(c0 >> (3 * L + 1));
        cz = (int)compact3(c0 >> (3 * L + 2));
        int sh = L + g.shift;
        long long q[3] = {ux, uy, uz};
        int c[3] = {cx, cy, cz};
        int m[3] = {g.umax.x, g.umax.y, g.umax.z};
        long long best = -1;
        for (int a = 0; a < 3; a++) {
            long long lo = (long long)(c[a] - 1) << sh, hi = (long long)(c[a] + 2) << sh;
            if (lo > 0 && (best < 0 || q[a] - lo + 1 < best)) best = q[a] - lo + 1;
            if (hi <= m[a] && (best < 0 || hi - q[a] < best)) best = hi - q[a];
        }
        if (best < 0 || lam <= (u64)best * (u64)best) return L;
    }
}

// Danger pairs (condition (B), k >= 2).  One warp per source x (key above
// tau, lam = k-th squared distance from x to keys below tau):
//   1. collect the candidates p (in P so far, key below x's) with d^2(x,p) < lam;
//   2. for 32 candidates at a time stream every live point y with
//      d^2(x,y) < lam and count, per candidate, the y != p with
//      d^2(x,y) <= d^2(x,p) and key(y) < key(p), stopping once all 32 counts
//      reach k; a count below k means p could enter x's k nearest before p is
//      popped: record (x, p).
// Candidates beyond the list capacity are rejected without counting.
struct DangerSmem {
    int c_j[DG_WARPS][DG_CAP];
    u64 c_d[DG_WARPS][DG_CAP];
    u64 st_d[DG_WARPS][32];  // staged points within the batch's farthest candidate:
    u64 st_k[DG_WARPS][32];  // d^2 to the source, key, input index, Morton position
    int st_o[DG_WARPS][32];
    int st_j[DG_WARPS][32];
};

__device__ void danger_one(const GridView& g, int x, const u64* __restrict__ prim,
                           const uint8_t* __restrict__ alive, const uint8_t* __restrict__ inP,
                           uint8_t* rej, const u64* __restrict__ lam, const int* __restrict__ nbr,
                           int S, int k, int2* pairs, int* npairs, int pair_cap, int* overflow,
                           unsigned long long* diag, const int* __restrict__ csorted,
                           const int* __restrict__ ncs, DangerSmem& sm, int w, int lane) {
    int(&c_j)[DG_WARPS][DG_CAP] = sm.c_j;
    u64(&c_d)[DG_WARPS][DG_CAP] = sm.c_d;
    u64(&st_d)[DG_WARPS][32] = sm.st_d;
    u64(&st_k)[DG_WARPS][32] = sm.st_k;
    int(&st_o)[DG_WARPS][32] = sm.st_o;
    int(&st_j)[DG_WARPS][32] = sm.st_j;
    __syncwarp();
    int4 xp = g.pos[x];
    u64 px = prim[x];
    u64 lx = lam[x];
    if (lx == ~0ull) {  // fewer than k low points in the cloud: host falls back
        if (lane == 0) *overflow = 1;
        return;
    }
    int ux = xp.x - g.origin.x, uy = xp.y - g.origin.y, uz = xp.z - g.origin.z;
    int cx, cy, cz;
    int L = cover_level(g, ux, uy, uz, g.code[x], g.leaf[x], lx, cx, cy, cz);
    int o = lane < 27 ? kCellOrder[lane] : 13;
    int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    uint32_t rb = 0, re = 0;
    int rl = L, rt = 0;
    if (lane < 27) rt = resolve_cell(g, L, cx + dx, cy + dy, cz + dz, rb, re, &rl);
    for (int j = 0; j < 27; j++) {
        uint32_t bj = __shfl_sync(FULLM, rb, j);
        int tj = __shfl_sync(FULLM, rt, j);
        if (j < lane && rt == 2 && tj == 2 && bj == rb) rt = 0;
    }
    // squared distance from x to each resolved range's box: ranges entirely
    // beyond lam (or beyond the candidates being counted) are skipped
    u64 rbox = ~0ull;
    if (rt) {
        int sh = rl - L;
        rbox = box_d2x(ux, uy, uz, (cx + dx) >> sh, (cy + dy) >> sh, (cz + dz) >> sh,
                       rl + g.shift);
        if (rbox >= lx) rt = 0;
    }
    // 1. candidates: when a Morton-sorted list of them is given, each range
    // [b, e) maps to a slice of that list by binary search; otherwise the
    // range's points are streamed and filtered
    int nc = 0;
    uint32_t cs_lo = 0, cs_hi = 0;
    if (csorted && rt) {
        int nlist = *ncs;
        int lo = 0, hi = nlist;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if ((uint32_t)csorted[mid] < rb) lo = mid + 1;
            else hi = mid;
        }
        cs_lo = (uint32_t)lo;
        hi = nlist;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if ((uint32_t)csorted[mid] < re) lo = mid + 1;
            else hi = mid;
        }
        cs_hi = (uint32_t)lo;
    }
    for (int r = 0; r < 27; r++) {
        int tr = __shfl_sync(FULLM, rt, r);
        if (!tr) continue;
        uint32_t b = __shfl_sync(FULLM, rb, r), e = __shfl_sync(FULLM, re, r);
        if (csorted) {
            b = __shfl_sync(FULLM, cs_lo, r);
            e = __shfl_sync(FULLM, cs_hi, r);
        }
        for (uint32_t c = b; c < e; c += 32) {
            uint32_t jj = c + lane;
            uint32_t j = (csorted && jj < e) ? (uint32_t)csorted[jj] : jj;
            bool take = false;
            u64 d2 = 0;
            if (jj < e && (int)j != x && alive[j] && inP[j]) {
                int4 v = g.pos[j];
                long long ddx = v.x - xp.x, ddy = v.y - xp.y, ddz = v.z - xp.z;
                d2 = (u64)(ddx * ddx + ddy * ddy + ddz * ddz);
                take = d2 < lx && key_gt(px, xp.w, prim[j], v.w);
            }
            unsigned bal = __ballot_sync(FULLM, take);
            int slot = nc + __popc(bal & ((1u << lane) - 1u));
            if (take) {
                if (slot < DG_CAP) {
                    c_j[w][slot] = (int)j;
                    c_d[w][slot] = d2;
                } else {
                    rej[j] = 1;
                }
            }
            nc += __popc(bal);
        }
    }
    if (diag && lane == 0) {
        if (nc > DG_CAP) atomicAdd(diag, (unsigned long long)(nc - DG_CAP));
    }
    nc = min(nc, DG_CAP);
    __syncwarp();
    // x's stored neighbours are live points near x: the cheapest shields
    int sn_j[PD_DG_SMAX];
    u64 sn_d[PD_DG_SMAX], sn_k[PD_DG_SMAX];
    int sn_i[PD_DG_SMAX];
#pragma unroll
    for (int i = 0; i < PD_DG_SMAX; i++) {
        sn_j[i] = -1;
        sn_d[i] = ~0ull;
        sn_k[i] = 0;
        sn_i[i] = 0;
        if (nbr && i < S && nc > 0) {
            int y = nbr[(int64_t)x * S + i];
            if (y >= 0) {
                int4 v = g.pos[y];
                long long ddx = v.x - xp.x, ddy = v.y - xp.y, ddz = v.z - xp.z;
                sn_j[i] = y;
                sn_d[i] = (u64)(ddx * ddx + ddy * ddy + ddz * ddz);
                sn_k[i] = prim[y];
                sn_i[i] = v.w;
            }
        }
    }
    // 2. counting, 32 candidates at a time
    for (int a0 = 0; a0 < nc; a0 += 32) {
        int a = a0 + lane;
        bool done = a >= nc;
        int p = done ? -1 : c_j[w][a];
        u64 dp = done ? 0 : c_d[w][a];
        u64 pp = done ? 0 : prim[p];
        int ip = done ? 0 : g.pos[p].w;
        int cnt = 0;
        if (!done) {
#pragma unroll
            for (int i = 0; i < PD_DG_SMAX; i++)
                if (sn_j[i] >= 0 && sn_j[i] != p && sn_d[i] <= dp &&
                    key_gt(pp, ip, sn_k[i], sn_i[i]))
                    cnt++;
            if (cnt >= k) done = true;
            cnt = 0;  // the stream below recounts every point (stored ones included)
        }
        u64 dmax = done ? 0 : dp;  // farthest candidate of this batch
        for (int o2 = 16; o2; o2 >>= 1) {
            u64 other = __shfl_xor_sync(FULLM, dmax, o2);
            dmax = other > dmax ? other : dmax;
        }
        for (int r = 0; r < 27; r++) {
            int tr = __shfl_sync(FULLM, rt, r);
            if (!tr) continue;
            if (__all_sync(FULLM, done)) break;
            if (__shfl_sync(FULLM, rbox, r) > dmax) continue;
            uint32_t b = __shfl_sync(FULLM, rb, r), e = __shfl_sync(FULLM, re, r);
            for (uint32_t c = b; c < e; c += 32) {
                // each lane loads one point and its distance to x; only points
                // within the batch's farthest open candidate can shield, and
                // they are compacted into the staging buffer
                uint32_t j = c + lane;
                bool near = false;
                u64 d2 = 0, ky = 0;
                int oy = 0;
                if (j < e) {  // independent loads, issued together
                    uint8_t al = alive[j];
                    int4 v = g.pos[j];
                    ky = prim[j];
                    long long ddx = v.x - xp.x, ddy = v.y - xp.y, ddz = v.z - xp.z;
                    d2 = (u64)(ddx * ddx + ddy * ddy + ddz * ddz);
                    near = al && (int)j != x && d2 <= dmax;
                    oy = v.w;
                }
                unsigned nb = __ballot_sync(FULLM, near);
                if (near) {
                    int slot = __popc(nb & ((1u << lane) - 1u));
                    st_d[w][slot] = d2;
                    st_k[w][slot] = ky;
                    st_o[w][slot] = oy;
                    st_j[w][slot] = (int)j;
                }
                __syncwarp();
                int mm = __popc(nb);
                if (!done) {
                    for (int tt = 0; tt < mm; tt++) {
                        if (st_j[w][tt] == p) continue;
                        if (st_d[w][tt] <= dp && key_gt(pp, ip, st_k[w][tt], st_o[w][tt])) {
                            if (++cnt >= k) {
                                done = true;
                                break;
                            }
                        }
                    }
                }
                __syncwarp();
                if (__all_sync(FULLM, done)) break;
            }
        }
        if (!done) {
            int ps = atomicAdd(npairs, 1);
            if (ps < pair_cap) pairs[ps] = make_int2(x, p);
            else *overflow = 1;
        }
    }
}

__global__ void __launch_bounds__(DG_WARPS * 32, DG_BLOCKS_PER_SM)
    danger_kernel(GridView g, const int* __restrict__ src, const int* __restrict__ nsrc,
                  const u64* __restrict__ prim, const uint8_t* __restrict__ alive,
                  const uint8_t* __restrict__ inP, uint8_t* rej, const u64* __restrict__ lam,
                  const int* __restrict__ nbr, int S, int k, int2* pairs, int* npairs,
                  int pair_cap, int* overflow, unsigned long long* diag,
                  const int* __restrict__ csorted, const int* __restrict__ ncs) {
    __shared__ DangerSmem sm;
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int ns = *nsrc;
    for (int t = blockIdx.x * DG_WARPS + w; t < ns; t += gridDim.x * DG_WARPS)
        danger_one(g, src[t], prim, alive, inP, rej, lam, nbr, S, k, pairs, npairs, pair_cap,
                   overflow, diag, csorted, ncs, sm, w, lane);
}

// Fallback: accept every live point with key >= tau (tau = the top key).
__global__ void accept_above_kernel(const u64* __restrict__ prim, const int4* __restrict__ pos,
                                    const uint8_t* __restrict__ alive, int64_t n, u64 tp, int ti,
                                    uint8_t* inP, int* cand, int* ncand) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n || !alive[s]) return;
    if (key_gt(tp, ti, prim[s], pos[s].w)) return;
    inP[s] = 1;
    cand[atomicAdd(ncand, 1)] = (int)s;
}

// (B) fixpoint over pairs: p is rejected while its source x is not in P.
__global__ void pair_fix_kernel(const int2* __restrict__ pairs, const int* __restrict__ npairs,
                                int pair_cap, const uint8_t* __restrict__ inP, uint8_t* rej,
                                int* changed) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int np = min(*npairs, pair_cap);
    if (t >= np) return;
    int2 pr = pairs[t];
    if (rej[pr.y]) return;
    if (!inP[pr.x] || rej[pr.x]) {
        rej[pr.y] = 1;
        *changed = 1;
    }
}

// ------------------------------------------------------------------ removal
__global__ void remove_kernel(const int* __restrict__ cand, const int* __restrict__ ncand,
                              uint8_t* inP, uint8_t* rej, uint8_t* alive,
                              unsigned long long* removed) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned c = 0;
    if (t < *ncand) {
        int s = cand[t];
        if (inP[s] && !rej[s]) {
            alive[s] = 0;
            c = 1;
        }
        inP[s] = 0;
        rej[s] = 0;
    }
    block_add(removed, c);
}

__global__ void keep_kernel(const int4* __restrict__ pos, const uint8_t* __restrict__ alive,
                            int64_t n, uint8_t* keep) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    if (alive[s]) keep[pos[s].w] = 1;
}

// cost / neighbour output in input order (pd_knn_cost)
__global__ void knn_out_kernel(const int4* __restrict__ pos, const double* __restrict__ cost_s,
                               const int* __restrict__ nbr, int64_t n, int S, int k,
                               double* cost, int32_t* knn) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = pos[s].w;
    if (cost) cost[i] = cost_s[s];
    if (knn) {
        for (int j = 0; j < k; j++) {
            int x = nbr[s * S + j];
            knn[(int64_t)i * k + j] = x >= 0 ? pos[x].w : -1;
        }
    }
}

// remap stored neighbours after a compaction of the live points
__global__ void remap_kernel(const int* __restrict__ live_list, int64_t nl, const int* old_nbr,
                             int* new_nbr, const int* __restrict__ newpos, int64_t nold, int S) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nl) return;
    int s = live_list[t];
    for (int i = 0; i < S; i++) {
        int x = old_nbr[(int64_t)s * S + i];
        new_nbr[t * S + i] = (x >= 0 && x < nold) ? newpos[x] : -1;
    }
}

template <typename T>
__global__ void take_kernel(const int* __restrict__ list, int64_t nl, const T* __restrict__ src,
                            T* dst) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nl) dst[t] = src[list[t]];
}

__global__ void newpos_kernel(const int* __restrict__ list, int64_t nl, int* newpos) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nl) newpos[list[t]] = (int)t;
}

// ------------------------------------------------------------------ launchers
#define GRID1(n) (unsigned)(((n) + 255) / 256), 256

cudaError_t launch_dup_flag(const u64* code, const int4* pos, int64_t n, uint8_t* dup,
                            unsigned long long* count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e) return e;
    dup_flag_kernel<<<GRID1(n), 0, st>>>(code, pos, n, dup, count); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_dup_remove(const uint8_t* dup, const int4* pos, int64_t n, int idx_min,
                              uint8_t* alive, cudaStream_t st) {
    dup_remove_kernel<<<GRID1(n), 0, st>>>(dup, pos, n, idx_min, alive); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_sel_hist(const u64* prim, const uint8_t* alive, int64_t n, const u64* lp,
                            const int* li, int64_t llen, int pass, const uint32_t* pre,
                            uint32_t* hist, cudaStream_t st) {
    SelPrefix sp;
    for (int i = 0; i < 8; i++) sp.d[i] = i < pass ? pre[i] : 0;
    cudaError_t e = cudaMemsetAsync(hist, 0, 4096 * sizeof(uint32_t), st);
    if (e) return e;
    int64_t len = lp ? llen : n;
    int blocks = (int)((len + 255) / 256);
    if (blocks > device_sms() * 4) blocks = device_sms() * 4;
    if (blocks < 1) blocks = 1;
    sel_hist_kernel<<<blocks, 256, 0, st>>>(prim, alive, n, lp, li, llen, pass, sp, hist); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_sel_compact(const u64* prim, const int4* pos, const uint8_t* alive, int64_t n,
                               const u64* lp, const int* li, int64_t llen, int pass,
                               const uint32_t* pre, u64* op, int* oi, int* ocount,
                               cudaStream_t st) {
    SelPrefix sp;
    for (int i = 0; i < 8; i++) sp.d[i] = i <= pass ? pre[i] : 0;
    cudaError_t e = cudaMemsetAsync(ocount, 0, sizeof(int), st);
    if (e) return e;
    int64_t len = lp ? llen : n;
    int blocks = (int)((len + 255) / 256);
    if (blocks > device_sms() * 8) blocks = device_sms() * 8;
    if (blocks < 1) blocks = 1;
    sel_compact_kernel<<<blocks, 256, 0, st>>>(prim, pos, alive, n, lp, li, llen, pass, sp, op,
                                               oi, ocount); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_k1_fix(const int* cand, const int* ncand, int max_cand, const int4* pos,
                          const int* nbr, const uint8_t* flg, int S, const uint8_t* inP,
                          uint8_t* rej, int* changed, cudaStream_t st) {
    if (max_cand <= 0) return cudaSuccess;
    k1_fix_kernel<<<GRID1(max_cand), 0, st>>>(cand, ncand, pos, nbr, flg, S, inP, rej, changed); note_launch();
    return cudaGetLastError();
}
cudaError_t round_launch_danger(const GridView& g, const int* src, const u64* prim,
                                const uint8_t* alive, const uint8_t* inP, uint8_t* rej,
                                const u64* lam, const int* nbr, int S, int k, int2* pairs,
                                int pair_cap, const int* csorted, RoundDev* rd, cudaStream_t st) {
    danger_kernel<<<device_sms() * DG_BLOCKS_PER_SM, DG_WARPS * 32, 0, st>>>(g, src, &rd->nsrc, prim, alive, inP, rej,
                                                     lam, S <= PD_DG_SMAX ? nbr : nullptr, S, k,
                                                     pairs, &rd->npairs, pair_cap, &rd->overflow,
                                                     &rd->cap_over, csorted, &rd->ncs); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_accept_above(const u64* prim, const int4* pos, const uint8_t* alive, int64_t n,
                                u64 tp, int ti, uint8_t* inP, int* cand, int* ncand,
                                cudaStream_t st) {
    accept_above_kernel<<<GRID1(n), 0, st>>>(prim, pos, alive, n, tp, ti, inP, cand, ncand); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_pair_fix(const int2* pairs, const int* npairs, int max_pairs, int pair_cap,
                            const uint8_t* inP, uint8_t* rej, int* changed, cudaStream_t st) {
    if (max_pairs <= 0) return cudaSuccess;
    pair_fix_kernel<<<GRID1(max_pairs), 0, st>>>(pairs, npairs, pair_cap, inP, rej, changed); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_remove(const int* cand, const int* ncand, int max_cand, uint8_t* inP,
                          uint8_t* rej, uint8_t* alive, unsigned long long* removed,
                          cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(removed, 0, sizeof(unsigned long long), st);
    if (e || max_cand <= 0) return e;
    remove_kernel<<<GRID1(max_cand), 0, st>>>(cand, ncand, inP, rej, alive, removed); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_keep(const int4* pos, const uint8_t* alive, int64_t n, uint8_t* keep,
                        cudaStream_t st) {
    keep_kernel<<<GRID1(n), 0, st>>>(pos, alive, n, keep); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_knn_out(const int4* pos, const double* cost_s, const int* nbr, int64_t n, int S,
                           int k, double* cost, int32_t* knn, cudaStream_t st) {
    knn_out_kernel<<<GRID1(n), 0, st>>>(pos, cost_s, nbr, n, S, k, cost, knn); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_newpos(const int* list, int64_t nl, int* newpos, cudaStream_t st) {
    newpos_kernel<<<GRID1(nl), 0, st>>>(list, nl, newpos); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_remap(const int* list, int64_t nl, const int* old_nbr, int* new_nbr,
                         const int* newpos, int64_t nold, int S, cudaStream_t st) {
    remap_kernel<<<GRID1(nl), 0, st>>>(list, nl, old_nbr, new_nbr, newpos, nold, S); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_take_u64(const int* list, int64_t nl, const u64* src, u64* dst,
                            cudaStream_t st) {
    take_kernel<u64><<<GRID1(nl), 0, st>>>(list, nl, src, dst); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_take_i4(const int* list, int64_t nl, const int4* src, int4* dst,
                           cudaStream_t st) {
    take_kernel<int4><<<GRID1(nl), 0, st>>>(list, nl, src, dst); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_take_u8(const int* list, int64_t nl, const uint8_t* src, uint8_t* dst,
                           cudaStream_t st) {
    take_kernel<uint8_t><<<GRID1(nl), 0, st>>>(list, nl, src, dst); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_take_uc4(const int* list, int64_t nl, const uchar4* src, uchar4* dst,
                            cudaStream_t st) {
    take_kernel<uchar4><<<GRID1(nl), 0, st>>>(list, nl, src, dst); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_take_f4(const int* list, int64_t nl, const float4* src, float4* dst,
                           cudaStream_t st) {
    take_kernel<float4><<<GRID1(nl), 0, st>>>(list, nl, src, dst); note_launch();
    return cudaGetLastError();
}

}  // namespace pd
