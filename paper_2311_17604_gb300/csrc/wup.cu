// wup.cu -- kernels of the paper's iterative w_up scheme (section
// "Sub-sampling algorithm"), its removal sweep restated as parallel rounds.
//
// An iteration recomputes every live point's S nearest neighbours and cost
// (a full search), takes w_up as the m-th smallest key (cost, index) and
// then removes points above w_up in rounds: a candidate (live, clean, key
// above w_up) goes when no adjacent candidate has a larger key, adjacency
// meaning that one of the two lies among the first k stored neighbours of
// the other.  Removed points leave their reverse neighbours' stored lists;
// a point with at least k stored points left takes its new cost from the
// first k of them, one with fewer is dirty until the next iteration (the
// paper's extended k+b neighbourhood and dirty flag).
//
//   wup_mark_kernel    every candidate raises mark_p[x] to its key's primary
//                      for each of its first k stored neighbours x
//   wup_mark2_kernel   ... and, where it holds that maximum, mark_i[x] to its
//                      index: (mark_p, mark_i) is the largest candidate key
//                      that stores x
//   wup_pick_kernel    a candidate whose own key beats that mark and every
//                      candidate among its first k stored neighbours is
//                      removed in this round
//   wup_update_kernel  removed points leave the stored lists; new cost from
//                      the first k, or the dirty flag
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_internal.cuh"
#include "pd_kernels.h"

namespace pd {

#define FULLM 0xffffffffu
#define WUP_SMAX 8

__device__ __forceinline__ bool wup_cand(const uint8_t* __restrict__ alive,
                                         const uint8_t* __restrict__ wdirty, u64 p, int i,
                                         const RoundDev* rd, int64_t s) {
    return alive[s] && !wdirty[s] && !key_gt(rd->tau_prim, rd->tau_idx, p, i);
}

__global__ void wup_setup_kernel(RoundDev* rd) {
    if (threadIdx.x != 0) return;
    rd->need = rd->live - rd->m;
    rd->rank = rd->need;  // the need-th largest key is the smallest one above w_up
    rd->done = 0;
    rd->len[0] = rd->len[1] = 0;
    rd->ncand = 0;
    rd->removed = 0;
    rd->overflow = 0;
}

// The key selection returns the lower boundary of the bin that holds the
// rank-th largest key, which counts the same keys but is not a key itself;
// w_up stays fixed while keys fall during an iteration, so it must be the
// key: the smallest live key at or above that boundary (two passes, primary
// then index).
__global__ void wup_tau_min_kernel(const u64* __restrict__ prim, const int4* __restrict__ pos,
                                   const uint8_t* __restrict__ alive, int64_t n,
                                   const RoundDev* rd, u64* tmin) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n || !alive[s]) return;
    u64 p = prim[s];
    if (!key_gt(rd->tau_prim, rd->tau_idx, p, pos[s].w)) atomicMin(tmin, p);
}

__global__ void wup_tau_min2_kernel(const u64* __restrict__ prim, const int4* __restrict__ pos,
                                    const uint8_t* __restrict__ alive, int64_t n,
                                    const RoundDev* rd, const u64* tmin, int* imin) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n || !alive[s]) return;
    u64 p = prim[s];
    int i = pos[s].w;
    if (p == *tmin && !key_gt(rd->tau_prim, rd->tau_idx, p, i)) atomicMin(imin, i);
}

__global__ void wup_tau_set_kernel(RoundDev* rd, const u64* tmin, const int* imin) {
    if (threadIdx.x != 0) return;
    rd->tau_prim = *tmin;
    rd->tau_idx = *imin;
}

__global__ void wup_round_reset_kernel(RoundDev* rd) {
    if (threadIdx.x != 0) return;
    rd->ncand = 0;
    rd->removed = 0;
}

__global__ void wup_mark_kernel(const BufView b, const uint8_t* __restrict__ alive,
                                const uint8_t* __restrict__ wdirty, int64_t n, int S, int k,
                                const RoundDev* rd, u64* mark_p) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    u64 ps = b.prim[s];
    if (!wup_cand(alive, wdirty, ps, b.pos[s].w, rd, s)) return;
    for (int i = 0; i < k; i++) {
        int x = b.nbr[s * S + i];
        if (x < 0) break;
        atomicMax(&mark_p[x], ps);
    }
}

__global__ void wup_mark2_kernel(const BufView b, const uint8_t* __restrict__ alive,
                                 const uint8_t* __restrict__ wdirty, int64_t n, int S, int k,
                                 const RoundDev* rd, const u64* __restrict__ mark_p, int* mark_i) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    u64 ps = b.prim[s];
    int is = b.pos[s].w;
    if (!wup_cand(alive, wdirty, ps, is, rd, s)) return;
    for (int i = 0; i < k; i++) {
        int x = b.nbr[s * S + i];
        if (x < 0) break;
        if (mark_p[x] == ps) atomicMax(&mark_i[x], is);
    }
}

__global__ void wup_pick_kernel(const BufView b, const uint8_t* __restrict__ alive,
                                const uint8_t* __restrict__ wdirty, int64_t n, int S, int k,
                                RoundDev* rd, const u64* __restrict__ mark_p,
                                const int* __restrict__ mark_i, uint8_t* pick) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool ok = false;
    if (s < n) {
        u64 ps = b.prim[s];
        int is = b.pos[s].w;
        if (wup_cand(alive, wdirty, ps, is, rd, s)) {
            ok = !key_gt(mark_p[s], mark_i[s], ps, is);
            for (int i = 0; i < k && ok; i++) {
                int x = b.nbr[s * S + i];
                if (x < 0) break;
                u64 px = b.prim[x];
                int ix = b.pos[x].w;
                if (wup_cand(alive, wdirty, px, ix, rd, x) && key_gt(px, ix, ps, is)) ok = false;
            }
        }
        pick[s] = ok ? 1 : 0;
    }
    block_add(&rd->removed, ok ? 1ull : 0ull);
}

__global__ void wup_remove_kernel(const uint8_t* __restrict__ pick, int64_t n, uint8_t* alive) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < n && pick[s]) alive[s] = 0;
}

// Removed points leave the stored lists (order kept); the cost is the sum of
// 1 / d^2 over the first k stored points left, nearest first, in binary64.
__global__ void wup_update_kernel(BufView b, const uint8_t* __restrict__ alive, int64_t n, int S,
                                  int k, uint8_t* wdirty, RoundDev* rd) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool upd = false;
    if (s < n && alive[s] && !wdirty[s]) {
        int ids[WUP_SMAX];
        int r = 0;
        bool dead = false;
#pragma unroll
        for (int i = 0; i < WUP_SMAX; i++) {
            ids[i] = -1;
            if (i < S) {
                int x = b.nbr[s * S + i];
                if (x >= 0) {
                    if (alive[x]) ids[r++] = x;
                    else dead = true;
                }
            }
        }
        if (dead) {
#pragma unroll
            for (int i = 0; i < WUP_SMAX; i++)
                if (i < S) b.nbr[s * S + i] = ids[i];
            if (r >= k) {
                int4 ps = b.pos[s];
                double c = 0.0;
                u64 dk = 0;
#pragma unroll
                for (int i = 0; i < WUP_SMAX; i++) {
                    if (i < k) {
                        u64 d2 = sqd(ps, b.pos[ids[i]]);
                        c = __dadd_rn(c, __ddiv_rn(1.0, (double)d2));
                        dk = d2;
                    }
                }
                b.prim[s] = key_prim_cost(c);
                b.rk2[s] = dk;
                upd = true;
            } else {
                wdirty[s] = 1;
            }
        }
    }
    block_add(&rd->tot_updated, upd ? 1ull : 0ull);
}

#define WGRID(n) (unsigned)(((n) + 255) / 256), 256

cudaError_t wup_launch_setup(RoundDev* rd, cudaStream_t st) {
    wup_setup_kernel<<<1, 32, 0, st>>>(rd);
    note_launch();
    return cudaGetLastError();
}

// w_up as a key: tau <- the smallest live key >= the selection's boundary.
// tw: one u64 and one int of device scratch.
cudaError_t wup_launch_exact_tau(const u64* prim, const int4* pos, const uint8_t* alive,
                                 int64_t n, RoundDev* rd, u64* tmin, int* imin,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(tmin, 0xff, sizeof(u64), st);
    if (!e) e = cudaMemsetAsync(imin, 0x7f, sizeof(int), st);
    if (e) return e;
    wup_tau_min_kernel<<<WGRID(n), 0, st>>>(prim, pos, alive, n, rd, tmin);
    wup_tau_min2_kernel<<<WGRID(n), 0, st>>>(prim, pos, alive, n, rd, tmin, imin);
    wup_tau_set_kernel<<<1, 32, 0, st>>>(rd, tmin, imin);
    for (int i = 0; i < 3; i++) note_launch();
    return cudaGetLastError();
}

// One removal round: marks, picks, removal, stored-list update.
cudaError_t wup_launch_round(const BufView& b, uint8_t* alive, uint8_t* wdirty, int64_t n, int S,
                             int k, RoundDev* rd, u64* mark_p, int* mark_i, uint8_t* pick,
                             cudaStream_t st) {
    if (S > WUP_SMAX || k > S || n <= 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(mark_p, 0, (size_t)n * sizeof(u64), st);
    if (!e) e = cudaMemsetAsync(mark_i, 0xff, (size_t)n * sizeof(int), st);
    if (e) return e;
    wup_round_reset_kernel<<<1, 32, 0, st>>>(rd);
    wup_mark_kernel<<<WGRID(n), 0, st>>>(b, alive, wdirty, n, S, k, rd, mark_p);
    wup_mark2_kernel<<<WGRID(n), 0, st>>>(b, alive, wdirty, n, S, k, rd, mark_p, mark_i);
    wup_pick_kernel<<<WGRID(n), 0, st>>>(b, alive, wdirty, n, S, k, rd, mark_p, mark_i, pick);
    wup_remove_kernel<<<WGRID(n), 0, st>>>(pick, n, alive);
    wup_update_kernel<<<WGRID(n), 0, st>>>(b, alive, n, S, k, wdirty, rd);
    for (int i = 0; i < 6; i++) note_launch();
    return cudaGetLastError();
}

}  // namespace pd
