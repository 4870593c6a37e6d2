// rounds_dev.cu -- removal rounds driven from device memory.
//
// One round is a fixed sequence of launches whose sizes never depend on
// counts computed in the round: the threshold tau comes from an on-device
// radix select, candidate / source / pair lists are appended with atomics and
// walked by grid-stride or persistent kernels, neighbour searches run over
// the leaf groups with a per-point flag, and the fixpoint runs a fixed number
// of sweeps.  The host reads the small RoundDev block once per round.
// The rules themselves (R2, A, B) are documented in rounds.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_internal.cuh"
#include "pd_kernels.h"

namespace pd {

#define FULLM 0xffffffffu
#define PERSIST_BLOCKS (device_sms() * 8)

// Appends s to list[*count ...] for every thread with want set, one atomic
// per block; every thread of the block must call it.
__device__ __forceinline__ void list_append(bool want, int s, int* count, int* list) {
    const int slot = block_append(want, count);
    if (want) list[slot] = s;
}

// ------------------------------------------------------------------ setup
__global__ void round_setup_kernel(RoundDev* rd) {
    if (threadIdx.x != 0) return;
    long long need = rd->live - rd->m;
    rd->need = need;
    long long rank = need;
    if (!rd->density_k1) {
        long long band_rank = (long long)(rd->band * (double)rd->live);
        long long quarter = (need + 3) / 4;
        rank = band_rank < quarter ? band_rank : quarter;
        if (rank < 1) rank = 1;
    }
    rd->rank = rank;
    rd->done = 0;
    rd->len[0] = rd->len[1] = 0;
    rd->ncand = rd->nslow = rd->nsrc = rd->npairs = rd->overflow = 0;
    rd->ndep = 0;
    rd->removed = 0;
    rd->cap_over = 0;
    rd->fix_unconverged = 0;
    for (int i = 0; i < PD_FIX_ITERS; i++) rd->changed[i] = 0;
}

__device__ __host__ inline double next_band(double band, double band_max, int band_mode,
                                            unsigned long long cap_over, long long ncand,
                                            unsigned long long removed) {
    bool shrink = cap_over != 0;
    double grow = 1.5;
    if (band_mode == 1) {
        double yield = ncand > 0 ? (double)removed / ncand : 1.0;
        shrink = shrink || yield < 0.5;
        grow = yield > 0.8 ? 1.25 : 1.0;
    }
    double b = shrink ? band * 0.5 : band * grow;
    if (b > band_max) b = band_max;
    if (b < 1e-7) b = 1e-7;
    return b;
}

__global__ void round_finish_kernel(RoundDev* rd) {
    if (threadIdx.x != 0) return;
    rd->live -= (long long)rd->removed;
    rd->tot_sources += (unsigned long long)rd->nsrc;
    // a held round (settled on the host) updates its band there, from the
    // points it finally removes: the band must not depend on whether the
    // device fixpoint happened to converge within its sweeps
    if (!rd->density_k1 && !(rd->overflow || rd->fix_unconverged)) {
        rd->band = next_band(rd->band, rd->band_max, rd->band_mode, rd->cap_over, rd->ncand,
                             rd->removed);
    }
}

double host_next_band(double band, double band_max, int band_mode, unsigned long long cap_over,
                      long long ncand, unsigned long long removed) {
    return next_band(band, band_max, band_mode, cap_over, ncand, removed);
}

// ------------------------------------------------------------------ selection
__device__ inline uint32_t sel_digit(u64 prim, int idx, int pass) {
    int lo = 84 - 12 * pass;
    uint32_t ui = (uint32_t)idx;
    if (lo >= 32) return (uint32_t)(prim >> (lo - 32)) & 0xfffu;
    if (lo + 12 <= 32) return (ui >> lo) & 0xfffu;
    int nlow = 32 - lo;
    return ((uint32_t)(prim << nlow) | (ui >> lo)) & 0xfffu;
}

// pass 0 reads every alive grid point; pass p > 0 reads the list compacted by
// pass p-1 (buffer (p-1)&1).
__global__ void seld_hist_kernel(const u64* __restrict__ prim, const uint8_t* __restrict__ alive,
                                 int64_t n, const u64* __restrict__ bp0, const int* __restrict__ bi0,
                                 const u64* __restrict__ bp1, const int* __restrict__ bi1,
                                 int pass, const RoundDev* rd, uint32_t* hist) {
    if (rd->done) return;
    __shared__ uint32_t h[4096];
    for (int x = threadIdx.x; x < 4096; x += blockDim.x) h[x] = 0;
    __syncthreads();
    const u64* lp = ((pass - 1) & 1) ? bp1 : bp0;
    const int* li = ((pass - 1) & 1) ? bi1 : bi0;
    int64_t len = pass ? (int64_t)rd->len[(pass - 1) & 1] : n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (pass) {
            atomicAdd(&h[sel_digit(lp[i], li[i], pass)], 1u);
        } else {
            if (!alive[i]) continue;
            atomicAdd(&h[(uint32_t)(prim[i] >> 52)], 1u);
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < 4096; x += blockDim.x)
        if (h[x]) atomicAdd(&hist[x], h[x]);
}

// One block of 256 threads: find the bin holding rank rd->rank (counted from
// the largest key), record the digit, and finish when the bin boundary is the
// exact threshold.  Clears the histogram for the next pass.
__global__ void seld_find_kernel(uint32_t* hist, int pass, RoundDev* rd) {
    __shared__ unsigned long long part[256];
    __shared__ int found_bin;
    __shared__ unsigned long long found_cum;
    if (rd->done) {
        for (int x = threadIdx.x; x < 4096; x += blockDim.x) hist[x] = 0;
        return;
    }
    int t = threadIdx.x;
    // thread t owns bins [4095 - 16t - 15, 4095 - 16t] (descending)
    unsigned long long s = 0;
    for (int j = 0; j < 16; j++) s += hist[4095 - 16 * t - j];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {  // inclusive scan over threads
        unsigned long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned long long before = t ? part[t - 1] : 0;
    long long r = rd->rank;
    if (t == 0) found_bin = -1;
    __syncthreads();
    if ((long long)before < r && (long long)part[t] >= r) {
        unsigned long long c = before;
        for (int j = 0; j < 16; j++) {
            int b = 4095 - 16 * t - j;
            if ((long long)(c + hist[b]) >= r) {
                found_bin = b;
                found_cum = c;
                break;
            }
            c += hist[b];
        }
    }
    __syncthreads();
    if (t == 0) {
        int b = found_bin;
        if (b < 0) {  // rank beyond the live count: cannot happen; stop selecting
            rd->done = 1;
            rd->overflow = 1;
        } else {
            rd->pre[pass] = (unsigned)b;
            unsigned long long hb = hist[b];
            bool exact = (long long)(found_cum + hb) == r || pass == 7;
            rd->rank = r - (long long)found_cum;
            if (exact) {
                unsigned __int128 v = 0;
                for (int p = 0; p < 8; p++) {
                    v <<= 12;
                    if (p <= pass) v |= rd->pre[p];
                }
                rd->tau_prim = (unsigned long long)(v >> 32);
                rd->tau_idx = (int)(uint32_t)v;
                rd->done = 1;
            }
            rd->len[pass & 1] = 0;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < 4096; x += blockDim.x) hist[x] = 0;
}

__global__ void seld_compact_kernel(const u64* __restrict__ prim, const int4* __restrict__ pos,
                                    const uint8_t* __restrict__ alive, int64_t n, u64* bp0, int* bi0,
                                    u64* bp1, int* bi1, int pass, RoundDev* rd) {
    if (rd->done) return;
    const u64* lp = ((pass - 1) & 1) ? bp1 : bp0;
    const int* li = ((pass - 1) & 1) ? bi1 : bi0;
    u64* op = (pass & 1) ? bp1 : bp0;
    int* oi = (pass & 1) ? bi1 : bi0;
    int64_t len = pass ? (int64_t)rd->len[(pass - 1) & 1] : n;
    uint32_t want = rd->pre[pass];
    // block-uniform trip count: the appends are aggregated per block
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < len;
         i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        u64 p = 0;
        int id = 0;
        bool take = false;
        if (i < len) {
            if (pass) {
                p = lp[i];
                id = li[i];
                take = sel_digit(p, id, pass) == want;
            } else if (alive[i]) {
                p = prim[i];
                take = (uint32_t)(p >> 52) == want;
                if (take) id = pos[i].w;
            }
        }
        const int slot = block_append(take, &rd->len[pass & 1]);
        if (take) {
            op[slot] = p;
            oi[slot] = id;
        }
    }
}

// ------------------------------------------------------------------ k = 1
__global__ void k1d_cand_kernel(const u64* __restrict__ prim, const int4* __restrict__ pos,
                                const uint8_t* __restrict__ alive, const int* __restrict__ nbr,
                                const int* __restrict__ nbr0,
                                const uint8_t* __restrict__ flg, int64_t n, int S, RoundDev* rd,
                                uint8_t* inP, int* cand, int* slow, int* dep) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool c = false, sl = false, dp = false;
    const bool in = s < n;
    const uint8_t al = in ? alive[s] : 0;
    const u64 ps = in ? prim[s] : 0;  // loaded beside the alive flag, not after it
    if (al) {
        u64 tp = rd->tau_prim;  // packed batch: the least threshold over the scans
        if (ps >= tp) {  // below the threshold on the primary: no index needed
            int ti = rd->tau_idx;
            int is;
            if (rd->seg) {  // packed batch: the threshold of the point's own scan
                const int4 p4 = pos[s];
                is = p4.w;
                round_tau(rd, p4, tp, ti);
            } else {
                is = pos[s].w;
            }
            if (!key_gt(tp, ti, ps, is)) {
                const uint8_t fl = flg[s];
                if (fl & 2) {
                    sl = true;
                } else {
                    // the shell (points at the nearest distance) is the first
                    // fl >> 2 stored neighbours; none: a lone point
                    const int shell = fl >> 2;
                    bool ok = shell == 0, larger = false;
                    for (int i = 0; i < shell; i++) {
                        const int x = i == 0 && nbr0 ? nbr0[s] : nbr[s * S + i];
                        const int ix = pos[x].w;
                        if (key_gt(ps, is, prim[x], ix)) ok = true;
                        if (ix > is) larger = true;
                    }
                    c = ok;
                    dp = ok && larger;
                }
            }
        }
    }
    // list appends aggregated per block (every thread reaches them)
    if (c) inP[s] = 1;
    list_append(c, (int)s, &rd->ncand, cand);
    list_append(sl, (int)s, &rd->nslow, slow);
    list_append(dp, (int)s, &rd->ndep, dep);
}

// overflowing shells: accept iff every live point at distance d1 has a
// smaller key (grid-stride over the slow list)
__global__ void k1d_slow_kernel(GridView g, const u64* __restrict__ prim,
                                const uint8_t* __restrict__ alive, const u64* __restrict__ rk2,
                                const int* __restrict__ slow, RoundDev* rd, uint8_t* inP,
                                int* cand) {
    int ns = rd->nslow;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ns; t += gridDim.x * blockDim.x) {
        int s = slow[t];
        int4 qp = g.pos[s];
        u64 r2 = rk2[s];
        u64 ps = prim[s];
        int ux = qp.x - g.origin.x, uy = qp.y - g.origin.y, uz = qp.z - g.origin.z;
        u64 c0 = g.code[s];
        bool ok = true;
        for (int L = g.leaf[s]; L <= g.B; L++) {
            int cx = 0, cy = 0, cz = 0;
            if (L < g.B) {
                cx = (int)compact3(c0 >> (3 * L));
                cy = (int)compact3(c0 >> (3 * L + 1));
                cz = (int)compact3(c0 >> (3 * L + 2));
            }
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
            bool covered = L >= g.B || best < 0 || r2 < (u64)best * (u64)best;
            if (!covered) continue;
            for (int o = 0; o < 27 && ok; o++) {
                int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
                uint32_t b, e;
                int lvl;
                if (!resolve_cell(g, L, cx + dx, cy + dy, cz + dz, b, e, &lvl)) continue;
                for (uint32_t j = b; j < e && ok; j++) {
                    if ((int)j == s || !alive[j]) continue;
                    int4 v = g.pos[j];
                    long long dx2 = v.x - qp.x, dy2 = v.y - qp.y, dz2 = v.z - qp.z;
                    u64 d2 = (u64)(dx2 * dx2 + dy2 * dy2 + dz2 * dz2);
                    if (d2 == r2 && key_gt(prim[j], v.w, ps, qp.w)) ok = false;
                }
            }
            break;
        }
        if (ok) {
            inP[s] = 1;
            cand[atomicAdd(&rd->ncand, 1)] = s;
        }
    }
}

__global__ void k1d_fix_kernel(const int* __restrict__ cand, const int4* __restrict__ pos,
                               const int* __restrict__ nbr, const uint8_t* __restrict__ flg, int S,
                               const uint8_t* __restrict__ inP, uint8_t* rej, int iter,
                               RoundDev* rd) {
    if (iter > 0 && !rd->changed[iter - 1]) return;
    int nc = rd->ndep;  // cand: the dep list (only its members can be rejected)
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += gridDim.x * blockDim.x) {
        int s = cand[t];
        if (rej[s]) continue;
        int is = pos[s].w;
        int shell = flg[s] >> 2;
        for (int i = 0; i < shell; i++) {
            int x = nbr[(int64_t)s * S + i];
            if (pos[x].w > is && (!inP[x] || rej[x])) {
                rej[s] = 1;
                rd->changed[iter] = 1;
                break;
            }
        }
    }
}

__global__ void kkd_accept_kernel(const uint8_t* __restrict__ fq_flag, const u64* __restrict__ prim,
                                  const u64* __restrict__ fprim, int64_t n, RoundDev* rd,
                                  uint8_t* inP, int* cand) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool acc = s < n && fq_flag[s] && fprim[s] == prim[s];
    if (acc) inP[s] = 1;
    list_append(acc, (int)s, &rd->ncand, cand);
}

__global__ void pairs_fix_kernel(const int2* __restrict__ pairs, int pair_cap, const uint8_t* inP,
                                 uint8_t* rej, int iter, RoundDev* rd) {
    if (iter > 0 && !rd->changed[iter - 1]) return;
    int np = min(rd->npairs, pair_cap);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < np; t += gridDim.x * blockDim.x) {
        int2 pr = pairs[t];
        if (rej[pr.y]) continue;
        if (!inP[pr.x] || rej[pr.x]) {
            rej[pr.y] = 1;
            rd->changed[iter] = 1;
        }
    }
}

// ------------------------------------------------------------------ removal
// Removes the accepted candidates unless the round must be settled on the
// host (danger overflow, or a fixpoint that did not converge in the fixed
// number of sweeps); candidate marks are cleared in the normal case.
__global__ void removed_kernel(const int* __restrict__ cand, uint8_t* inP, uint8_t* rej,
                               uint8_t* alive, RoundDev* rd) {
    __shared__ int hold;
    if (threadIdx.x == 0) {
        int fi = rd->fix_iters;
        if (fi < 1 || fi > PD_FIX_ITERS) fi = PD_FIX_ITERS;
        const int last = rd->changed[fi - 1];
        hold = rd->overflow || last;
        if (hold && blockIdx.x == 0) rd->fix_unconverged = last;
    }
    __syncthreads();
    if (hold) return;
    int nc = rd->ncand;
    unsigned c = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += gridDim.x * blockDim.x) {
        int s = cand[t];
        if (inP[s] && !rej[s]) {
            alive[s] = 0;
            c++;
        }
        inP[s] = 0;
        rej[s] = 0;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULLM, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&rd->removed, (unsigned long long)c);
}

__global__ void dirtyd_kernel(const uint8_t* __restrict__ alive, const int* __restrict__ nbr,
                              int64_t n, int S, int kchk, uint8_t* dirty, RoundDev* rd) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool d = false;
    if (s < n) {
        if (alive[s]) {
            for (int i = 0; i < kchk; i++) {
                int x = nbr[s * S + i];
                if (x >= 0 && !alive[x]) d = true;
            }
        }
        dirty[s] = d ? 1 : 0;
    }
    block_add(&rd->tot_requery, d ? 1ull : 0ull);
}

// ------------------------------------------------------------------ k = 1 buffer
// k = 1 density cost: every point stores its S nearest live points exactly,
// with the horizon h = the S-th squared distance at search time (any live
// point not stored lies at d^2 >= h; h = ~0 when all live points were
// stored).  After removals, the first live stored entry is the new nearest;
// its shell (the stored entries at that distance) is complete when that
// distance is below h, and the key follows without a search.  Otherwise, or
// when no stored entry is left, the point is searched again.
#define K1_SMAX 8

// 40 registers, 6 blocks of 256 per SM: the update waits on dependent loads,
// and more threads in flight measured faster (rules of the 100M-point scan
// 52.9 -> 51.5 ms)
__global__ void __launch_bounds__(256, 6) k1d_update_kernel(BufView b, const uint8_t* __restrict__ alive, int64_t n, int S,
                                  uint8_t* dirty, RoundDev* rd) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool upd = false, req = false;
    if (s < n) {
        uint8_t dv = 0;
        // only a removed shell member changes the key or the shell; removed
        // entries past the shell stay stored (stale) until the shell changes
        // the point's flag, shell size and first entry are loaded together
        // (the first entry from its coalesced copy: most shells hold one
        // point), so that only the entry's alive flag waits on them
        bool shell_hit = false;
        const uint8_t al = alive[s];
        const int shell = b.flg[s] >> 2;
        const int x0 = b.nbr0 ? b.nbr0[s] : b.nbr[s * S];
        if (al && shell > 0) {
            shell_hit = !alive[x0];
            for (int i = 1; i < shell && !shell_hit; i++) shell_hit = !alive[b.nbr[s * S + i]];
        }
        if (shell_hit) {
            int ids[K1_SMAX];
            int r = 0;
            bool dead = false;
#pragma unroll
            for (int i = 0; i < K1_SMAX; i++) {
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
                u64 h = b.hz[s];
                u64 d0 = ~0ull;
                int shell = 0;
                if (r > 0) {
                    int4 ps = b.pos[s];
                    d0 = sqd(ps, b.pos[ids[0]]);
                    shell = 1;
#pragma unroll
                    for (int i = 1; i < K1_SMAX; i++)
                        if (i < r && sqd(ps, b.pos[ids[i]]) == d0) shell++;
                }
                if (r > 0 && (h == ~0ull || d0 < h)) {
                    b.prim[s] = key_prim_d2(d0);
                    b.rk2[s] = d0;
                    b.flg[s] = (uint8_t)((shell >= 2 ? 1 : 0) | (shell << 2));
#pragma unroll
                    for (int i = 0; i < K1_SMAX; i++)
                        if (i < S) b.nbr[s * S + i] = ids[i];
                    if (b.nbr0) b.nbr0[s] = ids[0];
                    upd = true;
                } else {
                    dv = 1;
                    req = true;
                }
            }
        }
        dirty[s] = dv;
    }
    block_add2(&rd->tot_updated, upd ? 1ull : 0ull, &rd->tot_requery, req ? 1ull : 0ull);
}

// ------------------------------------------------------------------ k+b buffer
// Every point stores its S nearest live points exactly, plus the horizon h =
// the S-th squared distance when they were searched: any point not stored
// lies at d^2 >= h.  After removals the live stored entries, in order, are
// still the nearest live points, so as long as k of them remain the new cost
// follows without a search (the paper's extended k+b neighbourhood, section
// "Sub-sampling algorithm").  Fewer than k left: the point is searched again.
#define UPD_SMAX 8

// Held to 48 registers for 5 blocks per SM: the loop over the stored entries
// waits on dependent loads, and the recomputation that spills runs only for
// points that lost a neighbour.
__global__ void __launch_bounds__(256, 5) kkd_update_kernel(BufView b, const uint8_t* __restrict__ alive, int64_t n, int S,
                                  int k, uint8_t* dirty, RoundDev* rd) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool upd = false, req = false;
    if (s < n) {
        uint8_t dv = 0;
        if (alive[s]) {
            int ids[UPD_SMAX];
            int r = 0;
            bool dead = false;
#pragma unroll
            for (int i = 0; i < UPD_SMAX; i++) {
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
                if (r >= k) {
                    int4 ps = b.pos[s];
                    u64 h = b.hz[s];
                    double c = 0.0;
                    u64 dk = 0, dk1 = ~0ull;
#pragma unroll
                    for (int i = 0; i < UPD_SMAX; i++) {
                        if (i < r && i <= k) {
                            u64 d2 = sqd(ps, b.pos[ids[i]]);
                            if (i < k) {
                                double w = term_weight(b.term, b.weight, b.rgb, b.nrm, (int)s, ids[i]);
                                c = __dadd_rn(c, __ddiv_rn(w, (double)d2));
                                dk = d2;
                            } else {
                                dk1 = d2;
                            }
                        }
                    }
                    bool tie = (r > k && dk1 == dk) || (h != ~0ull && dk == h);
                    b.prim[s] = key_prim_cost(c);
                    b.rk2[s] = dk;
                    b.flg[s] = tie ? 1 : 0;
#pragma unroll
                    for (int i = 0; i < UPD_SMAX; i++)
                        if (i < S) b.nbr[s * S + i] = ids[i];
                    upd = true;
                } else {
                    dv = 1;
                    req = true;
                }
            }
        }
        dirty[s] = dv;
    }
    block_add2(&rd->tot_updated, upd ? 1ull : 0ull, &rd->tot_requery, req ? 1ull : 0ull);
}

// Candidate test (k >= 2) using the stored buffer where it suffices:
//   (A) the cost over smaller keys is the cost over the first k stored entries
//       of smaller key, when k of them are stored (any unstored point is at
//       least as far as every stored one); otherwise a filtered search.
//   lam (danger sources): the k-th stored squared distance of key below tau,
//       when k such entries are stored; otherwise a search.
__global__ void kkd_cand2_kernel(BufView b, const uint8_t* __restrict__ alive, int64_t n, int S,
                                 int k, RoundDev* rd, uint8_t* inP, int* cand, uint8_t* fq_flag,
                                 uint8_t* lq_flag, u64* lam, int* src) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool fq = false, lq = false, isc = false, iss = false;
    if (s < n) {
        if (alive[s]) {
            u64 ps = b.prim[s];
            int4 qs = b.pos[s];
            int is = qs.w;
            u64 tp = rd->tau_prim;
            int ti = rd->tau_idx;
            // packed batch: tp is the least threshold over the scans; a point
            // above it takes its own scan's threshold
            if (rd->seg && ps >= tp) round_tau(rd, qs, tp, ti);
            if (!key_gt(tp, ti, ps, is)) {
                uint8_t fl = b.flg[s];
                bool lower = !(fl & 1);
                bool band_nbr = (fl & 1) != 0;
                int nfound = 0;
                for (int i = 0; i < S; i++) {
                    int x = b.nbr[s * S + i];
                    if (x < 0) continue;
                    nfound++;
                    if (i >= k) continue;
                    u64 px = b.prim[x];
                    int ix = b.pos[x].w;
                    if (key_gt(px, ix, ps, is)) lower = false;
                    if (!key_gt(tp, ti, px, ix)) band_nbr = true;
                }
                if (nfound < k) band_nbr = true;
                bool acc = lower;
                if (!acc) {
                    // cost over the stored entries of smaller key
                    double c = 0.0;
                    int cnt = 0;
                    for (int i = 0; i < S && cnt < k; i++) {
                        int x = b.nbr[s * S + i];
                        if (x < 0) continue;
                        int4 px4 = b.pos[x];
                        if (!key_gt(ps, is, b.prim[x], px4.w)) continue;
                        double w = term_weight(b.term, b.weight, b.rgb, b.nrm, (int)s, x);
                        c = __dadd_rn(c, __ddiv_rn(w, (double)sqd(qs, px4)));
                        cnt++;
                    }
                    if (cnt >= k) acc = key_prim_cost(c) == ps;
                    else fq = true;
                }
                if (acc) {
                    inP[s] = 1;
                    isc = true;
                }
                if (key_gt(ps, is, tp, ti) && band_nbr) {
                    // danger source: lam from the stored entries of key below tau
                    int cnt = 0;
                    u64 l = ~0ull;
                    for (int i = 0; i < S && cnt < k; i++) {
                        int x = b.nbr[s * S + i];
                        if (x < 0) continue;
                        int4 px4 = b.pos[x];
                        if (!key_gt(tp, ti, b.prim[x], px4.w)) continue;
                        l = sqd(qs, px4);
                        cnt++;
                    }
                    if (cnt >= k) lam[s] = l;
                    else lq = true;
                    iss = true;
                }
            }
        }
        fq_flag[s] = fq ? 1 : 0;
        lq_flag[s] = lq ? 1 : 0;
    }
    list_append(isc, (int)s, &rd->ncand, cand);
    list_append(iss, (int)s, &rd->nsrc, src);
    block_add2(&rd->tot_filtered, fq ? 1ull : 0ull, &rd->tot_lambda, lq ? 1ull : 0ull);
}

// ------------------------------------------------------------------ launchers
#define GRID1(n) (unsigned)(((n) + 255) / 256), 256

cudaError_t round_launch_setup(RoundDev* rd, cudaStream_t st) {
    round_setup_kernel<<<1, 32, 0, st>>>(rd); note_launch();
    return cudaGetLastError();
}
cudaError_t round_launch_finish(RoundDev* rd, cudaStream_t st) {
    round_finish_kernel<<<1, 32, 0, st>>>(rd); note_launch();
    return cudaGetLastError();
}

cudaError_t round_launch_select(const u64* prim, const int4* pos, const uint8_t* alive, int64_t n,
                                SelBuffers& b, RoundDev* rd, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > device_sms() * 4) blocks = device_sms() * 4;
    if (blocks < 1) blocks = 1;
    for (int pass = 0; pass < 8; pass++) {
        seld_hist_kernel<<<blocks, 256, 0, st>>>(prim, alive, n, b.p[0], b.i[0], b.p[1], b.i[1],
                                                 pass, rd, b.hist); note_launch();
        seld_find_kernel<<<1, 256, 0, st>>>(b.hist, pass, rd); note_launch();
        if (pass < 7) {
            seld_compact_kernel<<<blocks, 256, 0, st>>>(prim, pos, alive, n, b.p[0], b.i[0],
                                                        b.p[1], b.i[1], pass, rd); note_launch();
        }
    }
    return cudaGetLastError();
}

cudaError_t round_launch_k1(const GridView& g, const u64* prim, const uint8_t* alive,
                            const int* nbr, const int* nbr0, const uint8_t* flg, const u64* rk2,
                            int64_t n, int S, RoundDev* rd, uint8_t* inP, uint8_t* rej, int* cand,
                            int* slow, int* dep, int fix_iters, cudaStream_t st) {
    if (fix_iters < 1 || fix_iters > PD_FIX_ITERS) return cudaErrorInvalidValue;
    k1d_cand_kernel<<<GRID1(n), 0, st>>>(prim, g.pos, alive, nbr, nbr0, flg, n, S, rd, inP, cand,
                                         slow, dep); note_launch();
    k1d_slow_kernel<<<PERSIST_BLOCKS, 128, 0, st>>>(g, prim, alive, rk2, slow, rd, inP, cand); note_launch();
    for (int it = 0; it < fix_iters; it++) {
        k1d_fix_kernel<<<PERSIST_BLOCKS, 256, 0, st>>>(dep, g.pos, nbr, flg, S, inP, rej, it, rd); note_launch();
    }
    return cudaGetLastError();
}

cudaError_t round_launch_kk_accept(const uint8_t* fq_flag, const u64* prim, const u64* fprim,
                                   int64_t n, RoundDev* rd, uint8_t* inP, int* cand,
                                   cudaStream_t st) {
    kkd_accept_kernel<<<GRID1(n), 0, st>>>(fq_flag, prim, fprim, n, rd, inP, cand); note_launch();
    return cudaGetLastError();
}

cudaError_t round_launch_pairs_fix(const int2* pairs, int pair_cap, const uint8_t* inP,
                                   uint8_t* rej, RoundDev* rd, cudaStream_t st) {
    for (int it = 0; it < PD_FIX_ITERS_KK; it++) {
        pairs_fix_kernel<<<PERSIST_BLOCKS, 256, 0, st>>>(pairs, pair_cap, inP, rej, it, rd); note_launch();
    }
    return cudaGetLastError();
}

cudaError_t round_launch_remove(const int* cand, uint8_t* inP, uint8_t* rej, uint8_t* alive,
                                RoundDev* rd, cudaStream_t st) {
    removed_kernel<<<PERSIST_BLOCKS, 256, 0, st>>>(cand, inP, rej, alive, rd); note_launch();
    return cudaGetLastError();
}

cudaError_t round_launch_dirty(const uint8_t* alive, const int* nbr, int64_t n, int S, int kchk,
                               uint8_t* dirty, RoundDev* rd, cudaStream_t st) {
    dirtyd_kernel<<<GRID1(n), 0, st>>>(alive, nbr, n, S, kchk, dirty, rd); note_launch();
    return cudaGetLastError();
}

}  // namespace pd

namespace pd {
cudaError_t round_launch_k1_update(const BufView& b, const uint8_t* alive, int64_t n, int S,
                                   uint8_t* dirty, RoundDev* rd, cudaStream_t st) {
    if (S > K1_SMAX) return cudaErrorInvalidValue;
    k1d_update_kernel<<<GRID1(n), 0, st>>>(b, alive, n, S, dirty, rd); note_launch();
    return cudaGetLastError();
}
cudaError_t round_launch_kk_update(const BufView& b, const uint8_t* alive, int64_t n, int S, int k,
                                   uint8_t* dirty, RoundDev* rd, cudaStream_t st) {
    kkd_update_kernel<<<GRID1(n), 0, st>>>(b, alive, n, S, k, dirty, rd); note_launch();
    return cudaGetLastError();
}
cudaError_t round_launch_kk_cand2(const BufView& b, const uint8_t* alive, int64_t n, int S, int k,
                                  RoundDev* rd, uint8_t* inP, int* cand, uint8_t* fq_flag,
                                  uint8_t* lq_flag, u64* lam, int* src, cudaStream_t st) {
    kkd_cand2_kernel<<<GRID1(n), 0, st>>>(b, alive, n, S, k, rd, inP, cand, fq_flag, lq_flag, lam,
                                          src); note_launch();
    return cudaGetLastError();
}
}  // namespace pd
