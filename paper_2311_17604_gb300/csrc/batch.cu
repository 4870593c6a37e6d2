// batch.cu -- packed batches: many independent scans decimated in one grid.
//
// The scans of a batch are moved into disjoint aligned tiles (scan i into
// the tile whose Morton index is i) and decimated as one cloud: one grid
// build, one first neighbour pass and one sequence of round launches for all
// of them.  Nothing on the neighbour path knows about scans: tiles are so far
// apart that every neighbour a search returns lies in the query's own scan.
// Only the removal threshold of a round (rule R2: a point may go only if its
// key is among the `need` largest of its cloud) is per scan, so it is
// selected here per scan, with the same 12-bit radix select the one-scan path
// uses, run over work items of PD_SEG_CHUNK grid positions that never cross
// a scan boundary.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_internal.cuh"
#include "pd_kernels.h"

namespace pd {

#define BATCH_BLOCKS (device_sms() * 8)

__device__ __forceinline__ int pack_scan_of(const PackScan* sc, int nsc, int w) {
    int lo = 0, hi = nsc - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sc[mid].chunk0 <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ packing
__global__ void pack_bbox_kernel(PackScan* sc, int nsc, int nchunks) {
    __shared__ int s_i;
    __shared__ long long s_lo, s_hi;
    __shared__ int red[6][32];
    for (int w = blockIdx.x; w < nchunks; w += gridDim.x) {
        if (threadIdx.x == 0) {
            int i = pack_scan_of(sc, nsc, w);
            long long lo = (long long)(w - sc[i].chunk0) * PD_SEG_CHUNK;
            long long hi = lo + PD_SEG_CHUNK < sc[i].n ? lo + PD_SEG_CHUNK : sc[i].n;
            s_i = i;
            s_lo = lo;
            s_hi = hi;
        }
        __syncthreads();
        const int i = s_i;
        const int32_t* x = sc[i].xyz;
        int v[6] = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000,
                    (int)0x80000000};
        for (long long j = s_lo + threadIdx.x; j < s_hi; j += blockDim.x) {
            for (int a = 0; a < 3; a++) {
                int c = x[3 * j + a];
                v[a] = c < v[a] ? c : v[a];
                v[3 + a] = c > v[3 + a] ? c : v[3 + a];
            }
        }
        for (int o = 16; o; o >>= 1)
            for (int a = 0; a < 6; a++) {
                int u = __shfl_xor_sync(0xffffffffu, v[a], o);
                v[a] = a < 3 ? (u < v[a] ? u : v[a]) : (u > v[a] ? u : v[a]);
            }
        const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0)
            for (int a = 0; a < 6; a++) red[a][wp] = v[a];
        __syncthreads();
        if (threadIdx.x < 6) {
            const int a = threadIdx.x;
            int r = red[a][0];
            for (int q = 1; q < (int)(blockDim.x >> 5); q++)
                r = a < 3 ? (red[a][q] < r ? red[a][q] : r) : (red[a][q] > r ? red[a][q] : r);
            if (a < 3) atomicMin(&sc[i].bb[a], r);
            else atomicMax(&sc[i].bb[a], r);
        }
        __syncthreads();
    }
}

__global__ void pack_copy_kernel(const PackScan* sc, int nsc, int nchunks, int32_t* out_xyz,
                                 uint8_t* out_rgb, float* out_nrm) {
    for (int w = blockIdx.x; w < nchunks; w += gridDim.x) {
        const int i = pack_scan_of(sc, nsc, w);  // uniform over the block
        const PackScan& s = sc[i];
        const long long lo = (long long)(w - s.chunk0) * PD_SEG_CHUNK;
        const long long hi = lo + PD_SEG_CHUNK < s.n ? lo + PD_SEG_CHUNK : s.n;
        for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
            const long long o = s.off + j;
            out_xyz[3 * o + 0] = s.xyz[3 * j + 0] + s.ox;
            out_xyz[3 * o + 1] = s.xyz[3 * j + 1] + s.oy;
            out_xyz[3 * o + 2] = s.xyz[3 * j + 2] + s.oz;
            if (out_rgb) {
                out_rgb[3 * o + 0] = s.rgb[3 * j + 0];
                out_rgb[3 * o + 1] = s.rgb[3 * j + 1];
                out_rgb[3 * o + 2] = s.rgb[3 * j + 2];
            }
            if (out_nrm) {
                out_nrm[3 * o + 0] = s.nrm[3 * j + 0];
                out_nrm[3 * o + 1] = s.nrm[3 * j + 1];
                out_nrm[3 * o + 2] = s.nrm[3 * j + 2];
            }
        }
    }
}

__global__ void pack_unpack_kernel(const PackScan* sc, int nsc, int nchunks,
                                   const uint8_t* __restrict__ keep) {
    for (int w = blockIdx.x; w < nchunks; w += gridDim.x) {
        const int i = pack_scan_of(sc, nsc, w);
        const PackScan& s = sc[i];
        const long long lo = (long long)(w - s.chunk0) * PD_SEG_CHUNK;
        const long long hi = lo + PD_SEG_CHUNK < s.n ? lo + PD_SEG_CHUNK : s.n;
        for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) s.keep[j] = keep[s.off + j];
    }
}

// ------------------------------------------------------------------ scan ranges
// b of scan i = the first grid position whose tile index is >= i (tile
// indices never decrease along the Morton order).
__global__ void seg_ranges_kernel(const int4* __restrict__ pos, int64_t ng, SegDev* seg,
                                  int nseg, int shift) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nseg) return;
    long long lo = 0, hi = ng;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (seg_of(pos[mid], shift) >= i) hi = mid;
        else lo = mid + 1;
    }
    if (i < nseg) seg[i].b = (int)lo;
    if (i > 0) seg[i - 1].e = (int)lo;
}

// chunk0[i] = work items of the scans before i, items[w] = the scan of work
// item w; one block of 1024 threads.
__global__ void seg_chunks_kernel(const SegDev* seg, int nseg, int* chunk0, int* items) {
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (nseg + 1023) / 1024;
    int loc[PD_SEG_MAX / 1024];
    int sum = 0;
    for (int j = 0; j < per; j++) {
        const int i = t * per + j;
        int c = 0;
        if (i < nseg) c = (seg[i].e - seg[i].b + PD_SEG_CHUNK - 1) / PD_SEG_CHUNK;
        loc[j] = c;
        sum += c;
    }
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int acc = t ? part[t - 1] : 0;
    for (int j = 0; j < per; j++) {
        const int i = t * per + j;
        if (i < nseg) {
            chunk0[i] = acc;
            for (int w = 0; w < loc[j]; w++) items[acc + w] = i;
        }
        acc += loc[j];
    }
    if (t == 1023) chunk0[nseg] = part[1023];
}

// ------------------------------------------------------------------ per-scan selection
__device__ __forceinline__ uint32_t seg_digit(u64 prim, int idx, int pass) {
    int lo = 84 - 12 * pass;
    uint32_t ui = (uint32_t)idx;
    if (lo >= 32) return (uint32_t)(prim >> (lo - 32)) & 0xfffu;
    if (lo + 12 <= 32) return (ui >> lo) & 0xfffu;
    int nlow = 32 - lo;
    return ((uint32_t)(prim << nlow) | (ui >> lo)) & 0xfffu;
}

__global__ void seg_setup_kernel(RoundDev* rd) {
    if (threadIdx.x != 0) return;
    rd->tau_prim = ~0ull;  // least threshold over the scans, lowered by seg_find
    rd->tau_idx = 0;
    rd->done = 1;          // the one-scan selection kernels do nothing
}

// The range of work item w in pass `pass`: grid positions (pass 0) or the
// scan's segment of the previous pass's list.  Empty for finished scans.
__device__ __forceinline__ void seg_item(const SegDev* seg, const int* chunk0, const int* items,
                                         int w, int pass, int& i, long long& lo, long long& hi) {
    i = items[w];
    const SegDev& s = seg[i];
    const long long off = (long long)(w - chunk0[i]) * PD_SEG_CHUNK;
    if (pass == 0) {
        lo = s.b + off;
        hi = lo + PD_SEG_CHUNK < s.e ? lo + PD_SEG_CHUNK : s.e;
    } else if (s.done) {
        lo = hi = 0;
    } else {
        const long long len = s.len[(pass - 1) & 1];
        lo = s.b + off;
        hi = s.b + (off + PD_SEG_CHUNK < len ? off + PD_SEG_CHUNK : len);
    }
}

__global__ void seg_hist_kernel(const u64* __restrict__ prim, const uint8_t* __restrict__ alive,
                                const u64* __restrict__ bp0, const int* __restrict__ bi0,
                                const u64* __restrict__ bp1, const int* __restrict__ bi1,
                                int pass, const SegDev* seg, const int* chunk0,
                                const int* items, int nseg, uint32_t* hist) {
    __shared__ uint32_t h[4096];
    __shared__ int s_i;
    __shared__ long long s_lo, s_hi;
    const u64* lp = ((pass - 1) & 1) ? bp1 : bp0;
    const int* li = ((pass - 1) & 1) ? bi1 : bi0;
    const int nch = chunk0[nseg];
    for (int w = blockIdx.x; w < nch; w += gridDim.x) {
        if (threadIdx.x == 0) {
            int i;
            long long lo, hi;
            seg_item(seg, chunk0, items, w, pass, i, lo, hi);
            s_i = i;
            s_lo = lo;
            s_hi = hi;
        }
        __syncthreads();
        const long long lo = s_lo, hi = s_hi;
        const int i = s_i;
        if (hi > lo) {  // uniform over the block
            for (int x = threadIdx.x; x < 4096; x += blockDim.x) h[x] = 0;
            __syncthreads();
            for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
                if (pass) {
                    atomicAdd(&h[seg_digit(lp[j], li[j], pass)], 1u);
                } else if (alive[j]) {
                    atomicAdd(&h[(uint32_t)(prim[j] >> 52)], 1u);
                }
            }
            __syncthreads();
            uint32_t* row = hist + (size_t)i * 4096;
            for (int x = threadIdx.x; x < 4096; x += blockDim.x)
                if (h[x]) atomicAdd(&row[x], h[x]);
        }
        __syncthreads();
    }
}

// One block of 256 threads per scan: the bin holding the scan's rank (from
// its largest key), as in the one-scan selection.  Pass 0 also counts the
// scan's live points and sets its need and rank.  Clears the scan's row.
__global__ void seg_find_kernel(uint32_t* hist, int pass, RoundDev* rd, SegDev* seg) {
    __shared__ unsigned long long part[256];
    __shared__ int found_bin;
    __shared__ unsigned long long found_cum;
    const int i = blockIdx.x;
    SegDev& S = seg[i];
    if (pass > 0 && S.done) return;  // its row was not touched
    uint32_t* row = hist + (size_t)i * 4096;
    const int t = threadIdx.x;
    unsigned long long s = 0;
    for (int j = 0; j < 16; j++) s += row[4095 - 16 * t - j];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        unsigned long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long r;
    if (pass == 0) {
        const long long live = (long long)part[255];
        const long long need = live - S.m;
        long long rank = need;
        if (rd->seg_rank_one) {
            rank = 1;
        } else if (!rd->density_k1) {
            long long band_rank = (long long)(rd->band * (double)live);
            long long quarter = (need + 3) / 4;
            rank = band_rank < quarter ? band_rank : quarter;
            if (rank < 1) rank = 1;
        }
        if (t == 0) {
            S.live = live;
            S.need = need;
            S.done = 0;
            S.len[0] = S.len[1] = 0;
        }
        if (need <= 0) {  // target reached: nothing of this scan goes this round
            if (t == 0) {
                S.rank = 0;
                S.done = 1;
                S.tau_prim = ~0ull;
                S.tau_idx = 0x7fffffff;
            }
            __syncthreads();
            for (int x = t; x < 4096; x += blockDim.x) row[x] = 0;
            return;
        }
        r = rank;
    } else {
        r = S.rank;
    }
    unsigned long long before = t ? part[t - 1] : 0;
    if (t == 0) found_bin = -1;
    __syncthreads();
    if ((long long)before < r && (long long)part[t] >= r) {
        unsigned long long c = before;
        for (int j = 0; j < 16; j++) {
            int b = 4095 - 16 * t - j;
            if ((long long)(c + row[b]) >= r) {
                found_bin = b;
                found_cum = c;
                break;
            }
            c += row[b];
        }
    }
    __syncthreads();
    if (t == 0) {
        int b = found_bin;
        if (b < 0) {  // rank beyond the live count: cannot happen; nothing goes
            S.done = 1;
            S.tau_prim = ~0ull;
            S.tau_idx = 0x7fffffff;
            rd->overflow = 1;
        } else {
            S.pre[pass] = (unsigned)b;
            unsigned long long hb = row[b];
            bool exact = (long long)(found_cum + hb) == r || pass == 7;
            S.rank = r - (long long)found_cum;
            if (exact) {
                unsigned __int128 v = 0;
                for (int p = 0; p < 8; p++) {
                    v <<= 12;
                    if (p <= pass) v |= S.pre[p];
                }
                S.tau_prim = (unsigned long long)(v >> 32);
                S.tau_idx = (int)(uint32_t)v;
                S.done = 1;
                atomicMin(&rd->tau_prim, S.tau_prim);
            }
            S.len[pass & 1] = 0;
        }
    }
    __syncthreads();
    for (int x = t; x < 4096; x += blockDim.x) row[x] = 0;
}

__global__ void seg_compact_kernel(const u64* __restrict__ prim, const int4* __restrict__ pos,
                                   const uint8_t* __restrict__ alive, u64* bp0, int* bi0,
                                   u64* bp1, int* bi1, int pass, SegDev* seg, const int* chunk0,
                                   const int* items, int nseg) {
    __shared__ int s_i;
    __shared__ long long s_lo, s_hi;
    const u64* lp = ((pass - 1) & 1) ? bp1 : bp0;
    const int* li = ((pass - 1) & 1) ? bi1 : bi0;
    u64* op = (pass & 1) ? bp1 : bp0;
    int* oi = (pass & 1) ? bi1 : bi0;
    const int nch = chunk0[nseg];
    for (int w = blockIdx.x; w < nch; w += gridDim.x) {
        if (threadIdx.x == 0) {
            int i;
            long long lo, hi;
            seg_item(seg, chunk0, items, w, pass, i, lo, hi);
            if (seg[i].done) lo = hi = 0;  // its threshold is exact already
            s_i = i;
            s_lo = lo;
            s_hi = hi;
        }
        __syncthreads();
        const long long lo = s_lo, hi = s_hi;
        const int i = s_i;
        if (hi > lo) {
            SegDev& S = seg[i];
            const uint32_t want = S.pre[pass];
            const int base = S.b;
            // block-uniform trip count: the appends are aggregated per block
            for (long long j0 = lo; j0 < hi; j0 += blockDim.x) {
                const long long j = j0 + threadIdx.x;
                u64 p = 0;
                int id = 0;
                bool take = false;
                if (j < hi) {
                    if (pass) {
                        p = lp[j];
                        id = li[j];
                        take = seg_digit(p, id, pass) == want;
                    } else if (alive[j]) {
                        p = prim[j];
                        take = (uint32_t)(p >> 52) == want;
                        if (take) id = pos[j].w;
                    }
                }
                const int slot = block_append(take, &S.len[pass & 1]);
                if (take) {
                    op[base + slot] = p;
                    oi[base + slot] = id;
                }
            }
        }
        __syncthreads();
    }
}

__global__ void seg_count_kernel(const uint8_t* __restrict__ flag, const int4* __restrict__ pos,
                                 int64_t ng, int shift, unsigned long long* cnt) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ng || !flag[s]) return;
    atomicAdd(&cnt[seg_of(pos[s], shift)], 1ull);
}

__global__ void seg_accept_kernel(const u64* __restrict__ prim, const int4* __restrict__ pos,
                                  const uint8_t* __restrict__ alive, int64_t ng,
                                  const RoundDev* rd, uint8_t* inP, int* cand, int* ncand) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ng || !alive[s]) return;
    const int4 p = pos[s];
    u64 tp;
    int ti;
    round_tau(rd, p, tp, ti);
    if (key_gt(tp, ti, prim[s], p.w)) return;
    inP[s] = 1;
    cand[atomicAdd(ncand, 1)] = (int)s;
}

// ------------------------------------------------------------------ launchers
static int grid_for(long long items) {
    long long b = items < BATCH_BLOCKS ? items : BATCH_BLOCKS;
    return b < 1 ? 1 : (int)b;
}

cudaError_t pack_launch_bbox(PackScan* sc, int nsc, int nchunks, cudaStream_t st) {
    pack_bbox_kernel<<<grid_for(nchunks), 256, 0, st>>>(sc, nsc, nchunks); note_launch();
    return cudaGetLastError();
}
cudaError_t pack_launch_copy(const PackScan* sc, int nsc, int nchunks, int32_t* out_xyz,
                             uint8_t* out_rgb, float* out_nrm, cudaStream_t st) {
    pack_copy_kernel<<<grid_for(nchunks), 256, 0, st>>>(sc, nsc, nchunks, out_xyz, out_rgb,
                                                        out_nrm); note_launch();
    return cudaGetLastError();
}
cudaError_t pack_launch_unpack(const PackScan* sc, int nsc, int nchunks, const uint8_t* keep,
                               cudaStream_t st) {
    pack_unpack_kernel<<<grid_for(nchunks), 256, 0, st>>>(sc, nsc, nchunks, keep); note_launch();
    return cudaGetLastError();
}
cudaError_t seg_launch_ranges(const int4* pos, int64_t ng, SegDev* seg, int* chunk0, int* items,
                              int nseg, int shift, cudaStream_t st) {
    if (nseg < 1 || nseg > PD_SEG_MAX) return cudaErrorInvalidValue;
    seg_ranges_kernel<<<(nseg + 1 + 255) / 256, 256, 0, st>>>(pos, ng, seg, nseg, shift); note_launch();
    seg_chunks_kernel<<<1, 1024, 0, st>>>(seg, nseg, chunk0, items); note_launch();
    return cudaGetLastError();
}
cudaError_t seg_launch_select(const u64* prim, const int4* pos, const uint8_t* alive, int64_t ng,
                              SelBuffers& b, uint32_t* hist, RoundDev* rd, SegDev* seg,
                              const int* chunk0, const int* items, int nseg, cudaStream_t st) {
    if (nseg < 1 || nseg > PD_SEG_MAX) return cudaErrorInvalidValue;
    // work items: at most ng / CHUNK + nseg; the launch size depends on the
    // layout only, so a captured round replays it unchanged
    const int blocks = grid_for(ng / PD_SEG_CHUNK + nseg);
    seg_setup_kernel<<<1, 32, 0, st>>>(rd); note_launch();
    for (int pass = 0; pass < 8; pass++) {
        seg_hist_kernel<<<blocks, 256, 0, st>>>(prim, alive, b.p[0], b.i[0], b.p[1], b.i[1], pass,
                                                seg, chunk0, items, nseg, hist); note_launch();
        seg_find_kernel<<<nseg, 256, 0, st>>>(hist, pass, rd, seg); note_launch();
        if (pass < 7) {
            seg_compact_kernel<<<blocks, 256, 0, st>>>(prim, pos, alive, b.p[0], b.i[0], b.p[1],
                                                       b.i[1], pass, seg, chunk0, items, nseg); note_launch();
        }
    }
    return cudaGetLastError();
}
cudaError_t seg_launch_count(const uint8_t* flag, const int4* pos, int64_t ng, int shift,
                             unsigned long long* cnt, cudaStream_t st) {
    if (ng < 1) return cudaSuccess;
    seg_count_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(flag, pos, ng, shift, cnt); note_launch();
    return cudaGetLastError();
}
cudaError_t seg_launch_accept(const u64* prim, const int4* pos, const uint8_t* alive, int64_t ng,
                              const RoundDev* rd, uint8_t* inP, int* cand, int* ncand,
                              cudaStream_t st) {
    if (ng < 1) return cudaSuccess;
    seg_accept_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(prim, pos, alive, ng, rd, inP,
                                                                    cand, ncand); note_launch();
    return cudaGetLastError();
}

}  // namespace pd
