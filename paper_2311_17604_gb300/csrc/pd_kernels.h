// pd_kernels.h -- host-side launchers of the libpd kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_internal.cuh"

namespace pd {

typedef unsigned long long u64;

// Scratch memory handed to launchers by the caller (the grid object).
struct Scratch {
    void* (*alloc)(void* self, size_t bytes);
    void (*free)(void* self, void* p);
    void* self;
    void* get(size_t bytes) const { return alloc(self, bytes); }
    void put(void* p) const { free(self, p); }
};

// ---------------------------------------------------------------- grid.cu
cudaError_t launch_bbox(const int32_t* xyz, int64_t n, int* out6, cudaStream_t st);
cudaError_t launch_morton(const int32_t* xyz, int64_t n, int3 origin, int shift, u64* keys,
                          uint32_t* vals, cudaStream_t st);
// Stable LSD radix sort of (keys, vals) on bits [0, bits); results land in
// keys/vals (ping-pong through tmp buffers).
cudaError_t radix_sort_pairs(u64* keys, uint32_t* vals, int64_t n, int bits, const Scratch& s,
                             cudaStream_t st);
cudaError_t exclusive_scan_u32(uint32_t* data, int64_t len, const Scratch& s, cudaStream_t st);
cudaError_t launch_gather(const int32_t* xyz, const uint8_t* rgb, const float* nrm,
                          const uint32_t* perm, int64_t n, int4* pos, uchar4* rgb_s,
                          float4* nrm_s, cudaStream_t st);
cudaError_t launch_gather_nrm(const float* nrm, const int4* pos, int64_t n, float4* out,
                              cudaStream_t st);
cudaError_t launch_leaf_levels(const u64* code, int64_t n, int T, int B, uint8_t* leaf,
                               cudaStream_t st);
cudaError_t launch_node_count(const u64* code, const uint8_t* leaf, int64_t n, int B,
                              unsigned long long* count, cudaStream_t st);
cudaError_t launch_node_insert(const u64* code, const uint8_t* leaf, int64_t n, int B,
                               HashSlot* tab, u64 mask, cudaStream_t st);
// Groups of <= 32 points of one leaf, for every point (full mode).
cudaError_t launch_leaf_groups(const GridView& g, int64_t n, int4* groups, int* ngroups,
                               cudaStream_t st);
// Stable compaction: out = ascending s with flag[s] != 0; *count on device.
cudaError_t stable_compact(const uint8_t* flag, int64_t n, int* out, int* count,
                           const Scratch& s, cudaStream_t st);

// ---------------------------------------------------------------- quality.cu
#define PD_QUALITY_MAXR 32
// Per retained point (grid order): neighbour counts within each radius (r2:
// ascending squared radii, nr <= PD_QUALITY_MAXR) over the 3x3x3 cells of
// level L (cell edge >= the largest radius); per radius the sums of N and
// N^2 and a histogram of N with H bins (the top bin holds N >= H - 1).
cudaError_t launch_radius_counts(const GridView& g, int64_t n, int L, const u64* r2, int nr,
                                 u64* sum_n, u64* sum_n2, uint32_t* hist, int H,
                                 cudaStream_t st);
// Per block of 256 points: least nearest squared distance and sum of sqrt.
cudaError_t launch_spacing(const u64* rk2, int64_t n, u64* bmin, double* bsum, cudaStream_t st);
// out[t] = xyz row list[t] for t < *count (cap >= *count rows are reserved).
cudaError_t launch_take_xyz(const int* list, const int* count, int64_t cap, const int32_t* xyz,
                            int32_t* out, cudaStream_t st);

// ---------------------------------------------------------------- round state
#define PD_FIX_ITERS 32    // device fixpoint sweeps of a k = 1 round (the most)
#define PD_FIX_ITERS_KK 8  // ... of a k >= 2 round (danger pairs)

// ---------------------------------------------------------------- packed batches
// Many independent scans decimated in one grid (batch.cu).  Scan i is moved
// into the aligned cube ("tile") of edge 2^shift mm whose Morton index is i;
// tiles are far enough apart that no neighbour search reaches another scan,
// and every scan occupies one contiguous range of the Morton order.  The
// removal threshold of a round (R2) is selected per scan.
#define PD_SEG_MAX 4096      // scans of one packed batch (16 tiles per axis)
#define PD_SEG_CHUNK 8192    // grid positions per work item of the per-scan passes
struct SegDev {
    long long live, m, need, rank;
    unsigned long long tau_prim;  // this round's threshold (~0: nothing to remove)
    int tau_idx;
    int done;                     // selection finished for this round
    unsigned pre[8];
    int len[2];                   // selection lists: [b, b + len) of the ping-pong buffers
    int b, e;                     // the scan's grid positions [b, e)
};

// Per-round control block in device memory (read by the host once per round).
struct RoundDev {
    long long live, m, need, rank;
    double band, band_max;
    unsigned long long removed, cap_over;
    unsigned long long tot_requery, tot_filtered, tot_sources, tot_updated, tot_lambda;
    unsigned long long tau_prim;
    int tau_idx;
    int done;
    unsigned pre[8];
    int len[2];
    int ncand, nslow, nsrc, npairs, overflow, ncs;
    int ndep;  // k = 1: candidates with a shell member of larger input index
    int changed[PD_FIX_ITERS];
    int fix_unconverged;
    int density_k1;
    int band_mode;  // 0: shrink on overflow only; 1: also on poor yield
    int fix_iters;  // device fixpoint sweeps per round (<= PD_FIX_ITERS)
    // packed batch (NULL seg: one scan).  Then tau_prim above is the least
    // threshold over the scans (a prefilter) and each point takes its own
    // scan's threshold.
    SegDev* seg;
    const int* seg_chunk0;  // nseg + 1 prefix counts of PD_SEG_CHUNK work items
    int nseg, seg_shift;
    int seg_rank_one;       // select each scan's largest key only (host settle)
};

#ifdef __CUDACC__
// The scan of a packed batch that holds grid point p (its tile's Morton index).
__device__ __forceinline__ int seg_of(int4 p, int shift) {
    return (int)morton3((uint32_t)p.x >> shift, (uint32_t)p.y >> shift, (uint32_t)p.z >> shift);
}
// The removal threshold of the round that applies to grid point p.
__device__ __forceinline__ void round_tau(const RoundDev* rd, int4 p, unsigned long long& tp,
                                          int& ti) {
    if (rd->seg) {
        const SegDev& s = rd->seg[seg_of(p, rd->seg_shift)];
        tp = s.tau_prim;
        ti = s.tau_idx;
    } else {
        tp = rd->tau_prim;
        ti = rd->tau_idx;
    }
}
#endif

struct SelBuffers {
    u64* p[2];
    int* i[2];
    uint32_t* hist;
};

// ---------------------------------------------------------------- knn.cu
enum { FILT_NONE = 0, FILT_BELOW_SELF = 1, FILT_BELOW_TAU = 2 };
#define PD_PAIR_SLOTS 64

struct KnnArgs {
    const int4* groups;
    int ngroups;
    const int* list;          // list mode: group.x is an offset into list
    const uint8_t* alive;     // NULL = every point live
    const u64* prim;          // keys (filter modes)
    int filter;
    u64 tau_prim;
    int tau_idx;
    const RoundDev* rd;       // when set, tau is read from rd (device)
    const uint8_t* qflag;     // when set, only flagged points of each group are queried
    int k;
    int S;                    // stored neighbours (template width)
    int density_k1;           // integer-ordered k = 1 density cost
    int term;
    double weight;
    const uchar4* rgb;
    const float4* nrm;
    // outputs (full / re-query mode)
    int* nbr;                 // n x S Morton positions
    int* nbr0_out;            // optional: the first stored entry again, one int per point
    u64* prim_out;            // key primary
    u64* rk2_out;             // k-th squared distance
    uint8_t* flg_out;
    u64* hz_out;              // horizon: S-th stored squared distance (~0 if fewer)
    double* cost_out;         // cost in Morton order (optional)
    // outputs (filter modes)
    u64* fprim_out;           // FILT_BELOW_SELF: key primary over lower keys
    u64* lam_out;             // FILT_BELOW_TAU: k-th squared distance over keys < tau
    unsigned long long* pairs_out;  // optional: + (query, candidate) pairs scanned, spread
                                    //   over PD_PAIR_SLOTS counters (their sum is the count)
    const u64* cmin;          // filtered searches: least live key primary of every aligned
                              //   32-position chunk (chunks above the threshold are skipped)
    const int* glist;         // group-list mode: process groups glist[0 .. *gcount)
    const int* gcount;        //   (device count; a persistent grid walks the list)
    int r_exact;              // full searches: nearest entries that must be exact
                              //   (0 = all S; the k = 1 density cost re-searches
                              //   with 1 and keeps the rest below the horizon)
};
// Flagged mode without a host read: list the groups that hold a flagged query
// (a.qflag), then run the search over that list only.  glist: ngroups ints,
// gcount: one int, both device scratch.
// cmin[c] = least key primary of the live points at Morton positions
// [32c, 32c + 32) (~0 when none), for the chunk skipping of filtered searches.
cudaError_t launch_chunk_min(const u64* prim, const uint8_t* alive, int64_t n, u64* cmin,
                             cudaStream_t st);
cudaError_t launch_knn_flagged(const GridView& g, const KnnArgs& a, int* glist, int* gcount,
                               cudaStream_t st);
cudaError_t launch_knn(const GridView& g, const KnnArgs& a, cudaStream_t st);
// Full (FILT_NONE) searches of the listed Morton positions list[0 .. *count)
// (count on the device, at most cap), 2 lanes per query, each over its own
// leaf cells: for sparse re-searches.
cudaError_t launch_knn_sparse(const GridView& g, const KnnArgs& a, const int* list,
                              const int* count, int64_t cap, cudaStream_t st);
// Internal neighbour-weight term: unit weights with equal distances ordered by
// input index (the normals' 16-NN order).
#define PD_TERM_INDEX_TIE 3

// ---------------------------------------------------------------- rounds.cu
struct SelectResult {
    u64 prim;
    int idx;
};

}  // namespace pd

namespace pd {
// ---------------------------------------------------------------- rounds_dev.cu
cudaError_t round_launch_setup(RoundDev* rd, cudaStream_t st);
// The candidate band of the next round (k >= 2 and weighted costs) from this
// round's counts; the same arithmetic runs on the device after a normal round
// and on the host after a round it settled.
double host_next_band(double band, double band_max, int band_mode, unsigned long long cap_over,
                      long long ncand, unsigned long long removed);
cudaError_t round_launch_finish(RoundDev* rd, cudaStream_t st);
cudaError_t round_launch_select(const u64* prim, const int4* pos, const uint8_t* alive, int64_t n,
                                SelBuffers& b, RoundDev* rd, cudaStream_t st);
// dep: list of the candidates that have a shell member of larger input index
// (the only ones condition (B) can reject; the fixpoint sweeps walk it).
// nbr0: the first stored entries apart (may be NULL).
cudaError_t round_launch_k1(const GridView& g, const u64* prim, const uint8_t* alive,
                            const int* nbr, const int* nbr0, const uint8_t* flg, const u64* rk2,
                            int64_t n, int S, RoundDev* rd, uint8_t* inP, uint8_t* rej, int* cand,
                            int* slow, int* dep, int fix_iters, cudaStream_t st);
cudaError_t round_launch_kk_accept(const uint8_t* fq_flag, const u64* prim, const u64* fprim,
                                   int64_t n, RoundDev* rd, uint8_t* inP, int* cand,
                                   cudaStream_t st);
cudaError_t round_launch_danger(const GridView& g, const int* src, const u64* prim,
                                const uint8_t* alive, const uint8_t* inP, uint8_t* rej,
                                const u64* lam, const int* nbr, int S, int k, int2* pairs,
                                int pair_cap, const int* csorted, RoundDev* rd, cudaStream_t st);
cudaError_t round_launch_pairs_fix(const int2* pairs, int pair_cap, const uint8_t* inP,
                                   uint8_t* rej, RoundDev* rd, cudaStream_t st);
cudaError_t round_launch_remove(const int* cand, uint8_t* inP, uint8_t* rej, uint8_t* alive,
                                RoundDev* rd, cudaStream_t st);
cudaError_t round_launch_dirty(const uint8_t* alive, const int* nbr, int64_t n, int S, int kchk,
                               uint8_t* dirty, RoundDev* rd, cudaStream_t st);
struct BufView {  // the k+b neighbour buffer of every point
    const int4* pos;
    u64* prim;
    int* nbr;
    int* nbr0;  // optional (k = 1 density): nbr[s * S] kept apart, read coalesced
    u64* rk2;
    uint8_t* flg;
    u64* hz;
    const uchar4* rgb;
    const float4* nrm;
    int term;
    double weight;
};
// k = 1 density cost: absorb removals in the stored nearest entries (the
// shell at the new nearest distance must lie below the search horizon);
// dirty[s] = 1 where a new search is needed.
cudaError_t round_launch_k1_update(const BufView& b, const uint8_t* alive, int64_t n, int S,
                                   uint8_t* dirty, RoundDev* rd, cudaStream_t st);
cudaError_t round_launch_kk_update(const BufView& b, const uint8_t* alive, int64_t n, int S, int k,
                                   uint8_t* dirty, RoundDev* rd, cudaStream_t st);
cudaError_t round_launch_kk_cand2(const BufView& b, const uint8_t* alive, int64_t n, int S, int k,
                                  RoundDev* rd, uint8_t* inP, int* cand, uint8_t* fq_flag,
                                  uint8_t* lq_flag, u64* lam, int* src, cudaStream_t st);
}  // namespace pd

// ---------------------------------------------------------------- normals.cu
struct pd_ctx;
struct pd_grid;
namespace pd {
struct GridNbrs {
    const int4* pos;
    const int* nbr;  // n x S Morton positions, nearest first, -1 past the found ones
    int S;
    int64_t n;
    pd_ctx* ctx;
};
// capi.cu: context allocator, error text, and the 16-NN pass over a grid
void* api_alloc(pd_ctx* c, size_t bytes, cudaStream_t st);
void api_free(pd_ctx* c, void* p, cudaStream_t st);
void api_error(pd_ctx* c, const char* what, long long v);
int grid_knn16(pd_grid* g, cudaStream_t st, GridNbrs* out);
cudaError_t launch_features(const int4* pos, const int* nbr, int S, int64_t n, uint16_t* feat,
                            float* pca, uint8_t* valid, cudaStream_t st);
cudaError_t launch_mlp_forward(const float* prm, const uint16_t* feat, const int* rows, int64_t n,
                               float* outn, float* onorm, float* h1s, float* h2s, float* raw,
                               cudaStream_t st);
// Partials: mlp_backward_part_floats() floats of scratch; the gradient is
// reduced over blocks in a fixed order (deterministic).
int64_t mlp_backward_part_floats();
cudaError_t launch_mlp_backward(const float* prm, const uint16_t* feat, const int* rows,
                                const float* labels, int64_t n, const float* h1s,
                                const float* h2s, const float* raw, float* grad, float* loss,
                                float* part, cudaStream_t st);
cudaError_t launch_adam(float* prm, float* m, float* v, const float* grad, int t, float lr,
                        cudaStream_t st);
cudaError_t launch_mlp_init(float* prm, u64 seed, cudaStream_t st);
cudaError_t launch_sample_rows(const int* pool, int64_t npool, u64 seed, long long t, int b,
                               int* rows, cudaStream_t st);
cudaError_t launch_normal_fallback(const float* mlp, const float* onorm, const float* pca,
                                   int64_t n, float min_norm, float* out, cudaStream_t st);
// ---------------------------------------------------------------- wup.cu
// The paper's iterative w_up scheme: set the rank (live - m) for the key
// selection of w_up, then run one removal round (marks, picks, removal,
// stored-list update).  S <= 8, k <= S.
cudaError_t wup_launch_setup(RoundDev* rd, cudaStream_t st);
// Replace the selection's bin boundary by the smallest live key at or above
// it (the exact rank-th largest key).  tmin, imin: device scratch words.
cudaError_t wup_launch_exact_tau(const u64* prim, const int4* pos, const uint8_t* alive,
                                 int64_t n, RoundDev* rd, u64* tmin, int* imin, cudaStream_t st);
cudaError_t wup_launch_round(const BufView& b, uint8_t* alive, uint8_t* wdirty, int64_t n, int S,
                             int k, RoundDev* rd, u64* mark_p, int* mark_i, uint8_t* pick,
                             cudaStream_t st);

// ---------------------------------------------------------------- batch.cu
// One scan of a packed batch (device array, host-built): its caller-owned
// buffers, its first packed position and work item, and the per-axis offset
// that moves it into its tile (packed = input + o).
struct PackScan {
    const int32_t* xyz;
    const uint8_t* rgb;
    const float* nrm;
    uint8_t* keep;
    long long n, off;
    int chunk0;
    int ox, oy, oz;
    int bb[6];  // bounding box (min x, y, z, max x, y, z), from pack_launch_bbox
};
// Bounding boxes of every scan (sc[i].bb, preset to empty boxes by the caller).
cudaError_t pack_launch_bbox(PackScan* sc, int nsc, int nchunks, cudaStream_t st);
// Packed coordinates (and colours, normals where out_rgb / out_nrm are set).
cudaError_t pack_launch_copy(const PackScan* sc, int nsc, int nchunks, int32_t* out_xyz,
                             uint8_t* out_rgb, float* out_nrm, cudaStream_t st);
// Every scan's keep mask from the packed one.
cudaError_t pack_launch_unpack(const PackScan* sc, int nsc, int nchunks, const uint8_t* keep,
                               cudaStream_t st);
// Grid ranges [b, e) of every scan, the prefix counts of their work items
// (chunk0[0..nseg]) and the scan of every work item (items: ng / PD_SEG_CHUNK
// + nseg entries at least), from the Morton-ordered positions.
cudaError_t seg_launch_ranges(const int4* pos, int64_t ng, SegDev* seg, int* chunk0, int* items,
                              int nseg, int shift, cudaStream_t st);
// Per-scan selection of the round's threshold (R2): every scan's rank-th
// largest live key, rank from its live count, target and the band.  hist:
// nseg x 4096 words, zero on entry and on return.
cudaError_t seg_launch_select(const u64* prim, const int4* pos, const uint8_t* alive, int64_t ng,
                              SelBuffers& b, uint32_t* hist, RoundDev* rd, SegDev* seg,
                              const int* chunk0, const int* items, int nseg, cudaStream_t st);
// cnt[scan] += flagged points of the scan.
cudaError_t seg_launch_count(const uint8_t* flag, const int4* pos, int64_t ng, int shift,
                             unsigned long long* cnt, cudaStream_t st);
// Candidates: every live point whose key reaches its scan's threshold.
cudaError_t seg_launch_accept(const u64* prim, const int4* pos, const uint8_t* alive, int64_t ng,
                              const RoundDev* rd, uint8_t* inP, int* cand, int* ncand,
                              cudaStream_t st);

}  // namespace pd
