// knn.cu -- exact k-nearest-neighbour search and cost (Eq. 10 / Eq. 11).
//
// One warp serves one group of <= 32 query points that share an octree leaf
// of level L.  The warp resolves the 3x3x3 level-L cells around the leaf in
// the hashed cell table (the own cell first), then scans their points in
// chunks of 32: every lane loads one candidate (a coalesced 16-byte int4
// load of {x, y, z, index}), the chunk is staged in shared memory, and every
// lane streams the whole chunk against its own query, keeping the S smallest
// (d^2, position) pairs in registers.  Squared distances are exact integers:
// uint32 at levels whose resolved cells are at most 2^13 mm wide (every
// coordinate difference within the 3x3x3 cells is then below 3 * 2^13, so
// d^2 < 2^32), uint64 otherwise.  A cell is skipped when its box is farther than
// the current bound for every lane.  Exactness: every point outside the
// searched cube lies at least g from the query (g = distance to the cube's
// faces); when the bound that matters is below g^2 the lane is done,
// otherwise the search repeats one level up (a cube of twice the size).
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_internal.cuh"
#include "pd_kernels.h"

namespace pd {

#define FULLM 0xffffffffu

// The S smallest (d^2, input index) pairs; id holds the Morton position.
// Equal distances are ordered by input index, as in the definition's reading
// (it matters only when neighbour weights differ, i.e. colour/orientation).
template <int S, bool W>
struct TopList;

// Density costs: any order among equal distances gives the same cost, so the
// Morton position serves as the tie order (no extra registers).
template <int S>
struct TopList<S, false> {
    u64 d[S];
    int id[S];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < S; i++) {
            d[i] = ~0ull;
            id[i] = 0x7fffffff;
        }
    }
    __device__ __forceinline__ int tie(int i) const { return id[i]; }
    __device__ __forceinline__ bool beats_last(u64 dd, int j, int) const {
        return dd < d[S - 1] || (dd == d[S - 1] && j < id[S - 1]);
    }
    __device__ __forceinline__ void insert(u64 dd, int j, int) {
        d[S - 1] = dd;
        id[S - 1] = j;
#pragma unroll
        for (int i = S - 1; i > 0; i--) {
            bool sw = d[i] < d[i - 1] || (d[i] == d[i - 1] && id[i] < id[i - 1]);
            u64 a = d[i], b = d[i - 1];
            int x = id[i], y = id[i - 1];
            d[i - 1] = sw ? a : b;
            d[i] = sw ? b : a;
            id[i - 1] = sw ? x : y;
            id[i] = sw ? y : x;
        }
    }
    __device__ __forceinline__ u64 at(int r) const {
        u64 v = d[0];
#pragma unroll
        for (int i = 1; i < S; i++)
            if (i == r) v = d[i];
        return v;
    }
    __device__ __forceinline__ u64 dist(int i) const { return d[i]; }
    __device__ __forceinline__ int ident(int i) const { return id[i]; }
    __device__ __forceinline__ bool has(int i) const { return d[i] != ~0ull; }
    // merge the list of lane (lane ^ off) into this lane's (active lanes only)
    __device__ __forceinline__ void merge_xor(int off, bool active) {
        u64 od[S];
        int oj[S], oo[S];
#pragma unroll
        for (int i = 0; i < S; i++) {
            od[i] = __shfl_xor_sync(0xffffffffu, d[i], off);
            oj[i] = __shfl_xor_sync(0xffffffffu, id[i], off);
            oo[i] = __shfl_xor_sync(0xffffffffu, tie(i), off);
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < S; i++)
                if (od[i] != ~0ull && beats_last(od[i], oj[i], oo[i])) insert(od[i], oj[i], oo[i]);
        }
    }
};

template <int S>
struct TopList<S, true> {
    u64 d[S];
    int id[S];
    int oi[S];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < S; i++) {
            d[i] = ~0ull;
            id[i] = 0x7fffffff;
            oi[i] = 0x7fffffff;
        }
    }
    __device__ __forceinline__ int tie(int i) const { return oi[i]; }
    __device__ __forceinline__ bool beats_last(u64 dd, int, int o) const {
        return dd < d[S - 1] || (dd == d[S - 1] && o < oi[S - 1]);
    }
    __device__ __forceinline__ void insert(u64 dd, int j, int o) {
        d[S - 1] = dd;
        id[S - 1] = j;
        oi[S - 1] = o;
#pragma unroll
        for (int i = S - 1; i > 0; i--) {
            bool sw = d[i] < d[i - 1] || (d[i] == d[i - 1] && oi[i] < oi[i - 1]);
            u64 a = d[i], b = d[i - 1];
            int x = id[i], y = id[i - 1];
            int u = oi[i], v = oi[i - 1];
            d[i - 1] = sw ? a : b;
            d[i] = sw ? b : a;
            id[i - 1] = sw ? x : y;
            id[i] = sw ? y : x;
            oi[i - 1] = sw ? u : v;
            oi[i] = sw ? v : u;
        }
    }
    __device__ __forceinline__ u64 at(int r) const {
        u64 v = d[0];
#pragma unroll
        for (int i = 1; i < S; i++)
            if (i == r) v = d[i];
        return v;
    }
    __device__ __forceinline__ u64 dist(int i) const { return d[i]; }
    __device__ __forceinline__ int ident(int i) const { return id[i]; }
    __device__ __forceinline__ bool has(int i) const { return d[i] != ~0ull; }
    // merge the list of lane (lane ^ off) into this lane's (active lanes only)
    __device__ __forceinline__ void merge_xor(int off, bool active) {
        u64 od[S];
        int oj[S], oo[S];
#pragma unroll
        for (int i = 0; i < S; i++) {
            od[i] = __shfl_xor_sync(0xffffffffu, d[i], off);
            oj[i] = __shfl_xor_sync(0xffffffffu, id[i], off);
            oo[i] = __shfl_xor_sync(0xffffffffu, tie(i), off);
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < S; i++)
                if (od[i] != ~0ull && beats_last(od[i], oj[i], oo[i])) insert(od[i], oj[i], oo[i]);
        }
    }
};


// The same lists when every squared distance of the search level is below
// 2^32: one 64-bit key (d^2 << 32 | tie) per entry, so that a compare-exchange
// stage is one 64-bit compare and select.  The order is the same as above
// ((d^2, tie) lexicographic), so results are identical.  W = false: the tie is
// the Morton position, which is also the neighbour; W = true: the tie is the
// input index and the Morton position is kept beside it.
template <int S, bool W>
struct TopPack {
    u64 key[S];
    int pid[W ? S : 1];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < S; i++) key[i] = ~0ull;
        if (W) {
#pragma unroll
            for (int i = 0; i < S; i++) pid[W ? i : 0] = 0x7fffffff;
        }
    }
    __device__ __forceinline__ static u64 pack(u64 dd, int j, int o) {
        return (dd << 32) | (uint32_t)(W ? o : j);
    }
    __device__ __forceinline__ int tie(int i) const { return (int)(uint32_t)key[i]; }
    __device__ __forceinline__ bool beats_last(u64 dd, int j, int o) const {
        return pack(dd, j, o) < key[S - 1];
    }
    __device__ __forceinline__ void insert(u64 dd, int j, int o) {
        key[S - 1] = pack(dd, j, o);
        if (W) pid[W ? S - 1 : 0] = j;
#pragma unroll
        for (int i = S - 1; i > 0; i--) {
            u64 a = key[i], b = key[i - 1];
            bool sw = a < b;
            key[i - 1] = sw ? a : b;
            key[i] = sw ? b : a;
            if (W) {
                int x = pid[W ? i : 0], y = pid[W ? i - 1 : 0];
                pid[W ? i - 1 : 0] = sw ? x : y;
                pid[W ? i : 0] = sw ? y : x;
            }
        }
    }
    __device__ __forceinline__ bool has(int i) const { return key[i] != ~0ull; }
    __device__ __forceinline__ u64 dist(int i) const {
        return key[i] == ~0ull ? ~0ull : (key[i] >> 32);
    }
    __device__ __forceinline__ int ident(int i) const {
        return W ? pid[W ? i : 0] : (int)(uint32_t)key[i];
    }
    __device__ __forceinline__ u64 at(int r) const {
        u64 v = key[0];
#pragma unroll
        for (int i = 1; i < S; i++)
            if (i == r) v = key[i];
        return v == ~0ull ? ~0ull : (v >> 32);
    }
    __device__ __forceinline__ void merge_xor(int off, bool active) {
        u64 ok[S];
        int op[W ? S : 1];
#pragma unroll
        for (int i = 0; i < S; i++) {
            ok[i] = __shfl_xor_sync(0xffffffffu, key[i], off);
            if (W) op[W ? i : 0] = __shfl_xor_sync(0xffffffffu, pid[W ? i : 0], off);
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < S; i++) {
                if (ok[i] != ~0ull && ok[i] < key[S - 1]) {
                    key[S - 1] = ok[i];
                    if (W) pid[W ? S - 1 : 0] = op[W ? i : 0];
#pragma unroll
                    for (int t = S - 1; t > 0; t--) {
                        u64 a = key[t], b = key[t - 1];
                        bool sw = a < b;
                        key[t - 1] = sw ? a : b;
                        key[t] = sw ? b : a;
                        if (W) {
                            int x = pid[W ? t : 0], y = pid[W ? t - 1 : 0];
                            pid[W ? t - 1 : 0] = sw ? x : y;
                            pid[W ? t : 0] = sw ? y : x;
                        }
                    }
                }
            }
        }
    }
};

__device__ inline u64 box_d2(int ux, int uy, int uz, int bx, int by, int bz, int sh) {
    long long q[3] = {ux, uy, uz};
    int c[3] = {bx, by, bz};
    u64 s = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long lo = (long long)c[a] << sh;
        long long hi = ((long long)(c[a] + 1) << sh) - 1;
        long long d = q[a] < lo ? lo - q[a] : (q[a] > hi ? q[a] - hi : 0);
        s += (u64)(d * d);
    }
    return s;
}

// The same in 32-bit arithmetic, for levels whose cell edge is at most
// 2^13 mm: the box is the query's own or an adjacent cell's leaf, so every
// coordinate gap is below 2 * 2^13 and the sum below 2^30.
__device__ inline u64 box_d2_32(int ux, int uy, int uz, int bx, int by, int bz, int sh) {
    const int q[3] = {ux, uy, uz};
    const int c[3] = {bx, by, bz};
    uint32_t s = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int lo = c[a] * (1 << sh);
        const int hi = (c[a] + 1) * (1 << sh) - 1;
        const int d = q[a] < lo ? lo - q[a] : (q[a] > hi ? q[a] - hi : 0);
        s += (uint32_t)(d * d);
    }
    return (u64)s;
}

// Squared distance from the query to the outside of the level-L cube of
// cells [c-1, c+1]; ~0 when the cube holds the whole cloud.
__device__ inline u64 gap2(const GridView& g, int ux, int uy, int uz, int L, int cx, int cy,
                           int cz) {
    int sh = L + g.shift;
    long long q[3] = {ux, uy, uz};
    int c[3] = {cx, cy, cz};
    int m[3] = {g.umax.x, g.umax.y, g.umax.z};
    long long best = -1;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long lo = (long long)(c[a] - 1) << sh;
        long long hi = (long long)(c[a] + 2) << sh;
        if (lo > 0) {
            long long d = q[a] - lo + 1;
            if (best < 0 || d < best) best = d;
        }
        if (hi <= m[a]) {
            long long d = hi - q[a];
            if (best < 0 || d < best) best = d;
        }
    }
    return best < 0 ? ~0ull : (u64)best * (u64)best;
}

__device__ inline double nbr_weight(const KnnArgs& a, int q, int j) {
    if (a.term == 1) {  // colour deviation
        uchar4 p = a.rgb[q], r = a.rgb[j];
        double dr = (double)p.x - (double)r.x;
        double dg = (double)p.y - (double)r.y;
        double db = (double)p.z - (double)r.z;
        double s = __dmul_rn(dr, dr);
        s = __dadd_rn(s, __dmul_rn(dg, dg));
        s = __dadd_rn(s, __dmul_rn(db, db));
        double dist = __dsqrt_rn(s);
        double scale = __dmul_rn(255.0, __dsqrt_rn(3.0));
        return __dsub_rn(1.0, __dmul_rn(a.weight, __ddiv_rn(dist, scale)));
    }
    if (a.term == 2) {  // orientation, Eq. 13 with |n_p . n_q|
        float4 p = a.nrm[q], r = a.nrm[j];
        double d = __dmul_rn((double)p.x, (double)r.x);
        d = __dadd_rn(d, __dmul_rn((double)p.y, (double)r.y));
        d = __dadd_rn(d, __dmul_rn((double)p.z, (double)r.z));
        return __dsub_rn(1.0, __dmul_rn(a.weight, __dsub_rn(1.0, fabs(d))));
    }
    return 1.0;
}

template <int S, class TL>
__device__ inline double cost_sum(const KnnArgs& a, int q, const TL& top, int k) {
    double c = 0.0;
#pragma unroll
    for (int i = 0; i < S; i++) {
        if (i < k && top.has(i)) {
            double w = nbr_weight(a, q, top.ident(i));
            c = __dadd_rn(c, __ddiv_rn(w, (double)top.dist(i)));
        }
    }
    return c;
}

// Stream one range [b, e) of Morton positions against every lane's query.
template <int S, int FILT, bool W, class TL, typename D>
__device__ __forceinline__ void scan_range(const GridView& g, const KnnArgs& a, uint32_t b,
                                           uint32_t e, int q, int4 qp, bool todo, u64 tp, int ti,
                                           u64 tpmax, TL& top, int4* sp, u64* sk, int* so,
                                           int lane, int sub, int lpq) {
    for (uint32_t c = b; c < e; c += 32) {
        if (FILT != FILT_NONE && a.cmin) {
            // no key of these 32 positions is below any lane's threshold: skip
            // (c, e and tpmax are warp-uniform, so the whole warp skips)
            uint32_t last = min(c + 31u, e - 1u);
            u64 m0 = a.cmin[c >> 5], m1 = a.cmin[last >> 5];
            if ((m0 < m1 ? m0 : m1) > tpmax) continue;
        }
        uint32_t j = c + lane;
        int4 v = make_int4(0, 0, 0, -1);
        if (j < e) {
            v = g.pos[j];
            bool ok = !a.alive || a.alive[j];
            if (FILT != FILT_NONE) sk[lane] = a.prim[j];
            if (FILT != FILT_NONE || W) so[lane] = v.w;
            v.w = ok ? (int)j : -1;
        }
        sp[lane] = v;
        __syncwarp();
        int m = (int)min(32u, e - c);
        if (todo) {
            for (int t = sub; t < m; t += lpq) {
                int4 cv = sp[t];
                if (cv.w < 0 || cv.w == q) continue;
                if (FILT != FILT_NONE) {
                    if (!key_gt(tp, ti, sk[t], so[t])) continue;  // keep keys below threshold
                }
                int dx = cv.x - qp.x, dy = cv.y - qp.y, dz = cv.z - qp.z;
                D dd;
                if (sizeof(D) == 4) {
                    dd = (D)(dx * dx) + (D)(dy * dy) + (D)(dz * dz);
                } else {
                    dd = (D)((long long)dx * dx) + (D)((long long)dy * dy) + (D)((long long)dz * dz);
                }
                int co = W ? so[t] : cv.w;
                if (top.beats_last((u64)dd, cv.w, co)) top.insert((u64)dd, cv.w, co);
            }
        }
        __syncwarp();
    }
}

// Results of a query whose list is exact (one lane per query).
// hzv: squared distance below which every live point is in the list (the
// searched cube's gap and the skipped cells' boxes; the S-th distance when
// the list is full).
template <int S, int FILT, bool W, class TL>
__device__ __forceinline__ void write_result(const KnnArgs& a, int q, const TL& top, u64 hzv) {
    int found = 0;
#pragma unroll
    for (int i = 0; i < S; i++) found += top.has(i);
    if (FILT == FILT_NONE) {
        if (a.density_k1) {
            // all S nearest are stored (the k+b buffer); the shell is the
            // prefix at the nearest distance d0, its size kept in flg >> 2
            u64 d0 = top.dist(0);
            int shell = 0;
#pragma unroll
            for (int i = 0; i < S; i++) {
                bool h = top.has(i);
                shell += (h && top.dist(i) == d0) ? 1 : 0;
                a.nbr[(int64_t)q * S + i] = h ? top.ident(i) : -1;
            }
            if (!W && a.nbr0_out) a.nbr0_out[q] = top.has(0) ? top.ident(0) : -1;
            a.prim_out[q] = key_prim_d2(d0);
            a.rk2_out[q] = d0;
            a.flg_out[q] = (uint8_t)((shell >= 2 ? 1 : 0) | (shell == S ? 2 : 0) | (shell << 2));
            if (a.hz_out) {
                u64 h = top.has(S - 1) ? top.dist(S - 1) : ~0ull;
                a.hz_out[q] = hzv < h ? hzv : h;
            }
            if (a.cost_out) a.cost_out[q] = d0 == ~0ull ? 0.0 : __ddiv_rn(1.0, (double)d0);
        } else {
            int k = a.k;
#pragma unroll
            for (int i = 0; i < S; i++) a.nbr[(int64_t)q * S + i] = top.has(i) ? top.ident(i) : -1;
            double c = cost_sum<S>(a, q, top, k);
            a.prim_out[q] = key_prim_cost(c);
            u64 dk = top.at(k - 1);
            a.rk2_out[q] = dk;
            bool tie = found > k && top.at(k) == dk;
            a.flg_out[q] = (uint8_t)(tie ? 1 : 0);
            if (a.hz_out) a.hz_out[q] = top.dist(S - 1);
            if (a.cost_out) a.cost_out[q] = c;
        }
    } else if (FILT == FILT_BELOW_SELF) {
        if (a.density_k1) {
            a.fprim_out[q] = key_prim_d2(top.dist(0));
        } else {
            a.fprim_out[q] = key_prim_cost(cost_sum<S>(a, q, top, a.k));
        }
    } else {
        a.lam_out[q] = top.at(a.k - 1);
    }
}

// One search level for the warp: scan the resolved 3x3x3 ranges, merge each
// query's partial lists, and finish the queries whose R-th distance is
// closer than the searched cube's faces.  PACK: every range of this level
// has squared distances below 2^32 (packed lists, 32-bit distances).
template <int S, int FILT, bool W, class TL, bool PACK>
__device__ __forceinline__ void knn_level(const GridView& g, const KnnArgs& a, int L, int R,
                                          int q, int4 qp, int ux, int uy, int uz, bool& todo,
                                          u64 tp, int ti, u64 tpmax, int lane, int sub, int lpq,
                                          int rt,
                                          uint32_t rb, uint32_t re, int rl, int bx, int by,
                                          int bz, int cx, int cy, int cz, int4* sp, u64* sk,
                                          int* so, unsigned long long& wpairs) {
    TL top;
    top.init();
    u64 hzl = ~0ull;  // smallest box distance of a range this lane did not scan
    for (int r = 0; r < 27; r++) {
        int tr = __shfl_sync(FULLM, rt, r);
        if (!tr) continue;
        uint32_t b = __shfl_sync(FULLM, rb, r), e = __shfl_sync(FULLM, re, r);
        int lv = __shfl_sync(FULLM, rl, r);
        int bxr = __shfl_sync(FULLM, bx, r), byr = __shfl_sync(FULLM, by, r),
            bzr = __shfl_sync(FULLM, bz, r);
        bool skip = true;
        u64 bd = ~0ull;
        if (todo) {
            u64 bound = top.at(R - 1);
            bd = PACK ? box_d2_32(ux, uy, uz, bxr, byr, bzr, lv + g.shift)
                      : box_d2(ux, uy, uz, bxr, byr, bzr, lv + g.shift);
            skip = bound != ~0ull && bd > bound;
        }
        // every lane of the warp scans a range unless none needs it: the
        // lanes that do not still fill their stored entries beyond the R
        // nearest from it (measured: skipping per lane halves the candidates
        // a lane takes but leaves sparser buffers, whose extra re-searches in
        // the removal rounds cost more than the pass saves)
        if (__all_sync(FULLM, skip)) {
            if (bd < hzl) hzl = bd;
            continue;
        }
        if (a.pairs_out) {  // warp-uniform count of the pairs this range costs
            int nqt = __popc(__ballot_sync(FULLM, todo && sub == 0));
            wpairs += (unsigned long long)(e - b) * (unsigned long long)nqt;
        }
        if (PACK || lv + g.shift <= 13)
            scan_range<S, FILT, W, TL, uint32_t>(g, a, b, e, q, qp, todo, tp, ti, tpmax, top, sp,
                                                 sk, so, lane, sub, lpq);
        else
            scan_range<S, FILT, W, TL, u64>(g, a, b, e, q, qp, todo, tp, ti, tpmax, top, sp, sk, so,
                                            lane, sub, lpq);
    }
    // merge the partial lists of each query's lanes (butterfly)
    for (int off = lpq >> 1; off >= 1; off >>= 1) top.merge_xor(off, todo);
    if (todo) {
        u64 gg = L >= g.B ? ~0ull : gap2(g, ux, uy, uz, L, cx, cy, cz);
        u64 bound = top.at(R - 1);
        if (gg == ~0ull || bound < gg) {
            todo = false;
            if (sub == 0) write_result<S, FILT, W>(a, q, top, hzl < gg ? hzl : gg);
        }
    }
}

// One leaf group (<= 32 queries) for one warp.
template <int S, int FILT, bool W>
__device__ __forceinline__ void knn_group(const GridView& g, const KnnArgs& a, int gid, int4* sp,
                                          u64* sk, int* so, int lane) {
    int4 G = a.groups[gid];
    int cnt = G.y;
    int L = G.z;
    int q = -1;
    if (lane < cnt) {
        q = a.list ? a.list[G.x + lane] : G.x + lane;
        if (a.qflag && !a.qflag[q]) q = -1;
    }
    // pack the active queries onto the 32 lanes: with nq queries each gets
    // lpq = 32 / nq (power of two) lanes that split every staged chunk; their
    // partial lists are merged before the exactness test
    unsigned act = __ballot_sync(FULLM, q >= 0);
    if (!act) return;
    int nq = __popc(act);
    int lpq = 32;
    while (lpq > 1 && nq * lpq > 32) lpq >>= 1;
    int qi = lane / lpq, sub = lane - qi * lpq;
    {
        int srcl = qi < nq ? (int)__fns(act, 0, qi + 1) : 0;
        int qq = __shfl_sync(FULLM, q, srcl);
        q = qi < nq ? qq : -1;
    }
    int q0 = a.list ? a.list[G.x] : G.x;
    u64 c0 = g.code[q0];
    int4 qp = q >= 0 ? g.pos[q] : make_int4(0, 0, 0, 0);
    int ux = qp.x - g.origin.x, uy = qp.y - g.origin.y, uz = qp.z - g.origin.z;
    u64 tp = 0;
    int ti = 0;
    if (FILT == FILT_BELOW_SELF && q >= 0) {
        tp = a.prim[q];
        ti = qp.w;
    } else if (FILT == FILT_BELOW_TAU) {
        if (a.rd && a.rd->seg) {
            // packed batch: the threshold of the query's own scan (its
            // neighbours are all in that scan)
            if (q >= 0) round_tau(a.rd, qp, tp, ti);
        } else if (a.rd) {
            tp = a.rd->tau_prim;
            ti = a.rd->tau_idx;
        } else {
            tp = a.tau_prim;
            ti = a.tau_idx;
        }
    }
    // the largest threshold of the warp's queries (chunk skipping); reduced
    // over all 32 lanes so that every lane holds the same value: the skip in
    // scan_range must be taken by the whole warp or by none of it
    u64 tpmax = q >= 0 ? tp : 0;
    if (FILT != FILT_NONE) {
        for (int off = 16; off; off >>= 1) {
            u64 o = __shfl_xor_sync(FULLM, tpmax, off);
            tpmax = o > tpmax ? o : tpmax;
        }
    }
    // exactness bound: the R-th smallest distance must be exact
    // full searches: all S stored neighbours exact (the k+b neighbour buffer,
    // so a removal can be absorbed without a new search; for the k = 1
    // density cost the nearest shell is then complete); filtered searches: k.
    const int R = FILT == FILT_NONE ? (a.r_exact > 0 && a.r_exact < S ? a.r_exact : S) : a.k;
    bool todo = q >= 0;
    unsigned long long wpairs = 0;
    if (FILT == FILT_BELOW_TAU && a.hz_out) {
        // a lambda search runs when fewer than k lower-key points are among a
        // query's stored neighbours; every live point closer than its horizon
        // hz is stored, so lambda >= hz: start at the first level whose cell
        // edge reaches sqrt(hz) (smallest over the group's queries)
        u64 h = q >= 0 ? a.hz_out[q] : ~0ull;
        for (int off = 16; off; off >>= 1) {
            u64 o = __shfl_xor_sync(FULLM, h, off);
            h = o < h ? o : h;
        }
        if (h != ~0ull)
            while (L < g.B && (1ull << (2 * (L + g.shift))) < h) L++;
    }
    while (__any_sync(FULLM, todo)) {
        int sh = 3 * L;
        int cx = (int)compact3(c0 >> sh), cy = (int)compact3(c0 >> (sh + 1)),
            cz = (int)compact3(c0 >> (sh + 2));
        if (L >= g.B) cx = cy = cz = 0;
        int o = lane < 27 ? kCellOrder[lane] : 13;
        int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
        uint32_t rb = 0, re = 0;
        int rl = L, rt = 0;
        if (lane < 27) rt = resolve_cell(g, L, cx + dx, cy + dy, cz + dz, rb, re, &rl);
        for (int j = 0; j < 27; j++) {  // a coarse leaf reached from two cells is scanned once
            uint32_t bj = __shfl_sync(FULLM, rb, j);
            int tj = __shfl_sync(FULLM, rt, j);
            if (j < lane && rt == 2 && tj == 2 && bj == rb) rt = 0;
        }
        int bx = 0, by = 0, bz = 0;
        if (rt) {
            bx = (cx + dx) >> (rl - L);
            by = (cy + dy) >> (rl - L);
            bz = (cz + dz) >> (rl - L);
        }
        // 32-bit distances and packed lists when every range of this level is
        // within 3 cells of 2^13 mm (squared distances < 3 * 24576^2 < 2^32)
        bool pack = __all_sync(FULLM, !rt || rl + g.shift <= 13);
        if (pack)
            knn_level<S, FILT, W, TopPack<S, W>, true>(g, a, L, R, q, qp, ux, uy, uz, todo, tp, ti,
                                                       tpmax, lane, sub, lpq, rt, rb, re, rl, bx, by, bz,
                                                       cx, cy, cz, sp, sk, so, wpairs);
        else
            knn_level<S, FILT, W, TopList<S, W>, false>(g, a, L, R, q, qp, ux, uy, uz, todo, tp,
                                                        ti, tpmax, lane, sub, lpq, rt, rb, re, rl, bx, by,
                                                        bz, cx, cy, cz, sp, sk, so, wpairs);
        L++;
    }
    // spread over PD_PAIR_SLOTS counters by SM (one address would serialise
    // in L2; the SM id is read here, so it holds no register during the search)
    if (a.pairs_out && lane == 0 && wpairs) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        atomicAdd(&a.pairs_out[smid % PD_PAIR_SLOTS], wpairs);
    }
}

// The first full pass of the density path (S = 8, no weights) is held to 64
// registers for 8 blocks per SM: more warps in flight measured faster than
// the few bytes it spills (first pass of the 100M-point scan 70.4 -> 67.1 ms).
template <int S, int FILT, bool W, bool LIST>
__global__ void __launch_bounds__(PD_WARPS * 32, (S == 8 && !W && !LIST) ? 8 : 1)
    knn_kernel(GridView g, KnnArgs a) {
    __shared__ int4 s_p[PD_WARPS][32];
    __shared__ u64 s_k[PD_WARPS][32];
    __shared__ int s_o[PD_WARPS][32];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (LIST) {  // persistent over the listed groups
        int ng = *a.gcount;
        for (int t = blockIdx.x * PD_WARPS + w; t < ng; t += gridDim.x * PD_WARPS)
            knn_group<S, FILT, W>(g, a, a.glist[t], s_p[w], s_k[w], s_o[w], lane);
    } else {
        int gid = blockIdx.x * PD_WARPS + w;
        if (gid < a.ngroups) knn_group<S, FILT, W>(g, a, gid, s_p[w], s_k[w], s_o[w], lane);
    }
}

// Sparse re-searches: the listed queries (Morton positions, list[0 .. *count))
// run SP_SLOTS to a warp, SP_LANES lanes per query, each query over the
// 3x3x3 cells of its own leaf level.  The lanes of a query resolve its 27
// cells (every SP_LANES-th one) into shared memory; a coarse leaf reached
// from two cells is kept once.  Each lane then walks the staged ranges on its
// own, taking positions b + sub, b + sub + SP_LANES, ... of every range whose
// box is not beyond its own partial bound (never closer than the merged one;
// the smallest box distance it skipped bounds the reported horizon), and
// keeps a partial list; the partial lists merge once per level.  Lists are
// packed (one 64-bit key per entry, 32-bit distances) when every range of the
// warp's level lies within 3 cells of 2^13 mm.  Used for the re-searches of
// the removal rounds, where the flagged queries are few per leaf group and a
// warp per group would idle most lanes.  2 lanes per query (16 queries per
// warp) measured faster than 4 or 8 and level with 1.
#define SP_LANES 2
#define SP_SLOTS (32 / SP_LANES)

template <int S, bool W, class TL, bool PACK>
__device__ __forceinline__ void sparse_level(const GridView& g, const KnnArgs& a, int R, int q,
                                             int4 qp, int ux, int uy, int uz, int L, int cx,
                                             int cy, int cz, int sub, bool& todo,
                                             const uint32_t* __restrict__ sb,
                                             const uint32_t* __restrict__ se,
                                             const uint8_t* __restrict__ sl) {
    TL top;
    top.init();
    u64 hzl = ~0ull;
    if (todo) {
        for (int r = 0; r < 27; r++) {
            const int lv = sl[r];
            if (lv == 0xff) continue;
            const uint32_t b = sb[r], e = se[r];
            const int o = kCellOrder[r];
            const int sh = lv - L;
            const u64 bd = box_d2(ux, uy, uz, (cx + o % 3 - 1) >> sh, (cy + (o / 3) % 3 - 1) >> sh,
                                  (cz + o / 9 - 1) >> sh, lv + g.shift);
            const u64 bound = top.at(R - 1);
            if (bound != ~0ull && bd > bound) {
                if (bd < hzl) hzl = bd;
                continue;
            }
            // 4 candidates per lane and step, their loads issued together
            for (uint32_t j0 = b + sub; j0 < e; j0 += 4 * SP_LANES) {
                int4 v4[4];
                bool ok[4];
#pragma unroll
                for (int w = 0; w < 4; w++) {
                    const uint32_t j = j0 + (uint32_t)(w * SP_LANES);
                    ok[w] = j < e && (int)j != q;
                    v4[w] = ok[w] ? g.pos[j] : make_int4(0, 0, 0, 0);
                    if (ok[w] && a.alive) ok[w] = a.alive[j] != 0;
                }
#pragma unroll
                for (int w = 0; w < 4; w++) {
                    if (!ok[w]) continue;
                    const int j = (int)(j0 + (uint32_t)(w * SP_LANES));
                    u64 dd;
                    if (PACK) {
                        const int dx = v4[w].x - qp.x, dy = v4[w].y - qp.y, dz = v4[w].z - qp.z;
                        dd = (u64)((uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz));
                    } else {
                        const long long dx = (long long)v4[w].x - qp.x,
                                        dy = (long long)v4[w].y - qp.y,
                                        dz = (long long)v4[w].z - qp.z;
                        dd = (u64)(dx * dx + dy * dy + dz * dz);
                    }
                    const int co = W ? v4[w].w : j;
                    if (top.beats_last(dd, j, co)) top.insert(dd, j, co);
                }
            }
        }
    }
    // merge the 4 partial lists and horizons of each query (all lanes take part)
    for (int off = SP_LANES >> 1; off >= 1; off >>= 1) {
        top.merge_xor(off, todo);
        const u64 ho = __shfl_xor_sync(FULLM, hzl, off);
        hzl = ho < hzl ? ho : hzl;
    }
    if (todo) {
        const u64 gg = L >= g.B ? ~0ull : gap2(g, ux, uy, uz, L, cx, cy, cz);
        const u64 bound = top.at(R - 1);
        if (gg == ~0ull || bound < gg) {
            todo = false;
            if (sub == 0) write_result<S, FILT_NONE, W>(a, q, top, hzl < gg ? hzl : gg);
        }
    }
}

template <int S, bool W>
__global__ void __launch_bounds__(PD_WARPS * 32) knn_sparse_kernel(GridView g, KnnArgs a,
                                                                  const int* __restrict__ list,
                                                                  const int* __restrict__ count) {
    __shared__ uint32_t s_b[PD_WARPS][SP_SLOTS][27], s_e[PD_WARPS][SP_SLOTS][27];
    __shared__ uint8_t s_l[PD_WARPS][SP_SLOTS][28];
    const int lane = threadIdx.x & 31, sub = lane & (SP_LANES - 1), slot = lane / SP_LANES;
    const int w = threadIdx.x >> 5;
    uint32_t* sb = s_b[w][slot];
    uint32_t* se = s_e[w][slot];
    uint8_t* sl = s_l[w][slot];
    const int nq = *count;
    const int wid = blockIdx.x * PD_WARPS + w;
    const int nwarps = gridDim.x * PD_WARPS;
    const int R = a.r_exact > 0 && a.r_exact < S ? a.r_exact : S;
    for (int base = wid * SP_SLOTS; base < nq; base += nwarps * SP_SLOTS) {  // warp-uniform
        const int qs = base + slot;
        const int q = qs < nq ? list[qs] : -1;
        bool todo = q >= 0;
        int4 qp = make_int4(0, 0, 0, 0);
        u64 c0 = 0;
        int L = 0;
        if (todo) {
            qp = g.pos[q];
            c0 = g.code[q];
            L = g.leaf[q];
        }
        const int ux = qp.x - g.origin.x, uy = qp.y - g.origin.y, uz = qp.z - g.origin.z;
        while (__any_sync(FULLM, todo)) {
            int cx = 0, cy = 0, cz = 0;
            if (L < g.B) {
                cx = (int)compact3(c0 >> (3 * L));
                cy = (int)compact3(c0 >> (3 * L + 1));
                cz = (int)compact3(c0 >> (3 * L + 2));
            }
            // resolve the 27 cells into shared memory, the lanes of a query
            // taking every SP_LANES-th one
            bool small = true;  // every range of this lane within 3 cells of 2^13 mm
            if (todo) {
                const int lim = 1 << (g.B - L);  // todo lanes have L < B or L == B
                for (int r = sub; r < 27; r += SP_LANES) {
                    const int o = kCellOrder[r];
                    const int ex = cx + o % 3 - 1, ey = cy + (o / 3) % 3 - 1, ez = cz + o / 9 - 1;
                    uint32_t b = 0, e = 0;
                    int rl = L;
                    int rt = resolve_cell(g, L, ex, ey, ez, b, e, &rl);
                    if (rt == 2) {
                        // a coarse leaf covers every cell that agrees with this one
                        // above its level: keep it at the first such cell only
                        const int sh = rl - L;
                        for (int r2 = 0; r2 < r; r2++) {
                            const int o2 = kCellOrder[r2];
                            const int fx = cx + o2 % 3 - 1, fy = cy + (o2 / 3) % 3 - 1,
                                      fz = cz + o2 / 9 - 1;
                            if (fx < 0 || fy < 0 || fz < 0 || fx >= lim || fy >= lim || fz >= lim)
                                continue;
                            if ((fx >> sh) == (ex >> sh) && (fy >> sh) == (ey >> sh) &&
                                (fz >> sh) == (ez >> sh)) {
                                rt = 0;
                                break;
                            }
                        }
                    }
                    sb[r] = b;
                    se[r] = e;
                    sl[r] = rt ? (uint8_t)rl : (uint8_t)0xff;
                    if (rt && rl + g.shift > 13) small = false;
                }
            }
            const bool pack = __all_sync(FULLM, small);
            __syncwarp();
            if (pack)
                sparse_level<S, W, TopPack<S, W>, true>(g, a, R, q, qp, ux, uy, uz, L, cx, cy, cz,
                                                        sub, todo, sb, se, sl);
            else
                sparse_level<S, W, TopList<S, W>, false>(g, a, R, q, qp, ux, uy, uz, L, cx, cy,
                                                         cz, sub, todo, sb, se, sl);
            __syncwarp();
            L++;
        }
    }
}

// One warp per aligned chunk of 32 Morton positions: the least live key primary.
__global__ void chunk_min_kernel(const u64* __restrict__ prim, const uint8_t* __restrict__ alive,
                                 int64_t n, u64* cmin) {
    int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int64_t nc = (n + 31) >> 5;
    if (c >= nc) return;  // whole warps leave together
    int64_t j = c * 32 + lane;
    u64 v = (j < n && alive[j]) ? prim[j] : ~0ull;
    for (int off = 16; off; off >>= 1) {
        u64 o = __shfl_xor_sync(FULLM, v, off);
        v = o < v ? o : v;
    }
    if (lane == 0) cmin[c] = v;
}

// Append every group holding a flagged query to glist (one atomic per warp).
__global__ void flagged_groups_kernel(const int4* __restrict__ groups, int ngroups,
                                      const uint8_t* __restrict__ qflag, int* glist, int* gcount) {
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    bool any = false;
    if (gid < ngroups) {
        int4 G = groups[gid];
        for (int i = 0; i < G.y && !any; i++) any = qflag[G.x + i] != 0;
    }
    const int slot = block_append(any, gcount);
    if (any) glist[slot] = gid;
}

template <int S, int FILT>
static cudaError_t launch_knn_t(const GridView& g, const KnnArgs& a, cudaStream_t st) {
    if (a.ngroups <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((a.ngroups + PD_WARPS - 1) / PD_WARPS);
    // list mode: a persistent grid (about 6 resident blocks per SM)
    if (a.glist && blocks > (unsigned)device_sms() * 6u) blocks = (unsigned)device_sms() * 6u;
    if (a.glist) {
        if (a.term != 0)
            knn_kernel<S, FILT, true, true><<<blocks, PD_WARPS * 32, 0, st>>>(g, a);
        else
            knn_kernel<S, FILT, false, true><<<blocks, PD_WARPS * 32, 0, st>>>(g, a);
    } else if (FILT == FILT_NONE) {  // full passes: one warp per group
        if (a.term != 0)
            knn_kernel<S, FILT_NONE, true, false><<<blocks, PD_WARPS * 32, 0, st>>>(g, a);
        else
            knn_kernel<S, FILT_NONE, false, false><<<blocks, PD_WARPS * 32, 0, st>>>(g, a);
    } else {
        return cudaErrorInvalidValue;  // filtered searches always run over a group list
    }
    note_launch();
    return cudaGetLastError();
}

template <int S>
static cudaError_t launch_knn_s(const GridView& g, const KnnArgs& a, cudaStream_t st) {
    switch (a.filter) {
        case FILT_NONE: return launch_knn_t<S, FILT_NONE>(g, a, st);
        case FILT_BELOW_SELF: return launch_knn_t<S, FILT_BELOW_SELF>(g, a, st);
        default: return launch_knn_t<S, FILT_BELOW_TAU>(g, a, st);
    }
}

cudaError_t launch_chunk_min(const u64* prim, const uint8_t* alive, int64_t n, u64* cmin,
                             cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t threads = ((n + 31) >> 5) * 32;
    chunk_min_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(prim, alive, n, cmin);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_knn_flagged(const GridView& g, const KnnArgs& a, int* glist, int* gcount,
                               cudaStream_t st) {
    if (a.ngroups <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(gcount, 0, sizeof(int), st);
    if (e) return e;
    flagged_groups_kernel<<<(unsigned)((a.ngroups + 255) / 256), 256, 0, st>>>(
        a.groups, a.ngroups, a.qflag, glist, gcount);
    note_launch();
    KnnArgs b = a;
    b.glist = glist;
    b.gcount = gcount;
    return launch_knn(g, b, st);
}

template <int S>
static cudaError_t launch_sparse_s(const GridView& g, const KnnArgs& a, const int* list,
                                   const int* count, int64_t cap, cudaStream_t st) {
    int64_t warps = (cap + 32 / SP_LANES - 1) / (32 / SP_LANES);
    int64_t blocks = (warps + PD_WARPS - 1) / PD_WARPS;
    int64_t lim = (int64_t)device_sms() * 12;
    if (blocks > lim) blocks = lim;
    if (blocks < 1) blocks = 1;
    if (a.term != 0)
        knn_sparse_kernel<S, true><<<(unsigned)blocks, PD_WARPS * 32, 0, st>>>(g, a, list, count);
    else
        knn_sparse_kernel<S, false><<<(unsigned)blocks, PD_WARPS * 32, 0, st>>>(g, a, list, count);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_knn_sparse(const GridView& g, const KnnArgs& a, const int* list,
                              const int* count, int64_t cap, cudaStream_t st) {
    if (a.filter != FILT_NONE || cap <= 0) return cap <= 0 ? cudaSuccess : cudaErrorInvalidValue;
    switch (a.S) {
        case 4: return launch_sparse_s<4>(g, a, list, count, cap, st);
        case 8: return launch_sparse_s<8>(g, a, list, count, cap, st);
        case 17: return launch_sparse_s<17>(g, a, list, count, cap, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_knn(const GridView& g, const KnnArgs& a, cudaStream_t st) {
    switch (a.S) {
        case 4: return launch_knn_s<4>(g, a, st);
        case 8: return launch_knn_s<8>(g, a, st);
        case 17: return launch_knn_s<17>(g, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pd
