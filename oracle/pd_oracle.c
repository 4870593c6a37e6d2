/*
 * pd_oracle.c -- CPU oracle for greedy kNN-cost point-cloud decimation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, calls or
 * executes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA library.
 *
 * What it computes (Comino-Trinidad, Chica, Andujar, "Revisiting Poisson-disk
 * Subsampling for Massive Point Cloud Decimation", arXiv 2311.17604):
 *
 *   - Problem statement (Eq. 1): keep a subset C' of C with |C'| = m points.
 *   - Cost of a point p (Eq. 10 for k = 1, Eq. 11 for k >= 2):
 *         w_p^k = sum over the k nearest other live points p' of 1 / d(p,p')^2
 *     Coordinates are int32 millimetres, squared distances are exact int64.
 *       * k = 1, density only: the cost order is the order of d1^2 ascending,
 *         compared as integers (no floating point at all).
 *       * otherwise: c = 0.0; for i = 1..k (d_1^2 <= ... <= d_k^2):
 *             c = c + w_i / (double)d_i^2
 *         in IEEE binary64 round-to-nearest, in exactly that order, with
 *         w_i = 1 for the density cost.  d^2 = 0 gives +inf.  Fewer than k
 *         other live points: the missing terms contribute nothing.
 *   - Optional per-neighbour weights (section "Additional cost terms", Eq. 13
 *     and the colour-deviation term, for which the paper prints no formula):
 *         orientation  w = 1 - a * (1 - |n_p . n_q|)
 *         colour       w = 1 - a * ||rgb_p - rgb_q||_2 / (255 * sqrt(3))
 *     Both weights are readings of the paper (it gives no colour formula,
 *     and the orientation term is read with |n_p . n_q| for unoriented
 *     normals).  The tests pin them to hand-worked clouds whose costs follow
 *     in closed form: identical colours weigh 1, black against white 1 - a,
 *     a pure red difference 1 - a / sqrt 3; parallel and antiparallel
 *     normals 1, orthogonal ones 1 - a, a 60 degree angle 1 - a / 2.
 *   - Greedy removal (section "Computing per-sample costs", after Eq. 7, and
 *     section "Sub-sampling algorithm", step 2): repeatedly remove the live
 *     point with the largest key (cost, index) -- among equal costs the larger
 *     input index goes first -- and recompute the cost of every live point
 *     whose stored k nearest neighbours contained the removed point (the set
 *     N(p) of step 2), until m points remain.  A max binary heap with
 *     per-point version stamps holds the keys; stale entries are skipped.
 *
 * Neighbour search backends (both exact, both skip removed points):
 *   ORC_BRUTE   every other live point is examined (the definition);
 *   ORC_KDTREE  a static kd-tree over the points (the paper's search
 *               structure, abstract and section "Scaling to massive point
 *               clouds"), pruned by bounding-box distance, rebuilt over the
 *               live points whenever half of them have been removed.
 * Stored neighbours are the k smallest (d^2, index) pairs in lexicographic
 * order, so both backends store identical lists.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BRUTE 0
#define ORC_KDTREE 1

#define ORC_TERM_NONE 0
#define ORC_TERM_COLOR 1
#define ORC_TERM_ORIENT 2

#define ORC_KMAX 32
#define D2_NONE INT64_MAX

/* ------------------------------------------------------------------------ */
/* geometry                                                                   */
/* ------------------------------------------------------------------------ */

static inline int64_t sqdist(const int32_t* a, const int32_t* b) {
    int64_t dx = (int64_t)a[0] - b[0];
    int64_t dy = (int64_t)a[1] - b[1];
    int64_t dz = (int64_t)a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

/* Insert (d2, j) into the ascending list (d2s, ids) of length *cnt <= k. */
static inline void topk_insert(int64_t* d2s, int32_t* ids, int* cnt, int k,
                               int64_t d2, int32_t j) {
    int c = *cnt;
    if (c == k) {
        if (d2 > d2s[k - 1] || (d2 == d2s[k - 1] && j > ids[k - 1])) return;
        c = k - 1; /* drop the current worst */
    }
    int pos = c;
    while (pos > 0 && (d2s[pos - 1] > d2 || (d2s[pos - 1] == d2 && ids[pos - 1] > j))) {
        d2s[pos] = d2s[pos - 1];
        ids[pos] = ids[pos - 1];
        pos--;
    }
    d2s[pos] = d2;
    ids[pos] = j;
    *cnt = c + 1;
}

/* ------------------------------------------------------------------------ */
/* kd-tree                                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t lo[3], hi[3];
    int64_t begin, end;
    int64_t left, right; /* -1 for leaves */
} kd_node;

typedef struct {
    const int32_t* xyz;
    int64_t* perm;
    kd_node* nodes;
    int64_t nnodes, cap;
} kd_tree;

#define KD_LEAF 8

static int kd_less(const int32_t* xyz, int ax, int64_t a, int64_t b) {
    int32_t va = xyz[3 * a + ax], vb = xyz[3 * b + ax];
    return va < vb || (va == vb && a < b);
}

/* Rearrange perm[lo, hi) so that perm[nth] is the element of rank nth. */
static void kd_select(const int32_t* xyz, int ax, int64_t* perm, int64_t lo, int64_t hi,
                      int64_t nth) {
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        /* median of three as pivot */
        int64_t a = perm[lo], b = perm[mid], c = perm[hi - 1], piv;
        if (kd_less(xyz, ax, a, b)) {
            if (kd_less(xyz, ax, b, c)) piv = b;
            else if (kd_less(xyz, ax, a, c)) piv = c;
            else piv = a;
        } else {
            if (kd_less(xyz, ax, a, c)) piv = a;
            else if (kd_less(xyz, ax, b, c)) piv = c;
            else piv = b;
        }
        /* three-way partition around piv */
        int64_t lt = lo, i = lo, gt = hi;
        while (i < gt) {
            int64_t e = perm[i];
            if (kd_less(xyz, ax, e, piv)) {
                perm[i] = perm[lt]; perm[lt] = e; lt++; i++;
            } else if (kd_less(xyz, ax, piv, e)) {
                gt--; perm[i] = perm[gt]; perm[gt] = e;
            } else {
                i++;
            }
        }
        if (nth < lt) hi = lt;
        else if (nth >= gt) lo = gt;
        else return;
    }
}

static int64_t kd_new_node(kd_tree* t) {
    if (t->nnodes == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->nodes = (kd_node*)realloc(t->nodes, (size_t)t->cap * sizeof(kd_node));
    }
    return t->nnodes++;
}

static int64_t kd_build_rec(kd_tree* t, int64_t begin, int64_t end) {
    int64_t id = kd_new_node(t);
    kd_node nd;
    nd.begin = begin;
    nd.end = end;
    nd.left = nd.right = -1;
    for (int a = 0; a < 3; a++) { nd.lo[a] = INT32_MAX; nd.hi[a] = INT32_MIN; }
    for (int64_t i = begin; i < end; i++) {
        const int32_t* p = t->xyz + 3 * t->perm[i];
        for (int a = 0; a < 3; a++) {
            if (p[a] < nd.lo[a]) nd.lo[a] = p[a];
            if (p[a] > nd.hi[a]) nd.hi[a] = p[a];
        }
    }
    if (end - begin > KD_LEAF) {
        int ax = 0;
        int64_t w0 = (int64_t)nd.hi[0] - nd.lo[0], w1 = (int64_t)nd.hi[1] - nd.lo[1],
                w2 = (int64_t)nd.hi[2] - nd.lo[2];
        if (w1 > w0 && w1 >= w2) ax = 1;
        else if (w2 > w0 && w2 > w1) ax = 2;
        int64_t mid = begin + (end - begin) / 2;
        kd_select(t->xyz, ax, t->perm, begin, end, mid);
        int64_t l = kd_build_rec(t, begin, mid);
        int64_t r = kd_build_rec(t, mid, end);
        nd.left = l;
        nd.right = r;
    }
    t->nodes[id] = nd;
    return id;
}

/* Build over the points i with live[i] != 0 (all points if live == NULL). */
static void kd_build(kd_tree* t, const int32_t* xyz, int64_t n, const uint8_t* live) {
    t->xyz = xyz;
    t->nnodes = 0;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; i++)
        if (!live || live[i]) t->perm[cnt++] = i;
    if (cnt > 0) kd_build_rec(t, 0, cnt);
}

static inline int64_t box_d2(const kd_node* nd, const int32_t* q) {
    int64_t s = 0;
    for (int a = 0; a < 3; a++) {
        int64_t d = 0;
        if (q[a] < nd->lo[a]) d = (int64_t)nd->lo[a] - q[a];
        else if (q[a] > nd->hi[a]) d = (int64_t)q[a] - nd->hi[a];
        s += d * d;
    }
    return s;
}

/* k nearest live points other than q; returns how many were found. */
static int kd_knn(const kd_tree* t, const uint8_t* live, int64_t q, int k,
                  int64_t* d2s, int32_t* ids) {
    int cnt = 0;
    if (t->nnodes == 0) return 0;
    const int32_t* qp = t->xyz + 3 * q;
    int64_t stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const kd_node* nd = &t->nodes[stack[--sp]];
        if (cnt == k && box_d2(nd, qp) > d2s[k - 1]) continue;
        if (nd->left < 0) {
            for (int64_t i = nd->begin; i < nd->end; i++) {
                int64_t j = t->perm[i];
                if (j == q || !live[j]) continue;
                topk_insert(d2s, ids, &cnt, k, sqdist(qp, t->xyz + 3 * j), (int32_t)j);
            }
        } else {
            const kd_node* L = &t->nodes[nd->left];
            const kd_node* R = &t->nodes[nd->right];
            int64_t dl = box_d2(L, qp), dr = box_d2(R, qp);
            /* push the farther child first so the nearer one is visited first */
            if (dl <= dr) { stack[sp++] = nd->right; stack[sp++] = nd->left; }
            else { stack[sp++] = nd->left; stack[sp++] = nd->right; }
        }
    }
    return cnt;
}

static int brute_knn(const int32_t* xyz, int64_t n, const uint8_t* live, int64_t q, int k,
                     int64_t* d2s, int32_t* ids) {
    int cnt = 0;
    const int32_t* qp = xyz + 3 * q;
    for (int64_t j = 0; j < n; j++) {
        if (j == q || !live[j]) continue;
        topk_insert(d2s, ids, &cnt, k, sqdist(qp, xyz + 3 * j), (int32_t)j);
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* cost                                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int k, term;
    double a; /* weight of the colour / orientation term */
    const uint8_t* rgb;
    const float* nrm;
} cost_cfg;

/* Integer ordering is used exactly when the cost is the plain k = 1 density. */
static inline int int_mode(const cost_cfg* c) { return c->k == 1 && c->term == ORC_TERM_NONE; }

static double nbr_weight(const cost_cfg* c, int64_t p, int64_t q) {
    if (c->term == ORC_TERM_COLOR) {
        const uint8_t* a = c->rgb + 3 * p;
        const uint8_t* b = c->rgb + 3 * q;
        double dr = (double)a[0] - (double)b[0];
        double dg = (double)a[1] - (double)b[1];
        double db = (double)a[2] - (double)b[2];
        double s = dr * dr;
        s = s + dg * dg;
        s = s + db * db;
        double dist = sqrt(s);
        double scale = 255.0 * sqrt(3.0);
        return 1.0 - c->a * (dist / scale);
    }
    if (c->term == ORC_TERM_ORIENT) {
        const float* a = c->nrm + 3 * p;
        const float* b = c->nrm + 3 * q;
        double d = (double)a[0] * (double)b[0];
        d = d + (double)a[1] * (double)b[1];
        d = d + (double)a[2] * (double)b[2];
        return 1.0 - c->a * (1.0 - fabs(d));
    }
    return 1.0;
}

/* Eq. 11 (with optional weights): sum in ascending-distance order. */
static double cost_of(const cost_cfg* c, int64_t p, const int64_t* d2s, const int32_t* ids,
                      int cnt) {
    double s = 0.0;
    for (int i = 0; i < cnt; i++) {
        double w = nbr_weight(c, p, ids[i]);
        s = s + w / (double)d2s[i];
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* binary max-heap of keys                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    double c;    /* cost (used unless integer mode) */
    int64_t d2;  /* d1^2 (integer mode); D2_NONE = no neighbour */
    int32_t idx;
    uint32_t ver;
} hentry;

typedef struct {
    hentry* a;
    int64_t size, cap;
    int imode;
} heap_t;

/* 1 if key x is larger than key y. */
static inline int key_gt(int imode, const hentry* x, const hentry* y) {
    if (imode) {
        if (x->d2 != y->d2) return x->d2 < y->d2;
    } else {
        if (x->c != y->c) return x->c > y->c;
    }
    return x->idx > y->idx;
}

static void heap_push(heap_t* h, hentry e) {
    if (h->size == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->a = (hentry*)realloc(h->a, (size_t)h->cap * sizeof(hentry));
    }
    int64_t i = h->size++;
    while (i > 0) {
        int64_t par = (i - 1) / 2;
        if (!key_gt(h->imode, &e, &h->a[par])) break;
        h->a[i] = h->a[par];
        i = par;
    }
    h->a[i] = e;
}

static hentry heap_pop(heap_t* h) {
    hentry top = h->a[0];
    hentry last = h->a[--h->size];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, best = i;
        const hentry* bv = &last;
        if (l < h->size && key_gt(h->imode, &h->a[l], bv)) { best = l; bv = &h->a[l]; }
        if (r < h->size && key_gt(h->imode, &h->a[r], bv)) { best = r; }
        if (best == i) break;
        h->a[i] = h->a[best];
        i = best;
    }
    if (h->size > 0) h->a[i] = last;
    return top;
}

/* ------------------------------------------------------------------------ */
/* public entry points                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    const int32_t* xyz;
    int64_t n;
    int backend;
    kd_tree tree;
    int64_t tree_live; /* live count when the tree was (re)built */
} searcher;

static void searcher_init(searcher* s, const int32_t* xyz, int64_t n, int backend,
                          const uint8_t* live) {
    memset(s, 0, sizeof(*s));
    s->xyz = xyz;
    s->n = n;
    s->backend = backend;
    if (backend == ORC_KDTREE) {
        s->tree.perm = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        kd_build(&s->tree, xyz, n, live);
        int64_t c = 0;
        for (int64_t i = 0; i < n; i++) c += live ? (live[i] != 0) : 1;
        s->tree_live = c;
    }
}

static void searcher_free(searcher* s) {
    free(s->tree.perm);
    free(s->tree.nodes);
}

static int searcher_knn(const searcher* s, const uint8_t* live, int64_t q, int k, int64_t* d2s,
                        int32_t* ids) {
    if (s->backend == ORC_KDTREE) return kd_knn(&s->tree, live, q, k, d2s, ids);
    return brute_knn(s->xyz, s->n, live, q, k, d2s, ids);
}

static int check_args(const int32_t* xyz, int64_t n, int k, int term, const uint8_t* rgb,
                      const float* nrm) {
    if (!xyz || n < 0 || k < 1 || k > ORC_KMAX) return -1;
    if (term == ORC_TERM_COLOR && !rgb) return -1;
    if (term == ORC_TERM_ORIENT && !nrm) return -1;
    if (term < 0 || term > 2) return -1;
    if (n > INT32_MAX) return -1;
    return 0;
}

/*
 * k nearest live neighbours and the cost of every live point.
 *   live     n flags (NULL = all live); removed points are neither queried
 *            nor returned as neighbours.
 *   d2_out   n*k int64, ascending; D2_NONE where fewer than k exist.
 *   idx_out  n*k int32 (-1 where missing).  May be NULL.
 *   cost_out n doubles (Eq. 10/11 with optional weights; for the plain
 *            k = 1 density this is 1.0 / d1^2 for reporting only).  May be NULL.
 * Queries run in parallel when compiled with OpenMP (they are independent).
 */
int orc_knn_cost(const int32_t* xyz, const uint8_t* rgb, const float* nrm, int64_t n,
                 const uint8_t* live, int k, int term, double a, int backend,
                 int64_t* d2_out, int32_t* idx_out, double* cost_out) {
    if (check_args(xyz, n, k, term, rgb, nrm) || !d2_out) return -1;
    uint8_t* lv = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) lv[i] = live ? (live[i] != 0) : 1;
    searcher s;
    searcher_init(&s, xyz, n, backend, lv);
    cost_cfg cc = {k, term, a, rgb, nrm};
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t q = 0; q < n; q++) {
        int64_t d2s[ORC_KMAX];
        int32_t ids[ORC_KMAX];
        int cnt = 0;
        if (lv[q]) cnt = searcher_knn(&s, lv, q, k, d2s, ids);
        for (int i = 0; i < k; i++) {
            d2_out[q * k + i] = i < cnt ? d2s[i] : D2_NONE;
            if (idx_out) idx_out[q * k + i] = i < cnt ? ids[i] : -1;
        }
        if (cost_out) {
            if (!lv[q]) cost_out[q] = 0.0;
            else cost_out[q] = cost_of(&cc, q, d2s, ids, cnt);
        }
    }
    searcher_free(&s);
    free(lv);
    return 0;
}

/* Per-point dynamic list of the points that store it as a neighbour. */
typedef struct {
    int32_t* v;
    int32_t n, cap;
} ivec;

static void ivec_push(ivec* a, int32_t x) {
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 4;
        a->v = (int32_t*)realloc(a->v, (size_t)a->cap * sizeof(int32_t));
    }
    a->v[a->n++] = x;
}

/*
 * Sequential greedy decimation to exactly m retained points.
 *   keep_out   n bytes: 1 = retained, 0 = removed.
 *   order_out  n - m ints (may be NULL): removal order.
 *   pkey_out   n - m doubles (may be NULL): cost of each removed point when it
 *              was removed (integer mode: d1^2 as a double, INFINITY if none).
 *   requeries  (may be NULL) number of neighbour re-searches performed.
 * Returns 0, or -1 on invalid arguments.
 */
int orc_decimate(const int32_t* xyz, const uint8_t* rgb, const float* nrm, int64_t n, int k,
                 int64_t m, int term, double a, int backend, uint8_t* keep_out,
                 int32_t* order_out, double* pkey_out, int64_t* requeries) {
    if (check_args(xyz, n, k, term, rgb, nrm) || !keep_out || m < 0 || m > n) return -1;
    cost_cfg cc = {k, term, a, rgb, nrm};
    int imode = int_mode(&cc);
    uint8_t* live = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    memset(live, 1, (size_t)n);
    int64_t* nd2 = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * k * sizeof(int64_t));
    int32_t* nid = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * k * sizeof(int32_t));
    int32_t* ncnt = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    double* cost = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    uint32_t* ver = (uint32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint32_t));
    uint32_t* mark = (uint32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(uint32_t));
    ivec* rev = (ivec*)calloc((size_t)(n > 0 ? n : 1), sizeof(ivec));
    int32_t* aff = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t nreq = 0;

    searcher s;
    searcher_init(&s, xyz, n, backend, live);

    /* initial costs of every point (independent queries) */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t q = 0; q < n; q++) {
        ncnt[q] = searcher_knn(&s, live, q, k, nd2 + q * k, nid + q * k);
        cost[q] = cost_of(&cc, q, nd2 + q * k, nid + q * k, ncnt[q]);
    }
    heap_t h = {NULL, 0, 0, imode};
    for (int64_t q = 0; q < n; q++) {
        for (int i = 0; i < ncnt[q]; i++) ivec_push(&rev[nid[q * k + i]], (int32_t)q);
        hentry e = {cost[q], ncnt[q] ? nd2[q * k] : D2_NONE, (int32_t)q, 0};
        heap_push(&h, e);
    }

    int64_t live_cnt = n, step = 0;
    while (live_cnt > m) {
        hentry top = heap_pop(&h);
        int32_t p = top.idx;
        if (!live[p] || top.ver != ver[p]) continue; /* stale entry */
        live[p] = 0;
        live_cnt--;
        if (order_out) order_out[step] = p;
        if (pkey_out) {
            if (imode) pkey_out[step] = top.d2 == D2_NONE ? INFINITY : (double)top.d2;
            else pkey_out[step] = top.c;
        }
        step++;
        if (s.backend == ORC_KDTREE && live_cnt > 0 && live_cnt * 2 < s.tree_live) {
            kd_build(&s.tree, xyz, n, live);
            s.tree_live = live_cnt;
        }
        /* affected points: live q whose stored neighbours contain p */
        int32_t na = 0;
        uint32_t stamp = (uint32_t)step;
        for (int32_t r = 0; r < rev[p].n; r++) {
            int32_t q = rev[p].v[r];
            if (!live[q] || mark[q] == stamp) continue;
            int hit = 0;
            for (int i = 0; i < ncnt[q]; i++) hit |= nid[q * k + i] == p;
            if (!hit) continue; /* stale reverse entry */
            mark[q] = stamp;
            aff[na++] = q;
        }
        free(rev[p].v);
        rev[p].v = NULL;
        rev[p].n = rev[p].cap = 0;
        for (int32_t t = 0; t < na; t++) {
            int32_t q = aff[t];
            ncnt[q] = searcher_knn(&s, live, q, k, nd2 + (int64_t)q * k, nid + (int64_t)q * k);
            nreq++;
            cost[q] = cost_of(&cc, q, nd2 + (int64_t)q * k, nid + (int64_t)q * k, ncnt[q]);
            for (int i = 0; i < ncnt[q]; i++) ivec_push(&rev[nid[(int64_t)q * k + i]], q);
            ver[q]++;
            hentry e = {cost[q], ncnt[q] ? nd2[(int64_t)q * k] : D2_NONE, q, ver[q]};
            heap_push(&h, e);
        }
    }
    for (int64_t i = 0; i < n; i++) keep_out[i] = live[i];
    if (requeries) *requeries = nreq;

    searcher_free(&s);
    for (int64_t i = 0; i < n; i++) free(rev[i].v);
    free(rev); free(aff); free(h.a); free(live); free(nd2); free(nid); free(ncnt);
    free(cost); free(ver); free(mark);
    return 0;
}

/* Number of threads the parallel loops use (1 without OpenMP). */
/*
 * Brute-force k nearest neighbours and density cost (Eq. 10/11, no weights)
 * of a few query points among all n points (every point live): the
 * definition, for spot checks of clouds too large for the greedy.
 *   queries  nq point indices.
 *   d2_out   nq*k int64, ascending (d^2, index); D2_NONE where missing.
 *   idx_out  nq*k int32 (-1 where missing).  May be NULL.
 *   cost_out nq doubles: sum of 1.0 / d_i^2 nearest first (+inf for a
 *            coincident neighbour).  May be NULL.
 * Queries run in parallel (each scans all n points).
 */
int orc_knn_query(const int32_t* xyz, int64_t n, const int64_t* queries, int64_t nq, int k,
                  int64_t* d2_out, int32_t* idx_out, double* cost_out) {
    if (!xyz || n < 0 || n > INT32_MAX || !queries || nq < 0 || k < 1 || k > ORC_KMAX ||
        !d2_out)
        return -1;
    for (int64_t t = 0; t < nq; t++)
        if (queries[t] < 0 || queries[t] >= n) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nq; t++) {
        int64_t d2s[ORC_KMAX];
        int32_t ids[ORC_KMAX];
        int cnt = 0;
        const int64_t q = queries[t];
        const int32_t* qp = xyz + 3 * q;
        for (int64_t j = 0; j < n; j++) {
            if (j == q) continue;
            int64_t d2 = sqdist(qp, xyz + 3 * j);
            if (cnt == k && d2 > d2s[k - 1]) continue;
            topk_insert(d2s, ids, &cnt, k, d2, (int32_t)j);
        }
        double c = 0.0;
        for (int i = 0; i < k; i++) {
            d2_out[t * k + i] = i < cnt ? d2s[i] : D2_NONE;
            if (idx_out) idx_out[t * k + i] = i < cnt ? ids[i] : -1;
            if (i < cnt) c = c + 1.0 / (double)d2s[i];
        }
        if (cost_out) cost_out[t] = c;
    }
    return 0;
}

/*
 * Neighbour counts of the quality report (section "Results and Discussion",
 * the cube experiment): for every point p and radius r_j,
 *     counts[p * nr + j] = #{q != p : d(p,q)^2 <= r2[j]}
 * by brute force over all n points (exact int64 squared distances).
 */
int orc_radius_counts(const int32_t* xyz, int64_t n, const int64_t* r2, int nr,
                      int64_t* counts) {
    if (!xyz || n < 0 || !r2 || nr < 1 || !counts) return -1;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < n; p++) {
        for (int j = 0; j < nr; j++) counts[p * nr + j] = 0;
        for (int64_t q = 0; q < n; q++) {
            if (q == p) continue;
            int64_t d2 = sqdist(xyz + 3 * p, xyz + 3 * q);
            for (int j = 0; j < nr; j++)
                if (d2 <= r2[j]) counts[p * nr + j]++;
        }
    }
    return 0;
}

/*
 * The paper's iterative scheme (section "Sub-sampling algorithm"), with its
 * sweep restated as parallel rounds so that a GPU can run it and reproduce it
 * exactly.  Density cost (Eq. 10/11), k nearest, a buffer of S >= k stored
 * neighbours (the k+b extended neighbourhood).  Until m points remain:
 *
 *   1. Cost updates: the S nearest live points, in (d^2, index) order, and
 *      the cost of every live point are recomputed exactly; no point is
 *      dirty.
 *   2. w_up = the m-th smallest key (cost, index) among the live points:
 *      the points above it are the live - m largest keys.
 *   3. Point removal, in rounds until no clean live point lies above w_up:
 *      a candidate is a clean live point whose key is above w_up; a
 *      candidate is removed when no other candidate adjacent to it has a
 *      larger key, adjacency meaning that one of the two lies among the k
 *      first stored neighbours of the other.  Every live point that stored
 *      a removed point drops it; with at least k stored points left its
 *      cost is recomputed from the first k of them (the stored points are
 *      the nearest live points, ties aside, so that cost is exact), with
 *      fewer it is flagged dirty and is not removed before the next
 *      iteration's cost update.
 *
 * The paper sweeps its voxels in order, removing every point above w_up
 * and updating its reverse neighbours as it goes; here all non-interacting
 * removals of a sweep happen at once, the largest key first among
 * interacting ones.  Removals never raise a cost, so at most live - m
 * points leave per iteration (never fewer than m remain) and at least one
 * leaves (the largest key is never blocked).
 *   keep_out    n bytes.  iters_out, rounds_out: may be NULL.
 *   round_log   (may be NULL) per round: (iteration << 40) | points removed,
 *               the first log_cap rounds.
 * Returns 0, or -1 on invalid arguments (k in [1, S], S <= ORC_KMAX).
 */
static inline int keygt(double ca, int32_t ia, double cb, int32_t ib) {
    return ca > cb || (ca == cb && ia > ib);
}

typedef struct {
    double c;
    int32_t i;
} ckey;

/* descending key order */
static int ckey_cmp(const void* a, const void* b) {
    const ckey* x = (const ckey*)a;
    const ckey* y = (const ckey*)b;
    if (keygt(x->c, x->i, y->c, y->i)) return -1;
    if (keygt(y->c, y->i, x->c, x->i)) return 1;
    return 0;
}

int orc_decimate_wup(const int32_t* xyz, int64_t n, int k, int S, int64_t m, int backend,
                     uint8_t* keep_out, int32_t* iters_out, int64_t* rounds_out,
                     int64_t* round_log, int64_t log_cap) {
    if (!xyz || n < 0 || n > INT32_MAX || k < 1 || S < k || S > ORC_KMAX || !keep_out ||
        m < 0 || m > n)
        return -1;
    const int64_t N = n > 0 ? n : 1;
    uint8_t* live = (uint8_t*)malloc((size_t)N);
    uint8_t* dirty = (uint8_t*)malloc((size_t)N);
    uint8_t* cand = (uint8_t*)malloc((size_t)N);
    uint8_t* pick = (uint8_t*)malloc((size_t)N);
    int64_t* nd2 = (int64_t*)malloc((size_t)N * S * sizeof(int64_t));
    int32_t* nid = (int32_t*)malloc((size_t)N * S * sizeof(int32_t));
    int32_t* ncnt = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    double* cost = (double*)malloc((size_t)N * sizeof(double));
    double* bc = (double*)malloc((size_t)N * sizeof(double));  /* largest adjacent key: cost */
    int32_t* bi = (int32_t*)malloc((size_t)N * sizeof(int32_t)); /* ... and index */
    ckey* order = (ckey*)malloc((size_t)N * sizeof(ckey));
    memset(live, 1, (size_t)n);
    int64_t nlive = n, rounds = 0;
    int32_t iters = 0;
    cost_cfg cc = {k, ORC_TERM_NONE, 0.0, NULL, NULL};
    while (nlive > m) {
        iters++;
        /* 1. exact S nearest and cost of every live point */
        searcher sr;
        searcher_init(&sr, xyz, n, backend, live);
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t q = 0; q < n; q++) {
            if (!live[q]) continue;
            ncnt[q] = searcher_knn(&sr, live, q, S, nd2 + q * S, nid + q * S);
            cost[q] = cost_of(&cc, q, nd2 + q * S, nid + q * S, ncnt[q] < k ? ncnt[q] : k);
            dirty[q] = 0;
        }
        searcher_free(&sr);
        /* 2. w_up: the (nlive - m)-th largest key is the smallest one above it */
        int64_t nl = 0;
        for (int64_t q = 0; q < n; q++)
            if (live[q]) {
                order[nl].c = cost[q];
                order[nl].i = (int32_t)q;
                nl++;
            }
        qsort(order, (size_t)nl, sizeof(ckey), ckey_cmp);
        const double tc = order[nlive - m - 1].c;
        const int32_t ti = order[nlive - m - 1].i;
        /* 3. rounds of removals above w_up */
        for (;;) {
            int64_t nc = 0;
            for (int64_t q = 0; q < n; q++) {
                cand[q] = live[q] && !dirty[q] && !keygt(tc, ti, cost[q], (int32_t)q);
                nc += cand[q];
                bc[q] = -1.0;
                bi[q] = -1;
            }
            if (!nc) break;
            /* the largest candidate key that stores each point among its first k */
            for (int64_t q = 0; q < n; q++) {
                if (!cand[q]) continue;
                int lim = ncnt[q] < k ? ncnt[q] : k;
                for (int i = 0; i < lim; i++) {
                    int32_t x = nid[q * S + i];
                    if (keygt(cost[q], (int32_t)q, bc[x], bi[x])) {
                        bc[x] = cost[q];
                        bi[x] = (int32_t)q;
                    }
                }
            }
            int64_t np = 0;
            for (int64_t q = 0; q < n; q++) {
                pick[q] = 0;
                if (!cand[q]) continue;
                if (keygt(bc[q], bi[q], cost[q], (int32_t)q)) continue;
                int ok = 1, lim = ncnt[q] < k ? ncnt[q] : k;
                for (int i = 0; i < lim && ok; i++) {
                    int32_t x = nid[q * S + i];
                    if (cand[x] && keygt(cost[x], x, cost[q], (int32_t)q)) ok = 0;
                }
                pick[q] = (uint8_t)ok;
                np += ok;
            }
            if (round_log && rounds < log_cap) round_log[rounds] = ((int64_t)iters << 40) | np;
            rounds++;
            for (int64_t q = 0; q < n; q++)
                if (pick[q]) live[q] = 0;
            nlive -= np;
            /* drop removed points from the stored lists */
            for (int64_t q = 0; q < n; q++) {
                if (!live[q]) continue;
                int r = 0, dead = 0;
                for (int i = 0; i < ncnt[q]; i++) {
                    int32_t x = nid[q * S + i];
                    if (live[x]) {
                        nid[q * S + r] = x;
                        nd2[q * S + r] = nd2[q * S + i];
                        r++;
                    } else {
                        dead = 1;
                    }
                }
                if (!dead) continue;
                ncnt[q] = r;
                if (r >= k) cost[q] = cost_of(&cc, q, nd2 + q * S, nid + q * S, k);
                else dirty[q] = 1;
            }
            if (nlive <= m) break;
        }
    }
    for (int64_t q = 0; q < n; q++) keep_out[q] = live[q];
    if (iters_out) *iters_out = iters;
    if (rounds_out) *rounds_out = rounds;
    free(live); free(dirty); free(cand); free(pick); free(nd2); free(nid); free(ncnt);
    free(cost); free(bc); free(bi); free(order);
    return 0;
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
