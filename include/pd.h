/*
 * pd.h -- C ABI of libpd: greedy kNN-cost point-cloud decimation on one GPU.
 *
 * Method: Comino-Trinidad, Chica, Andujar, "Revisiting Poisson-disk
 * Subsampling for Massive Point Cloud Decimation" (arXiv 2311.17604).
 *
 *   Problem (Eq. 1): given a cloud C and a target count m, keep a subset
 *   C' of C with |C'| = m whose local densities are as even as possible.
 *   Cost of a point p (Eq. 10 for k = 1, Eq. 11 for k >= 2):
 *       w_p^k = sum over the k nearest other live points p' of 1 / d(p,p')^2
 *   Greedy (section "Computing per-sample costs", section "Sub-sampling
 *   algorithm"): repeatedly remove the point of largest cost -- among equal
 *   costs the larger input index first -- and update the costs of the points
 *   that had it among their k nearest neighbours, until m points remain.
 *
 * The library reproduces the sequential greedy result exactly (same retained
 * index set) for the density cost, with all work in CUDA kernels.
 *
 * Conventions for every entry point:
 *   - Points are int32 millimetre coordinates, n x 3 row-major (x, y, z).
 *     Their spread per axis must stay below 2^25 mm so every squared distance
 *     (below 3 * 2^50) is exact in an int64 and in a binary64.
 *   - "_dev" pointers are device memory owned by the caller; the library
 *     never frees them.  "_host" pointers are host memory owned by the caller.
 *   - Output arrays are indexed by the caller's input order.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     ordered on that stream.  Documented host synchronisations:
 *     pd_build_grid (reads back the cloud's extent and the cell count),
 *     pd_decimate_* (reads back counters once per removal round and waits for
 *     the result before returning).
 *   - All library-owned device memory comes from the allocator given to
 *     pd_ctx_create (stream-ordered on the call's stream), or from
 *     cudaMallocAsync when none is given.
 *   - Every call returns PD_OK or an error code and never aborts the process;
 *     pd_last_error() returns a description of the last failure on a context.
 */
#ifndef PD_H
#define PD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PD_OK 0
#define PD_EINVAL 1    /* invalid argument (NULL pointer, n < 1, m outside [0,n], k outside [1,16]) */
#define PD_ERANGE 2    /* coordinate spread >= 2^25 mm on some axis */
#define PD_ENOMEM 3    /* the allocator returned NULL */
#define PD_ECUDA 4     /* a CUDA runtime call failed */
#define PD_ETIMEOUT 5  /* a device-side bounded wait gave up */
#define PD_EINTERNAL 6 /* an internal consistency check failed (no progress) */

/* neighbour-weight terms (section "Additional cost terms") */
#define PD_TERM_NONE 0
#define PD_TERM_COLOR 1  /* w = 1 - weight * ||rgb_p - rgb_q||_2 / (255 sqrt 3) */
#define PD_TERM_ORIENT 2 /* w = 1 - weight * (1 - |n_p . n_q|)   (Eq. 13)      */

#define PD_KMAX 16

typedef struct pd_ctx pd_ctx;   /* allocator, last error, tuning cache */
typedef struct pd_grid pd_grid; /* one resident cloud: sorted points, cell table, state */

/* Stream-ordered allocator callbacks (e.g. a framework's caching allocator). */
typedef struct {
    void* (*alloc)(void* user, size_t bytes, void* stream); /* NULL on failure */
    void (*free)(void* user, void* ptr, void* stream);
    void* user;
} pd_allocator;

typedef struct {
    int32_t leaf_max;   /* most points per octree leaf cell, 4..32 (0 = the context's
                           pd_autotune choice, else 32) */
    int32_t reserved[7];
} pd_grid_params;

typedef struct {
    int32_t k;                /* neighbours in the cost, 1..PD_KMAX (Eq. 11) */
    int32_t term;             /* PD_TERM_* */
    double weight;            /* weight of the colour / orientation term */
    const float* normals_dev; /* n x 3 float32, input order (PD_TERM_ORIENT) */
    double band;              /* fraction of live points examined per removal
                                 round (k >= 2 or weighted costs); 0 = default
                                 (0.02, at least 4096 points; 0.01 with a
                                 colour/orientation term).  Never changes a
                                 density-cost result. */
    int32_t reserved[6];
} pd_cost_params;

typedef struct {
    int64_t n, m;
    int32_t rounds;           /* removal rounds after duplicate removal */
    int32_t grid_builds;      /* cell-table (re)builds during decimation */
    int64_t dup_removed;      /* points removed in the duplicate phase */
    int64_t requeries;        /* neighbour searches after the first pass */
    int64_t filtered_queries; /* k >= 2 invariance searches */
    int64_t danger_queries;   /* k >= 2 protected-radius searches */
    double ms_total;          /* device time of the last pd_decimate_* call */
    double ms_knn;            /* of which: all neighbour searches */
    double ms_build;          /* of which: cell-table rebuilds */
    double ms_knn_first;      /* the first full neighbour pass (one launch) */
    int64_t q_first;          /* queries of that pass */
    double ms_knn_requery;    /* re-searches of points that lost a neighbour */
    double ms_rules;          /* removal-rule kernels and key selection */
    int64_t launches;         /* kernels launched by the call */
    double ms_select;         /* of rules: on-device selection of the key threshold */
    double ms_danger;         /* of rules: k >= 2 danger-pair analysis */
    int64_t pairs_first;      /* (query, candidate) pairs the first pass scanned */
    int32_t leaf_max;         /* the grid's octree leaf capacity */
    int32_t iterations;       /* pd_decimate_wup: cost-update iterations (0 otherwise) */
    double ms_grid;           /* device time of the pd_build_grid call that made the grid */
    int64_t live_rounds;      /* sum over the removal rounds of the live count */
    int64_t graph_rounds;     /* rounds replayed from a captured CUDA graph (their phases
                                 are in ms_total only, not in the phase timers) */
} pd_stats;

/* Context: owns nothing but the allocator hooks, the error string and caches. */
int pd_ctx_create(const pd_allocator* alloc /* may be NULL */, pd_ctx** out);
void pd_ctx_destroy(pd_ctx* ctx);

/*
 * Clouds larger than device memory (section "Scaling to massive point
 * clouds": the paper keeps voxels out of core and pages them in; here the
 * second tier is the host's memory, which a Grace-Blackwell GPU addresses
 * directly over NVLink-C2C).  After this call the context tracks its blocks:
 *   - a block of at least max(1 MiB, spill_min) bytes that would take the
 *     context's device bytes past `bytes`, and every such block the library
 *     marks cold (input copies of pd_decimate_host, its keep staging, the
 *     Morton codes, the k-th distances and horizons), is allocated as pinned,
 *     mapped host memory (cudaHostAlloc) instead;
 *   - the kernels address those blocks in place (unified addressing), so a
 *     decimation gives the same result at any budget, only slower;
 *   - blocks below 1 MiB (control blocks, counters, histograms: they take
 *     device atomics) always stay in device memory.
 * bytes = 0 lifts the budget: nothing more spills (blocks already in host
 * memory stay there until freed).  Freeing a host block waits for the stream
 * it was used on.  The budget
 * counts the context's own allocations only (not the caller's buffers).
 * Call it between calls, not while another thread uses the context.
 */
typedef struct {
    uint64_t budget;        /* current budget (0: none) */
    uint64_t device_bytes;  /* tracked device bytes now held */
    uint64_t device_peak;   /* ... and their peak since the budget was set / reset */
    uint64_t host_bytes;    /* pinned host bytes now held */
    uint64_t host_peak;
    int32_t tracked;        /* 1 once a budget was ever set on this context */
    int32_t reserved[3];
} pd_memory;
int pd_ctx_set_device_budget(pd_ctx* ctx, uint64_t bytes, uint64_t spill_min);
int pd_ctx_memory(pd_ctx* ctx, pd_memory* out);
int pd_ctx_reset_peaks(pd_ctx* ctx);
const char* pd_strerror(int code);
const char* pd_last_error(const pd_ctx* ctx);

/*
 * Build the voxel grid of a cloud (section "Sub-sampling algorithm": the
 * paper voxelises the cloud; here one Morton-order radix sort yields cells of
 * every power-of-two size, an adaptive leaf level per point, and a hashed
 * table of cell ranges).
 *   xyz_dev  n x 3 int32, device.  Copied; may be freed after the call.
 *   rgb_dev  n x 3 uint8, device, or NULL (needed for PD_TERM_COLOR).  Copied.
 *   params   may be NULL.
 * Synchronises the stream once (extent and cell count).
 */
int pd_build_grid(pd_ctx* ctx, const int32_t* xyz_dev, const uint8_t* rgb_dev, int64_t n,
                  const pd_grid_params* params, void* stream, pd_grid** out);
int pd_grid_free(pd_grid* grid);

/*
 * Cost of every point of the full cloud (Eq. 10 / Eq. 11, optional weights).
 *   cost_dev  n doubles (may be NULL): binary64 sum over the k nearest, in
 *             ascending-distance order; 1/d^2 for k = 1; +inf if a neighbour
 *             coincides; 0 for a cloud of one point.
 *   knn_dev   n x k int32 input indices of the k nearest, ascending (d^2,
 *             tie order unspecified), -1 where fewer exist.  May be NULL.
 */
int pd_knn_cost(pd_grid* grid, const pd_cost_params* cp, double* cost_dev, int32_t* knn_dev,
                void* stream);

/*
 * Greedy decimation to exactly m points (Eq. 1, |C'| = m).
 *   keep_dev  n bytes: 1 = retained, 0 = removed, input order.
 * The grid's point state is consumed: build a new grid to decimate again.
 * Density-only costs give the sequential greedy's exact result.
 */
int pd_decimate_count(pd_grid* grid, const pd_cost_params* cp, int64_t m, uint8_t* keep_dev,
                      void* stream);
/* Same with m = floor(ratio * n) computed in binary64 (lambda = m / |C|). */
int pd_decimate_ratio(pd_grid* grid, const pd_cost_params* cp, double ratio, uint8_t* keep_dev,
                      void* stream);
/*
 * The paper's own iterative scheme (section "Sub-sampling algorithm"), an
 * alternative to the exact greedy: not the sequential greedy's result, but
 * fewer, larger passes.  Until m points remain, each iteration
 *   1. recomputes the S = 8 nearest neighbours (the extended k+b
 *      neighbourhood, equal distances ordered by input index) and the
 *      density cost (Eq. 10 / 11) of every live point;
 *   2. takes w_up = the m-th smallest key (cost, input index);
 *   3. removes points above w_up in rounds: a clean live point above w_up
 *      is removed when no other such point adjacent to it has a larger key
 *      (adjacent: one of the two lies among the first k stored neighbours of
 *      the other).  Removed points leave their reverse neighbours' stored
 *      lists; a point with at least k stored neighbours left takes its cost
 *      from the first k of them, one with fewer is dirty (not removed) until
 *      the next iteration.
 * The paper removes the points above w_up in a sequential sweep over its
 * voxels; here every round removes, at once, the points no larger-key
 * candidate interacts with.  Removals never raise a cost, so the count never
 * drops below m, and every round of every iteration's start removes at least
 * the largest key.
 *   cp        density cost (term PD_TERM_NONE), k in [1, 6].
 *   keep_dev  n bytes: 1 = retained (exactly m ones), input order.
 * The grid is consumed.  pd_grid_stats reports iterations and rounds.
 * Reads one counter per round back to the host (a synchronisation).
 */
int pd_decimate_wup(pd_grid* grid, const pd_cost_params* cp, int64_t m, uint8_t* keep_dev,
                    void* stream);

/*
 * Autotuner for the octree leaf capacity (the cell size of the neighbour
 * search).  The paper picks its voxel size by hand (section "Sub-sampling
 * algorithm"); here the choice never changes a result (every search is exact
 * at any leaf size), only the speed: large leaves favour the dense first
 * pass, small ones the sparse searches of the removal rounds.  The call
 * decimates the first min(n, sample) points (sample <= 0: all) of xyz_dev
 * with cost cp and keep ratio `ratio` once per capacity in {12, 16, 24, 32}
 * (after one untimed warm-up pass), times grid build + decimation with CUDA
 * events on `stream`, and keeps the fastest.  The choice is stored in the
 * context: pd_build_grid with leaf_max = 0 (or NULL params) uses it from then
 * on.  *leaf_max_out (may be NULL) receives it.  Device scratch comes from
 * the context's allocator; the stream is synchronised before returning.
 */
int pd_autotune(pd_ctx* ctx, const int32_t* xyz_dev, const uint8_t* rgb_dev, int64_t n,
                const pd_cost_params* cp, double ratio, int64_t sample, void* stream,
                int32_t* leaf_max_out);

/* Counters of the last pd_decimate_* call on this grid. */
int pd_grid_stats(const pd_grid* grid, pd_stats* out);

/*
 * End-to-end call on host buffers: copy xyz (and rgb / normals) to the device,
 * build the grid, decimate to m points and copy the keep mask back.
 *   xyz_host n x 3 int32; rgb_host n x 3 uint8 or NULL; normals_host n x 3
 *   float32 or NULL (used when cp->term == PD_TERM_ORIENT); keep_host n bytes.
 * Synchronises the stream before returning.
 */
int pd_decimate_host(pd_ctx* ctx, const int32_t* xyz_host, const uint8_t* rgb_host,
                     const float* normals_host, int64_t n, const pd_cost_params* cp, int64_t m,
                     uint8_t* keep_host, void* stream, pd_stats* stats /* may be NULL */);

/*
 * Batch of independent scans (many clouds of uneven size; the sequential
 * greedy of section "Sub-sampling algorithm" applied to each scan on its own,
 * with its own target m or floor(ratio * n)).
 *
 * concurrency == PD_BATCH_PACKED: every scan is moved (a copy; the caller's
 * buffers are only read) into its own aligned tile of one packed cloud, and
 * the whole batch is decimated as ONE grid: one grid build, one first
 * neighbour pass, and one sequence of removal rounds whose every launch
 * covers all scans.  The tiles are at least 2^T - E apart (E the largest
 * per-axis extent of any scan, 2^T >= 3E + 2), farther than any two points
 * of one scan, so no search leaves its scan; only the removal threshold of a
 * round is selected per scan.  For the density cost each scan gets exactly
 * its stand-alone result (the sequential greedy's retained set).  With a
 * colour or orientation term the rounds of the batch differ from those of a
 * scan alone, so the result is the same within the tolerance those terms
 * have alone.  A scan's stats are those of the whole batch, with its own n
 * and m.  Extra device memory: the packed copy and its keep mask (13 B per
 * point, 16 with colours, 25 with normals) and one grid over all points.  A
 * batch that cannot be packed falls back to 8 slots (below): more than
 * PD_BATCH_MAX_SCANS scans or 2^31 - 64 points, a target of k points or
 * fewer, a missing colour or normal array, tiles beyond the coordinate range
 * (2^25 mm), or a scan with more coincident points than it must lose.
 *
 * concurrency >= 0: scans run through `concurrency` slots (0 = 8); each slot
 * has its own stream and host thread and runs pd_build_grid +
 * pd_decimate_count on its scans, so the slots' kernels overlap on the
 * device.  Every scan gets the same result it gets alone.
 *
 * The work is ordered after what is queued on `stream`, and `stream` waits
 * for all of it; the call returns when every scan is done.
 * Returns PD_OK, or the first error of any scan (each scan's own status is in
 * its descriptor).
 */
#define PD_BATCH_PACKED (-1)
#define PD_BATCH_MAX_SCANS 4096
typedef struct {
    const int32_t* xyz_dev;    /* n x 3 int32, device */
    const uint8_t* rgb_dev;    /* n x 3 uint8, device, or NULL */
    const float* normals_dev;  /* n x 3 float32, device, or NULL */
    int64_t n;
    int64_t m;                 /* points to keep; < 0: floor(ratio * n) */
    double ratio;
    uint8_t* keep_dev;         /* n bytes, device (output) */
    int32_t status;            /* output: PD_OK or an error code */
    pd_stats stats;            /* output */
} pd_scan_desc;
int pd_decimate_batch(pd_ctx* ctx, pd_scan_desc* scans, int nscans, const pd_cost_params* cp,
                      int concurrency, void* stream);

/*
 * Allocation-free variant of the neighbour/cost pass (no counterpart in the
 * paper: it exists for callers that cannot allocate device memory when they
 * call us, e.g. a real-time ingest loop whose memory budget is fixed at
 * start-up, or a plug-in that must not touch its host's allocator).
 *
 * Computes exactly what pd_build_grid (default parameters) followed by
 * pd_knn_cost with the density cost (term PD_TERM_NONE) computes, for clouds
 * of at most PD_STATIC_MAX_POINTS points:
 *   xyz_dev   n x 3 int32, device, caller-owned (read only).
 *   cost_dev  n doubles, device (may be NULL);  knn_dev n x k int32, device
 *             (may be NULL) -- the same layout as pd_knn_cost.
 * All temporaries live in one file-scope device array of
 * PD_STATIC_SCRATCH_BYTES bytes that every GPU loading the library holds until
 * the process exits (each device has its own copy).  The call makes no
 * cudaMalloc / cudaFree / cudaMallocAsync and uses no allocating library
 * routine.  The first call on a device looks up the array's device address on
 * that device (cudaGetSymbolAddress) and caches it for the process: make that
 * first call before any stream capture.  A cudaDeviceReset (or any teardown of
 * the device's primary context) invalidates the cached address; do not call
 * this entry point on that device afterwards.  Every call reuses the same
 * array and overwrites it; it clears what must start at zero.  Two calls that
 * overlap on the same device (for example on two streams) race on the array:
 * serialise them.  Calls on different devices use different copies and do
 * not race.  The call synchronises the stream (it reads the cloud's extent
 * and cell count, like pd_build_grid).
 * Returns PD_EINVAL (NULL xyz, n < 1, k outside [1, 16]), PD_ERANGE (n above
 * PD_STATIC_MAX_POINTS, or a coordinate spread >= 2^25 mm), PD_ENOMEM (a
 * guard: the cloud needs more octree cells than the fixed table holds; with
 * at most PD_STATIC_MAX_POINTS points and leaves of 32 points the cell count
 * stays far below the table's size), PD_ECUDA.
 */
#define PD_STATIC_MAX_POINTS 65536
#define PD_STATIC_SCRATCH_BYTES (16u << 20)
int pd_knn_cost_static(const int32_t* xyz_dev, int64_t n, int k, double* cost_dev,
                       int32_t* knn_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PD_H */
