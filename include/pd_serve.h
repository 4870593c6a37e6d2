/*
 * pd_serve.h -- a request loop that decimates arriving scans on one GPU.
 *
 * The paper decimates one cloud at a time and has no serving layer; this is
 * the library's own.  Scans arrive at any time (pd_serve_submit) and wait in
 * a FIFO queue.  A scan is admitted when one of `slots` workers is idle and
 * its device-memory estimate fits next to the scans already admitted (the
 * queue head waits until both hold, so no scan is overtaken).  Each worker
 * owns a CUDA stream and a host thread and runs, for its scan: host-to-device
 * copy, pd_build_grid, optional normals (pd_normals_pca, then the network
 * through pd_normals_mlp with PCA as the fallback), pd_decimate_count and the
 * device-to-host copy of the keep mask.  Workers run concurrently, so copies
 * and kernels of different scans overlap on the device, and a finished scan
 * frees its slot and memory for the next one at once (continuous batching).
 * Every scan gets the result it gets alone: workers share no device state.
 *
 * Memory: device buffers come from the context's allocator; the admission
 * budget counts PD_SERVE_BYTES_PER_POINT (PD_SERVE_BYTES_PER_POINT_NORMALS
 * with network normals) per point of every admitted scan.  pd_serve_open
 * sets the release threshold of the device's default memory pool to its
 * maximum, so that the stream-ordered buffers of finished scans stay cached
 * in this process for the next ones.
 */
#ifndef PD_SERVE_H
#define PD_SERVE_H

#include <stdint.h>

#include "pd.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PD_SERVE_BYTES_PER_POINT 240
#define PD_SERVE_BYTES_PER_POINT_NORMALS 400

typedef struct pd_server pd_server;

typedef struct {
    int slots;                   /* concurrent scans on the device (0 = 4) */
    int64_t mem_budget;          /* device bytes for admitted scans (0 = 80 % of the free memory at open) */
    pd_cost_params cost;         /* cost of every scan; cost.normals_dev is ignored */
    const float* mlp_params_dev; /* PD_MLP_PARAMS floats, or NULL: PCA normals */
    int normals;                 /* 1: compute normals for the orientation term (cost.term == PD_TERM_ORIENT) */
} pd_serve_params;

typedef struct {
    int32_t status;        /* PD_OK or the scan's error code */
    int64_t n, m;
    double t_submit_ms;    /* host wall clock, ms since pd_serve_open */
    double t_admit_ms;     /* admitted to a slot */
    double t_done_ms;      /* keep mask in host memory */
    double gpu_ms;         /* the worker's stream time from admission to done */
    pd_stats stats;        /* the decimation's counters */
} pd_serve_result;

/* Start the workers.  ctx must outlive the server. */
int pd_serve_open(pd_ctx* ctx, const pd_serve_params* params, pd_server** out);

/*
 * Queue one scan.  xyz_host (n x 3 int32), rgb_host (n x 3 uint8 or NULL)
 * and keep_host (n bytes, output) are owned by the caller and must stay valid
 * until pd_serve_poll reports the scan done; page-locked host memory lets the
 * copies run asynchronously.  m < 0 selects floor(ratio * n).
 * Returns a ticket >= 0, or -PD_EINVAL (bad arguments), -PD_ENOMEM (the
 * scan's estimate exceeds the whole budget) or -PD_EINTERNAL (server closed).
 */
int64_t pd_serve_submit(pd_server* srv, const int32_t* xyz_host, const uint8_t* rgb_host,
                        int64_t n, int64_t m, double ratio, uint8_t* keep_host);

/*
 * Wait up to wait_ms (< 0: without limit) for a scan.  PD_OK and *out filled
 * when it is done; PD_ETIMEOUT if it is still queued or running; PD_EINVAL
 * for an unknown ticket.  A ticket can be polled again after completion.
 */
int pd_serve_poll(pd_server* srv, int64_t ticket, int wait_ms, pd_serve_result* out);

/* Scans queued, running and done so far. */
int pd_serve_counts(pd_server* srv, int64_t* queued, int64_t* running, int64_t* done);

/* Finish every queued scan, stop the workers and free the server. */
int pd_serve_close(pd_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* PD_SERVE_H */
