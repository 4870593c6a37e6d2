/*
 * pd_quality.h -- quality report of a decimated cloud (libpd).
 *
 * Section "Results and Discussion" (the cube experiment) judges a decimated
 * cloud by counting, around every retained point, the retained points that
 * fall within a growing radius r: on an evenly sampled surface the count
 * grows linearly with the neighbourhood's area pi r^2.  The paper plots the
 * fractile bands of the counts against the area (0.01-0.99, 0.1-0.9,
 * 0.25-0.75) with their mean, takes the least-squares slope as the density
 * estimate (points per m^2), and reads R^2 and RMSE as the goodness of fit
 * (small R^2 or large RMSE: clusters and gaps).  Eq. 2's quantity, the
 * smallest nearest-neighbour distance of the retained set, is reported too.
 *
 * Definitions used here (P = retained points, radii r_1 < ... < r_J in mm):
 *   N_j(p)    = #{q retained, q != p : d(p,q)^2 <= r_j^2}  (exact int64 d^2)
 *   fractile  f of {N_j(p)}: the smallest v with #{p : N_j(p) <= v} >=
 *             ceil(f * P) (f in {0.01, 0.1, 0.25, 0.5, 0.75, 0.9, 0.99})
 *   regression over the P * J samples (x = pi r_j^2 in m^2, y = N_j(p)):
 *             slope = cov(x, y) / var(x), intercept = mean(y) - slope mean(x),
 *             R^2 = cov^2 / (var(x) var(y)), RMSE = sqrt(mean squared residual)
 *   spacing   d_p^2 = the squared distance from p to its nearest other
 *             retained point; min_spacing2 = min over p (Eq. 2's d_p),
 *             mean_spacing = mean of d_p (mm).
 */
#ifndef PD_QUALITY_H
#define PD_QUALITY_H

#include <stdint.h>

#include "pd.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PD_QUALITY_MAX_RADII 32
#define PD_QUALITY_NFRAC 7       /* fractiles 0.01 0.1 0.25 0.5 0.75 0.9 0.99 */
#define PD_QUALITY_HIST 16384    /* counts at or above this are clipped (see count_clipped) */

typedef struct {
    int64_t points;                 /* P: retained points */
    int32_t nr;                     /* radii used */
    int32_t reserved0;
    int32_t radius_mm[PD_QUALITY_MAX_RADII];
    double mean[PD_QUALITY_MAX_RADII];                       /* mean N_j */
    int32_t fractile[PD_QUALITY_MAX_RADII][PD_QUALITY_NFRAC]; /* fractiles of N_j */
    double slope_per_m2;            /* density estimate: points per m^2 */
    double intercept;
    double r2;
    double rmse;
    int64_t min_spacing2_mm2;       /* Eq. 2: min over p of d_p^2 (-1 when P < 2) */
    double mean_spacing_mm;         /* mean of d_p (0 when P < 2) */
    int64_t count_clipped;          /* (p, j) counts >= PD_QUALITY_HIST (fractiles clipped) */
    double ms;                      /* device time of the call */
    double ms_counts;               /* of which: the radius-count kernel */
    int64_t reserved[6];
} pd_quality;

/*
 * Quality report of the retained subset of a cloud.
 *   xyz_dev   n x 3 int32 mm, device (caller-owned, read only).
 *   keep_dev  n bytes, device: 1 = retained (e.g. the output of
 *             pd_decimate_*), or NULL = every point.
 *   radii_mm  nr host ints, strictly ascending, 1 .. 2^24 mm; nr in
 *             [1, PD_QUALITY_MAX_RADII].
 *   out       host struct, filled on success.
 * Device scratch comes from the context's allocator; the stream is
 * synchronised before returning.  Returns PD_OK, PD_EINVAL (bad arguments),
 * PD_ERANGE (coordinate spread >= 2^25 mm), PD_ENOMEM, PD_ECUDA.
 */
int pd_quality_report(pd_ctx* ctx, const int32_t* xyz_dev, const uint8_t* keep_dev, int64_t n,
                      const int32_t* radii_mm, int nr, pd_quality* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PD_QUALITY_H */
