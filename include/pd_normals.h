/*
 * pd_normals.h -- unit normals for the orientation cost term.
 *
 * The orientation term (section "Additional cost terms", Eq. 13) weighs each
 * neighbour by how well its normal agrees with the point's own; the paper
 * takes the normals as given with the input and names no estimator.  These
 * calls supply them on the device:
 *
 *   1. pd_normals_pca: for every point, its 16 nearest neighbours (ascending
 *      squared distance, equal distances by input index), the PCA normal of
 *      those 16 points and a 48-value feature row (the 16 offsets q_i - p
 *      divided by their RMS length);
 *   2. a three-layer network 48 -> 64 -> 64 -> 3 (ReLU, ReLU, linear, output
 *      normalised) that maps a feature row to a unit normal, trained on the
 *      PCA normals by pd_mlp_train (Adam) and run by pd_mlp_forward;
 *   3. pd_normals_mlp: network normals with the PCA normal as the fallback.
 *
 * Numerics: feature rows and the network's weights and hidden activations are
 * bfloat16; products accumulate in float32 on the tensor cores.  Gradients,
 * master weights and Adam state are float32.  Normals are unoriented: the
 * training loss per point is 1 - (n . label)^2 and the orientation term uses
 * |n_p . n_q|.
 *
 * Parameter vector (PD_MLP_PARAMS float32 values, device), row-major:
 *   W1[64][48] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]
 *
 * All pointers named *_dev are device memory.  Errors: PD_EINVAL for a NULL
 * required pointer or a size out of range, PD_ENOMEM when scratch allocation
 * fails, PD_ECUDA for a CUDA error.  Calls are ordered on `stream`.
 */
#ifndef PD_NORMALS_H
#define PD_NORMALS_H

#include <stdint.h>

#include "pd.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PD_NORMAL_K 16
#define PD_MLP_IN 48
#define PD_MLP_HIDDEN 64
#define PD_MLP_PARAMS (64 * 48 + 64 + 64 * 64 + 64 + 3 * 64 + 3)
#define PD_NORMAL_DEFINED 1
#define PD_NORMAL_PLANAR 2
#define PD_PLANAR_RATIO 0.05

/*
 * 16-NN features and PCA normals of every point of a grid that has not been
 * decimated.  Outputs in input order:
 *   feat_dev   n x 48 bfloat16 (raw 16-bit patterns): neighbour i's offset
 *              (dx, dy, dz) / rms at columns 3i..3i+2, rms = sqrt(mean of the
 *              squared offset lengths), each rounded once to bfloat16 (round
 *              to nearest even); rows of clouds with fewer than 17 points are
 *              zero-padded.
 *   pca_dev    n x 3 float32: unit eigenvector of the smallest eigenvalue of
 *              the 16 neighbours' covariance (centred on their mean, the
 *              point itself excluded); 0 where undefined.
 *   valid_dev  n bytes or NULL: PD_NORMAL_DEFINED where the PCA normal is
 *              defined (at least 3 neighbours, smallest eigenvalue simple),
 *              plus PD_NORMAL_PLANAR where the neighbourhood is planar: the
 *              variance along the normal (n^T C n) is at most
 *              PD_PLANAR_RATIO times the middle eigenvalue.  Planar rows are
 *              the confident training labels.
 * The stream is synchronised before returning.
 */
int pd_normals_pca(pd_grid* grid, uint16_t* feat_dev, float* pca_dev, uint8_t* valid_dev,
                   void* stream);

/* Initial parameters: weights uniform in +-sqrt(6 / fan_in) (last layer
 * +-sqrt(3 / 64)) from a splitmix64 counter stream of `seed`; biases 0. */
int pd_mlp_init(float* params_dev, uint64_t seed, void* stream);

/*
 * Network normals of n feature rows.
 *   normals_dev n x 3 float32: o / |o| (0 where o = 0), o the raw output.
 *   norm_dev    n float32 or NULL: |o|.
 */
int pd_mlp_forward(const float* params_dev, const uint16_t* feat_dev, int64_t n,
                   float* normals_dev, float* norm_dev, void* stream);

/*
 * Mean loss and its gradient over n rows: loss_dev[0] = mean of
 * 1 - (u . label)^2 with u the network normal; grad_dev (PD_MLP_PARAMS) its
 * gradient with respect to the parameters, taken through the bfloat16-rounded
 * weights and activations as if the rounding were the identity.  Rows whose
 * raw output is 0 contribute neither loss nor gradient.  Blocks' partial sums
 * are added in a fixed order, so the result is the same bit for bit on every
 * call (and training is reproducible).  Device scratch of about 520 bytes per
 * row plus 30 KB per SM comes from the context's allocator.
 */
int pd_mlp_grad(pd_ctx* ctx, const float* params_dev, const uint16_t* feat_dev,
                const float* labels_dev, int64_t n, float* grad_dev, float* loss_dev,
                void* stream);

typedef struct {
    int steps;      /* Adam steps */
    int batch;      /* rows per step, sampled with replacement from the valid rows */
    float lr;       /* step size (beta1 0.9, beta2 0.999, eps 1e-8) */
    uint64_t seed;  /* row sampling: row i of step t is pool[splitmix64(seed ^ (t << 32) ^ i) % |pool|] */
} pd_train_params;

/*
 * Train params_dev in place on (feature row, PCA label) pairs.
 *   adam_dev   2 x PD_MLP_PARAMS float32 (first and second moments), zero for
 *              a fresh run; step0 = the number of steps already taken with it.
 *   valid_dev  n bytes or NULL (every row valid): rows that may be sampled
 *              (any nonzero byte), e.g. the PD_NORMAL_PLANAR rows.
 *   loss_dev   tp->steps float32 or NULL: mean batch loss of every step.
 */
int pd_mlp_train(pd_ctx* ctx, float* params_dev, float* adam_dev, int step0,
                 const uint16_t* feat_dev, const float* labels_dev, const uint8_t* valid_dev,
                 int64_t n, const pd_train_params* tp, float* loss_dev, void* stream);

/*
 * Normals for the orientation term: the network normal where params_dev is
 * set and the raw output norm is >= min_norm (1e-3 when min_norm <= 0), the
 * PCA normal otherwise.  params_dev = NULL gives the PCA normals.
 */
int pd_normals_mlp(pd_ctx* ctx, const float* params_dev, const uint16_t* feat_dev,
                   const float* pca_dev, int64_t n, float min_norm, float* normals_dev,
                   void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PD_NORMALS_H */
