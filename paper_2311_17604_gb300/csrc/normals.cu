// normals.cu -- unit normals for the orientation term (Eq. 13): PCA of the 16
// nearest neighbours, and a small network that maps the 16 neighbour offsets
// to a normal, trained on the PCA normals by the kernels below.
//
// The paper takes oriented input as given (section "Additional cost terms")
// and names no estimator; these kernels supply the normals.
//
// Parameter layout (float32, PD_MLP_PARAMS values):
//   W1[64][48] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]
// Forward: h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), o = h2 W3^T + b3,
// normal = o / |o|.  x, W1..W3, h1 and h2 are bfloat16; products accumulate
// in float32 on the tensor cores (mma.sync m16n8k16, bf16 in, f32 out).
// Loss per row: 1 - (u . y)^2 with u = o / |o| (labels are unoriented).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pd.h"
#include "../../include/pd_normals.h"
#include "pd_internal.cuh"
#include "pd_kernels.h"

namespace pd {

#define NF PD_MLP_IN
#define NH PD_MLP_HIDDEN
#define O_W1 0
#define O_B1 (O_W1 + NH * NF)
#define O_W2 (O_B1 + NH)
#define O_B2 (O_W2 + NH * NH)
#define O_W3 (O_B2 + NH)
#define O_B3 (O_W3 + 3 * NH)
#define N_PARAMS (O_B3 + 3)
static_assert(N_PARAMS == PD_MLP_PARAMS, "parameter count");
static_assert(NF == 3 * PD_NORMAL_K, "feature width");

// ------------------------------------------------------------------ PCA + features
// Unit eigenvector of the smallest eigenvalue of the symmetric matrix
// (c00 c01 c02 / . c11 c12 / . . c22): the eigenvalue from the trigonometric
// closed form of O. K. Smith (CACM 4(4), 1961), the eigenvector as the longest
// cross product of two rows of (A - lambda I).  False when that product's
// length is <= 1e-6 trace(A)^2 (the smallest eigenvalue is not simple).
// *lmid receives the middle eigenvalue.
__device__ inline bool smallest_eigvec(double a00, double a01, double a02, double a11,
                                       double a12, double a22, double out[3], double* lmid) {
    double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    double q = (a00 + a11 + a22) / 3.0;
    double lam;
    if (p1 == 0.0) {
        lam = fmin(a00, fmin(a11, a22));
        *lmid = a00 + a11 + a22 - lam - fmax(a00, fmax(a11, a22));
    } else {
        double e0 = a00 - q, e1 = a11 - q, e2 = a22 - q;
        double p = sqrt((e0 * e0 + e1 * e1 + e2 * e2 + 2.0 * p1) / 6.0);
        double b00 = e0 / p, b11 = e1 / p, b22 = e2 / p;
        double b01 = a01 / p, b02 = a02 / p, b12 = a12 / p;
        double det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) +
                     b02 * (b01 * b12 - b11 * b02);
        double r = fmin(1.0, fmax(-1.0, det / 2.0));
        // eigenvalues q + 2p cos(acos(r)/3 + 2 pi j / 3); j = 1 is the smallest
        double phi = acos(r) / 3.0;
        lam = q + 2.0 * p * cos(phi + 2.0943951023931957);
        *lmid = q + 2.0 * p * cos(phi + 4.1887902047863905);  // j = 2: the middle one
    }
    double r0x = a00 - lam, r0y = a01, r0z = a02;
    double r1x = a01, r1y = a11 - lam, r1z = a12;
    double r2x = a02, r2y = a12, r2z = a22 - lam;
    double c0x = r0y * r1z - r0z * r1y, c0y = r0z * r1x - r0x * r1z, c0z = r0x * r1y - r0y * r1x;
    double c1x = r0y * r2z - r0z * r2y, c1y = r0z * r2x - r0x * r2z, c1z = r0x * r2y - r0y * r2x;
    double c2x = r1y * r2z - r1z * r2y, c2y = r1z * r2x - r1x * r2z, c2z = r1x * r2y - r1y * r2x;
    double n0 = c0x * c0x + c0y * c0y + c0z * c0z;
    double n1 = c1x * c1x + c1y * c1y + c1z * c1z;
    double n2 = c2x * c2x + c2y * c2y + c2z * c2z;
    double best = n0, bx = c0x, by = c0y, bz = c0z;
    if (n1 > best) {
        best = n1;
        bx = c1x;
        by = c1y;
        bz = c1z;
    }
    if (n2 > best) {
        best = n2;
        bx = c2x;
        by = c2y;
        bz = c2z;
    }
    double tr = a00 + a11 + a22;
    if (!(best > 1e-12 * (tr * tr) * (tr * tr))) return false;
    double inv = 1.0 / sqrt(best);
    out[0] = bx * inv;
    out[1] = by * inv;
    out[2] = bz * inv;
    return true;
}

// One thread per point (Morton position s).  Offsets are exact int32; the
// moment sums are exact int64, so the covariance scaled by m^2 is the exact
// integer m * sum(u v) - sum(u) sum(v) before its conversion to binary64.
__global__ void __launch_bounds__(128)
    features_kernel(const int4* __restrict__ pos, const int* __restrict__ nbr, int S, int64_t n,
                    uint4* __restrict__ feat, float* __restrict__ pca, uint8_t* valid) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int4 p = pos[s];
    int64_t out = p.w;
    int ox[PD_NORMAL_K], oy[PD_NORMAL_K], oz[PD_NORMAL_K];
    int m = 0;
    long long sx = 0, sy = 0, sz = 0, sxx = 0, sxy = 0, sxz = 0, syy = 0, syz = 0, szz = 0;
#pragma unroll
    for (int i = 0; i < PD_NORMAL_K; i++) {
        int x = i < S ? nbr[s * S + i] : -1;
        int4 q = x >= 0 ? pos[x] : p;
        int dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
        ox[i] = dx;
        oy[i] = dy;
        oz[i] = dz;
        m += x >= 0;
        sx += dx;
        sy += dy;
        sz += dz;
        sxx += (long long)dx * dx;
        sxy += (long long)dx * dy;
        sxz += (long long)dx * dz;
        syy += (long long)dy * dy;
        syz += (long long)dy * dz;
        szz += (long long)dz * dz;
    }
    // neighbours are stored nearest first, so the missing ones are the last
    // (their offsets are 0 and add nothing to the sums)
    long long ss = sxx + syy + szz;
    double rms = m ? sqrt((double)ss / (double)m) : 0.0;
    uint32_t w[NF / 2];
#pragma unroll
    for (int c = 0; c < NF; c += 2) {
        int i0 = c / 3, c0 = c % 3, i1 = (c + 1) / 3, c1 = (c + 1) % 3;
        int v0 = c0 == 0 ? ox[i0] : (c0 == 1 ? oy[i0] : oz[i0]);
        int v1 = c1 == 0 ? ox[i1] : (c1 == 1 ? oy[i1] : oz[i1]);
        __nv_bfloat16 f0 = __double2bfloat16(rms > 0.0 ? (double)v0 / rms : 0.0);
        __nv_bfloat16 f1 = __double2bfloat16(rms > 0.0 ? (double)v1 / rms : 0.0);
        w[c / 2] = (uint32_t)__bfloat16_as_ushort(f0) | ((uint32_t)__bfloat16_as_ushort(f1) << 16);
    }
    uint4* fr = feat + out * (NF / 8);
#pragma unroll
    for (int j = 0; j < NF / 8; j++)
        fr[j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
    long long mm = m;
    double nv[3] = {0.0, 0.0, 0.0};
    double a00 = (double)(mm * sxx - sx * sx), a11 = (double)(mm * syy - sy * sy),
           a22 = (double)(mm * szz - sz * sz);
    double lmid = 0.0;
    bool ok = m >= 3 && smallest_eigvec(a00, (double)(mm * sxy - sx * sy),
                                        (double)(mm * sxz - sx * sz), a11,
                                        (double)(mm * syz - sy * sz), a22, nv, &lmid);
    // planar: the smallest eigenvalue (A n . n) at most PD_PLANAR_RATIO of the middle one
    bool planar = false;
    if (ok) {
        double c01 = (double)(mm * sxy - sx * sy), c02 = (double)(mm * sxz - sx * sz),
               c12 = (double)(mm * syz - sy * sz);
        double an0 = a00 * nv[0] + c01 * nv[1] + c02 * nv[2];
        double an1 = c01 * nv[0] + a11 * nv[1] + c12 * nv[2];
        double an2 = c02 * nv[0] + c12 * nv[1] + a22 * nv[2];
        double l0 = an0 * nv[0] + an1 * nv[1] + an2 * nv[2];
        planar = lmid > 0.0 && l0 <= PD_PLANAR_RATIO * lmid;
    }
    pca[out * 3 + 0] = ok ? (float)nv[0] : 0.f;
    pca[out * 3 + 1] = ok ? (float)nv[1] : 0.f;
    pca[out * 3 + 2] = ok ? (float)nv[2] : 0.f;
    if (valid) valid[out] = (uint8_t)((ok ? PD_NORMAL_DEFINED : 0) | (planar ? PD_NORMAL_PLANAR : 0));
}

// ------------------------------------------------------------------ forward (tensor cores)
__device__ inline uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ inline float2 unpack_bf16(uint32_t u) {
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&u);
    return make_float2(__bfloat162float(v.x), __bfloat162float(v.y));
}

// D = A B + D for one m16n8k16 tile (A row-major 16x16, B column-major 16x8).
__device__ inline void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

#define MLP_WARPS 8
#define MLP_BLOCKS_PER_SM 3

// Weight rows are padded (56 and 72 bf16 = 28 and 36 words) so that the
// eight row groups of a B-fragment load fall in distinct shared-memory banks.
#define W1_LD 56
#define W2_LD 72
struct MlpSmem {
    __nv_bfloat16 w1[NH * W1_LD];
    __nv_bfloat16 w2[NH * W2_LD];
    __nv_bfloat16 w3[8 * W2_LD];  // rows 3..7 zero
    float b1[NH], b2[NH], b3[8];
};

// Accumulators of two adjacent n-tiles (one 16-column k-slice) -> the next
// layer's A fragment, after ReLU and rounding to bfloat16.
__device__ inline void relu_pack(const float lo[4], const float hi[4], uint32_t a[4]) {
    a[0] = pack_bf16(fmaxf(lo[0], 0.f), fmaxf(lo[1], 0.f));
    a[1] = pack_bf16(fmaxf(lo[2], 0.f), fmaxf(lo[3], 0.f));
    a[2] = pack_bf16(fmaxf(hi[0], 0.f), fmaxf(hi[1], 0.f));
    a[3] = pack_bf16(fmaxf(hi[2], 0.f), fmaxf(hi[3], 0.f));
}

// Store a warp's 16 x 64 bf16 activations as float (training only).
__device__ inline void store_act(const uint32_t a[4][4], float* dst, int64_t ra, int64_t rb,
                                 int64_t n, int t) {
#pragma unroll
    for (int kk = 0; kk < 4; kk++) {
#pragma unroll
        for (int qd = 0; qd < 4; qd++) {
            float2 v = unpack_bf16(a[kk][qd]);
            int col = 16 * kk + (qd >= 2 ? 8 : 0) + 2 * t;
            int64_t row = (qd & 1) ? rb : ra;
            if (row < n) *reinterpret_cast<float2*>(dst + row * NH + col) = v;
        }
    }
}

// Persistent: one warp = one 16-row tile at a time, weights rounded into
// shared memory once per block.  rows = NULL: row r is feature row r.
// Outputs per row: unit normal and |o| (at the feature row's index); for
// training also the activations and the raw output (at the batch row).
__global__ void __launch_bounds__(MLP_WARPS * 32, MLP_BLOCKS_PER_SM)
    mlp_forward_kernel(const float* __restrict__ prm, const uint32_t* __restrict__ feat,
                       const int* __restrict__ rows, int64_t n, float* outn, float* onorm,
                       float* h1s, float* h2s, float* raw) {
    __shared__ MlpSmem sm;
    for (int i = threadIdx.x; i < NH * NF; i += blockDim.x)
        sm.w1[(i / NF) * W1_LD + i % NF] = __float2bfloat16_rn(prm[O_W1 + i]);
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x)
        sm.w2[(i / NH) * W2_LD + i % NH] = __float2bfloat16_rn(prm[O_W2 + i]);
    for (int i = threadIdx.x; i < 8 * NH; i += blockDim.x)
        sm.w3[(i / NH) * W2_LD + i % NH] = __float2bfloat16_rn(i < 3 * NH ? prm[O_W3 + i] : 0.f);
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        sm.b1[i] = prm[O_B1 + i];
        sm.b2[i] = prm[O_B2 + i];
    }
    if (threadIdx.x < 8) sm.b3[threadIdx.x] = threadIdx.x < 3 ? prm[O_B3 + threadIdx.x] : 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t ntiles = (n + 15) / 16;
    const int64_t wstride = (int64_t)gridDim.x * MLP_WARPS;
    for (int64_t tile = (int64_t)blockIdx.x * MLP_WARPS + (threadIdx.x >> 5); tile < ntiles;
         tile += wstride) {
        int64_t ra = tile * 16 + g, rb = ra + 8;
        bool va = ra < n, vb = rb < n;
        int64_t xa = va ? (rows ? rows[ra] : ra) : 0, xb = vb ? (rows ? rows[rb] : rb) : 0;
        const uint32_t* fa = feat + xa * (NF / 2);
        const uint32_t* fb = feat + xb * (NF / 2);
        // layer 1: K = 48 (3 k-slices), N = 64 (8 n-tiles)
        float c1[8][4];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float b0 = sm.b1[8 * j + 2 * t], b1v = sm.b1[8 * j + 2 * t + 1];
            c1[j][0] = b0;
            c1[j][1] = b1v;
            c1[j][2] = b0;
            c1[j][3] = b1v;
        }
#pragma unroll
        for (int kk = 0; kk < 3; kk++) {
            uint32_t a[4];
            a[0] = va ? fa[8 * kk + t] : 0u;
            a[1] = vb ? fb[8 * kk + t] : 0u;
            a[2] = va ? fa[8 * kk + 4 + t] : 0u;
            a[3] = vb ? fb[8 * kk + 4 + t] : 0u;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const uint32_t* wr =
                    reinterpret_cast<const uint32_t*>(sm.w1 + (8 * j + g) * W1_LD + 16 * kk);
                mma16816(c1[j], a, wr[t], wr[4 + t]);
            }
        }
        uint32_t a2[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; kk++) relu_pack(c1[2 * kk], c1[2 * kk + 1], a2[kk]);
        if (h1s) store_act(a2, h1s, ra, rb, n, t);
        // layer 2: K = 64, N = 64
        float c2[8][4];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float b0 = sm.b2[8 * j + 2 * t], b1v = sm.b2[8 * j + 2 * t + 1];
            c2[j][0] = b0;
            c2[j][1] = b1v;
            c2[j][2] = b0;
            c2[j][3] = b1v;
        }
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const uint32_t* wr =
                    reinterpret_cast<const uint32_t*>(sm.w2 + (8 * j + g) * W2_LD + 16 * kk);
                mma16816(c2[j], a2[kk], wr[t], wr[4 + t]);
            }
        }
        uint32_t a3[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; kk++) relu_pack(c2[2 * kk], c2[2 * kk + 1], a3[kk]);
        if (h2s) store_act(a3, h2s, ra, rb, n, t);
        // layer 3: K = 64, N = 8 (3 used)
        float c3[4] = {sm.b3[2 * t], sm.b3[2 * t + 1], sm.b3[2 * t], sm.b3[2 * t + 1]};
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            const uint32_t* wr = reinterpret_cast<const uint32_t*>(sm.w3 + g * W2_LD + 16 * kk);
            mma16816(c3, a3[kk], wr[t], wr[4 + t]);
        }
        // columns 0,1 sit on lane t = 0 and column 2 on t = 1 of each row
        float o2a = __shfl_down_sync(0xffffffffu, c3[0], 1);
        float o2b = __shfl_down_sync(0xffffffffu, c3[2], 1);
        if (t == 0) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                int64_t row = h ? rb : ra;
                if (row >= n) continue;
                float o0 = h ? c3[2] : c3[0], o1 = h ? c3[3] : c3[1], o2 = h ? o2b : o2a;
                float nr = sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
                int64_t dst = h ? xb : xa;
                if (raw) {
                    raw[row * 3 + 0] = o0;
                    raw[row * 3 + 1] = o1;
                    raw[row * 3 + 2] = o2;
                }
                if (onorm) onorm[dst] = nr;
                if (outn) {
                    float inv = nr > 0.f ? 1.f / nr : 0.f;
                    outn[dst * 3 + 0] = o0 * inv;
                    outn[dst * 3 + 1] = o1 * inv;
                    outn[dst * 3 + 2] = o2 * inv;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ backward (tensor cores)
// Persistent over tiles of TR = 64 rows; 4 warps per block, warp w owning
// rows 16w..16w+15 of a tile for the row-wise products and the 16-row slice
// w of the weight gradients.  All matrix products run as mma.sync m16n8k16
// (bf16 in, fp32 accumulate):
//   dh1 = (dh2 W2) relu'(h1)            A = dh2 [row][j], B = W2 (as W2^T [c][j])
//   dW2 = dh2^T h1                       A = dh2^T [j][row], B = h1 (as h1^T [c][row])
//   dW1 = dh1^T x                        A = dh1^T [a][row], B = x (as x^T [f][row])
// x, h1 and the weights are bfloat16 values already (what the forward used).
// The gradients dh1 and dh2 are float32: each enters as the sum of two
// bfloat16 parts hi + lo (hi = bf16(v), lo = bf16(v - hi)), two products per
// tile, so the result keeps about 16 bits of the float32 value.  The small
// pieces (dh2 = do W3 masked, dW3, the biases, the loss) run on the CUDA
// cores.  Weights enter as the bfloat16 values the forward used; rounding is
// treated as the identity (a straight-through gradient).
#define BT_ROWS 64
#define BT_THREADS 128
#define BT_LD 72  // row stride (bf16) of the shared tiles: 144 bytes
#define BT_BLOCKS_PER_SM 2

struct BwSmem {
    __nv_bfloat16 w2t[NH][BT_LD];      // W2^T [c][j]
    __nv_bfloat16 xt[NF][BT_LD];       // x^T  [f][row]
    __nv_bfloat16 h1t[NH][BT_LD];      // h1^T [c][row]
    __nv_bfloat16 d2[2][BT_ROWS][BT_LD];   // dh2 [row][j], hi and lo
    __nv_bfloat16 d2t[2][NH][BT_LD];       // dh2^T [j][row], hi and lo
    __nv_bfloat16 d1t[2][NH][BT_LD];       // dh1^T [a][row], hi and lo
    float w3[3][NH];
    float dout[BT_ROWS][4];            // d loss / d o (divided by n)
    float red[BT_THREADS][4];          // end-of-kernel reductions
    float db1w[4][NH];                 // per-warp column sums of dh1
};

__device__ inline uint32_t ld32(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

__global__ void __launch_bounds__(BT_THREADS, BT_BLOCKS_PER_SM)
    mlp_backward_tc_kernel(const float* __restrict__ prm, const uint16_t* __restrict__ feat,
                           const int* __restrict__ rows, const float* __restrict__ labels,
                           int64_t n, const float* __restrict__ h1s,
                           const float* __restrict__ h2s, const float* __restrict__ raw,
                           float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    BwSmem& sm = *reinterpret_cast<BwSmem*>(smraw);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const float inv_n = 1.0f / (float)n;
    for (int i = tid; i < NH * NH; i += BT_THREADS) {
        int j = i / NH, c = i % NH;  // W2 is [j][c] (out, in)
        sm.w2t[c][j] = __float2bfloat16_rn(prm[O_W2 + i]);
    }
    for (int i = tid; i < 3 * NH; i += BT_THREADS)
        sm.w3[i / NH][i % NH] = __bfloat162float(__float2bfloat16_rn(prm[O_W3 + i]));
    // accumulators: dW1 rows a = 16w.. (6 n-tiles of f), dW2 rows j = 16w.. (8 n-tiles of c)
    float g1[6][4], g2[8][4];
#pragma unroll
    for (int i = 0; i < 6; i++) g1[i][0] = g1[i][1] = g1[i][2] = g1[i][3] = 0.f;
#pragma unroll
    for (int i = 0; i < 8; i++) g2[i][0] = g2[i][1] = g2[i][2] = g2[i][3] = 0.f;
    float db1[16];  // columns 8 nt + 2 t (+1) of dh1, this lane's rows
#pragma unroll
    for (int i = 0; i < 16; i++) db1[i] = 0.f;
    float db2 = 0.f, dw3[3] = {0.f, 0.f, 0.f}, db3[3] = {0.f, 0.f, 0.f}, lsum = 0.f;
    const int jcol = tid & 63;  // the dh2 column this thread computes
    const int64_t ntiles = (n + BT_ROWS - 1) / BT_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * BT_ROWS;
        const int nr = (int)min((int64_t)BT_ROWS, n - r0);
        __syncthreads();  // the previous tile's readers are done
        for (int i = tid; i < BT_ROWS * NF; i += BT_THREADS) {
            int r = i / NF, f = i % NF;
            uint16_t v = 0;
            if (r < nr) {
                int64_t x = rows ? rows[r0 + r] : r0 + r;
                v = feat[x * NF + f];
            }
            sm.xt[f][r] = __ushort_as_bfloat16(v);
        }
        for (int i = tid; i < BT_ROWS * NH; i += BT_THREADS) {
            int r = i / NH, c = i % NH;
            float v = r < nr ? h1s[(r0 + r) * NH + c] : 0.f;
            sm.h1t[c][r] = __float2bfloat16_rn(v);  // exact: h1 holds bfloat16 values
        }
        if (tid < BT_ROWS) {  // d loss / d o for row tid, already divided by n
            int r = tid;
            float d0 = 0.f, d1 = 0.f, d2 = 0.f;
            if (r < nr) {
                int64_t x = rows ? rows[r0 + r] : r0 + r;
                float o0 = raw[(r0 + r) * 3], o1 = raw[(r0 + r) * 3 + 1], o2 = raw[(r0 + r) * 3 + 2];
                float y0 = labels[x * 3], y1 = labels[x * 3 + 1], y2 = labels[x * 3 + 2];
                float nrm = sqrtf(o0 * o0 + o1 * o1 + o2 * o2);
                if (nrm > 0.f) {
                    float u0 = o0 / nrm, u1 = o1 / nrm, u2 = o2 / nrm;
                    float dot = u0 * y0 + u1 * y1 + u2 * y2;
                    lsum += 1.f - dot * dot;
                    // dL/du = -2 dot y; dL/do = (dL/du - (dL/du . u) u) / |o|
                    float q0 = -2.f * dot * y0, q1 = -2.f * dot * y1, q2 = -2.f * dot * y2;
                    float gu = q0 * u0 + q1 * u1 + q2 * u2;
                    float sc = inv_n / nrm;
                    d0 = (q0 - gu * u0) * sc;
                    d1 = (q1 - gu * u1) * sc;
                    d2 = (q2 - gu * u2) * sc;
                }
            }
            sm.dout[r][0] = d0;
            sm.dout[r][1] = d1;
            sm.dout[r][2] = d2;
            db3[0] += d0;
            db3[1] += d1;
            db3[2] += d2;
        }
        __syncthreads();
        // dh2 = (do W3) relu'(h2): thread (jcol, rows tid/64 + 2i); dW3 and db2 on the side
        for (int r = tid >> 6; r < BT_ROWS; r += BT_THREADS / 64) {
            float v = 0.f;
            if (r < nr) {
                float h2 = h2s[(r0 + r) * NH + jcol];
                float d0 = sm.dout[r][0], d1 = sm.dout[r][1], d2 = sm.dout[r][2];
                dw3[0] += d0 * h2;
                dw3[1] += d1 * h2;
                dw3[2] += d2 * h2;
                v = d0 * sm.w3[0][jcol] + d1 * sm.w3[1][jcol] + d2 * sm.w3[2][jcol];
                if (!(h2 > 0.f)) v = 0.f;
            }
            db2 += v;
            __nv_bfloat16 hi = __float2bfloat16_rn(v);
            __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
            sm.d2[0][r][jcol] = hi;
            sm.d2[1][r][jcol] = lo;
            sm.d2t[0][jcol][r] = hi;
            sm.d2t[1][jcol][r] = lo;
        }
        __syncthreads();
        // dh1 = (dh2 W2) relu'(h1) for rows 16w.. of the tile (tensor cores)
        {
            float acc[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
            const int ra = 16 * w + g, rb = ra + 8;
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
#pragma unroll
                for (int part_ = 0; part_ < 2; part_++) {
                    uint32_t a[4];
                    a[0] = ld32(&sm.d2[part_][ra][16 * kk + 2 * t]);
                    a[1] = ld32(&sm.d2[part_][rb][16 * kk + 2 * t]);
                    a[2] = ld32(&sm.d2[part_][ra][16 * kk + 8 + 2 * t]);
                    a[3] = ld32(&sm.d2[part_][rb][16 * kk + 8 + 2 * t]);
#pragma unroll
                    for (int nt = 0; nt < 8; nt++) {
                        uint32_t b0 = ld32(&sm.w2t[8 * nt + g][16 * kk + 2 * t]);
                        uint32_t b1 = ld32(&sm.w2t[8 * nt + g][16 * kk + 8 + 2 * t]);
                        mma16816(acc[nt], a, b0, b1);
                    }
                }
            }
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    int r = (e & 2) ? rb : ra;
                    int c = 8 * nt + 2 * t + (e & 1);
                    float v = acc[nt][e];
                    if (!(__bfloat162float(sm.h1t[c][r]) > 0.f)) v = 0.f;
                    db1[2 * nt + (e & 1)] += v;
                    __nv_bfloat16 hi = __float2bfloat16_rn(v);
                    sm.d1t[0][c][r] = hi;
                    sm.d1t[1][c][r] = __float2bfloat16_rn(v - __bfloat162float(hi));
                }
            }
        }
        __syncthreads();
        // weight gradients over the tile's rows (K = 64): slice w of dW1 and dW2
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            const int ma = 16 * w + g, mb = ma + 8;
#pragma unroll
            for (int part_ = 0; part_ < 2; part_++) {
                uint32_t a1[4], a2[4];
                a1[0] = ld32(&sm.d1t[part_][ma][16 * kk + 2 * t]);
                a1[1] = ld32(&sm.d1t[part_][mb][16 * kk + 2 * t]);
                a1[2] = ld32(&sm.d1t[part_][ma][16 * kk + 8 + 2 * t]);
                a1[3] = ld32(&sm.d1t[part_][mb][16 * kk + 8 + 2 * t]);
                a2[0] = ld32(&sm.d2t[part_][ma][16 * kk + 2 * t]);
                a2[1] = ld32(&sm.d2t[part_][mb][16 * kk + 2 * t]);
                a2[2] = ld32(&sm.d2t[part_][ma][16 * kk + 8 + 2 * t]);
                a2[3] = ld32(&sm.d2t[part_][mb][16 * kk + 8 + 2 * t]);
#pragma unroll
                for (int nt = 0; nt < 6; nt++) {
                    uint32_t b0 = ld32(&sm.xt[8 * nt + g][16 * kk + 2 * t]);
                    uint32_t b1 = ld32(&sm.xt[8 * nt + g][16 * kk + 8 + 2 * t]);
                    mma16816(g1[nt], a1, b0, b1);
                }
#pragma unroll
                for (int nt = 0; nt < 8; nt++) {
                    uint32_t b0 = ld32(&sm.h1t[8 * nt + g][16 * kk + 2 * t]);
                    uint32_t b1 = ld32(&sm.h1t[8 * nt + g][16 * kk + 8 + 2 * t]);
                    mma16816(g2[nt], a2, b0, b1);
                }
            }
        }
    }
    // this block's partial sums; grad_reduce_kernel adds the blocks in a fixed
    // order, so the gradient is the same bit for bit on every run
    float* mine = part + (int64_t)blockIdx.x * (N_PARAMS + 1);
    {
        const int ma = 16 * w + g, mb = ma + 8;
#pragma unroll
        for (int nt = 0; nt < 6; nt++) {
            int f = 8 * nt + 2 * t;
            mine[O_W1 + ma * NF + f] = g1[nt][0];
            mine[O_W1 + ma * NF + f + 1] = g1[nt][1];
            mine[O_W1 + mb * NF + f] = g1[nt][2];
            mine[O_W1 + mb * NF + f + 1] = g1[nt][3];
        }
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            int c = 8 * nt + 2 * t;
            mine[O_W2 + ma * NH + c] = g2[nt][0];
            mine[O_W2 + ma * NH + c + 1] = g2[nt][1];
            mine[O_W2 + mb * NH + c] = g2[nt][2];
            mine[O_W2 + mb * NH + c + 1] = g2[nt][3];
        }
    }
    // db1: sum this lane's rows over the 8 lanes of equal t, then the 4 warps
#pragma unroll
    for (int i = 0; i < 16; i++) {
        float v = db1[i];
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        db1[i] = v;
    }
    if (g == 0) {
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            sm.db1w[w][8 * nt + 2 * t] = db1[2 * nt];
            sm.db1w[w][8 * nt + 2 * t + 1] = db1[2 * nt + 1];
        }
    }
    __syncthreads();
    if (tid < NH) {
        float v = 0.f;
        for (int ww = 0; ww < 4; ww++) v += sm.db1w[ww][tid];
        mine[O_B1 + tid] = v;
    }
    __syncthreads();
    // db2, dW3: two threads per column (tid and tid + 64)
    sm.red[tid][0] = db2;
    sm.red[tid][1] = dw3[0];
    sm.red[tid][2] = dw3[1];
    sm.red[tid][3] = dw3[2];
    __syncthreads();
    if (tid < NH) {
        mine[O_B2 + tid] = sm.red[tid][0] + sm.red[tid + 64][0];
        for (int c = 0; c < 3; c++) mine[O_W3 + c * NH + tid] = sm.red[tid][1 + c] + sm.red[tid + 64][1 + c];
    }
    __syncthreads();
    // db3 and the loss: rows tid < 64
    sm.red[tid][0] = db3[0];
    sm.red[tid][1] = db3[1];
    sm.red[tid][2] = db3[2];
    sm.red[tid][3] = lsum;
    __syncthreads();
    if (tid < 4) {
        float v = 0.f;
        for (int r = 0; r < BT_ROWS; r++) v += sm.red[r][tid];
        if (tid < 3) mine[O_B3 + tid] = v;
        else mine[N_PARAMS] = v * inv_n;
    }
}

// grad[i] (and the loss, entry N_PARAMS) = sum of the blocks' partials in block order.
__global__ void grad_reduce_kernel(const float* __restrict__ part, int nblocks, float* grad,
                                   float* loss) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N_PARAMS) return;
    float v = 0.f;
    for (int b = 0; b < nblocks; b++) v += part[(int64_t)b * (N_PARAMS + 1) + i];
    if (i < N_PARAMS) grad[i] = v;
    else *loss = v;
}

// ------------------------------------------------------------------ Adam, init, sampling
// Adam (Kingma & Ba, ICLR 2015) with bias correction; t = step number (1-based).
__global__ void adam_kernel(float* prm, float* m, float* v, const float* grad, int t, float lr,
                            float b1, float b2, float eps) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N_PARAMS) return;
    float g = grad[i];
    float mi = b1 * m[i] + (1.f - b1) * g;
    float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / (1.f - powf(b1, (float)t));
    float vh = vi / (1.f - powf(b2, (float)t));
    prm[i] -= lr * mh / (sqrtf(vh) + eps);
}

// splitmix64 output function (Steele, Lea and Flood, OOPSLA 2014) of state x
__device__ inline u64 splitmix64(u64 x) {
    u64 z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void mlp_init_kernel(float* prm, u64 seed) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N_PARAMS) return;
    u64 h = splitmix64(seed * 0x100000001b3ull + (u64)i);
    float u = (float)(h >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f;  // exact, in [-1, 1)
    float v = 0.f;
    if (i < O_B1) v = u * sqrtf(6.0f / NF);
    else if (i >= O_W2 && i < O_B2) v = u * sqrtf(6.0f / NH);
    else if (i >= O_W3 && i < O_B3) v = u * sqrtf(3.0f / NH);
    prm[i] = v;
}

__global__ void sample_rows_kernel(const int* __restrict__ pool, int64_t npool, u64 seed,
                                   long long t, int b, int* rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b) return;
    u64 h = splitmix64(seed ^ ((u64)t << 32) ^ (u64)i);
    rows[i] = pool[h % (u64)npool];
}

__global__ void fallback_kernel(const float* __restrict__ mlp, const float* __restrict__ onorm,
                                const float* __restrict__ pca, int64_t n, float min_norm,
                                float* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool use = mlp && onorm[i] >= min_norm;
    const float* src = use ? mlp : pca;
    out[i * 3] = src[i * 3];
    out[i * 3 + 1] = src[i * 3 + 1];
    out[i * 3 + 2] = src[i * 3 + 2];
}

__global__ void iota_kernel(int* out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)i;
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_iota(int* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    iota_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_features(const int4* pos, const int* nbr, int S, int64_t n, uint16_t* feat,
                            float* pca, uint8_t* valid, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    features_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(pos, nbr, S, n, (uint4*)feat,
                                                                pca, valid);
    note_launch();
    return cudaGetLastError();
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

cudaError_t launch_mlp_forward(const float* prm, const uint16_t* feat, const int* rows, int64_t n,
                               float* outn, float* onorm, float* h1s, float* h2s, float* raw,
                               cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t tiles = (n + 15) / 16;
    int64_t blocks = (tiles + MLP_WARPS - 1) / MLP_WARPS;
    int64_t cap = (int64_t)sm_count() * MLP_BLOCKS_PER_SM;
    if (blocks > cap) blocks = cap;
    mlp_forward_kernel<<<(unsigned)blocks, MLP_WARPS * 32, 0, st>>>(
        prm, (const uint32_t*)feat, rows, n, outn, onorm, h1s, h2s, raw);
    note_launch();
    return cudaGetLastError();
}

static int64_t bt_blocks() { return (int64_t)sm_count() * BT_BLOCKS_PER_SM; }

int64_t mlp_backward_part_floats() { return bt_blocks() * (N_PARAMS + 1); }

cudaError_t launch_mlp_backward(const float* prm, const uint16_t* feat, const int* rows,
                                const float* labels, int64_t n, const float* h1s,
                                const float* h2s, const float* raw, float* grad, float* loss,
                                float* part, cudaStream_t st) {
    if (n <= 0) {
        cudaError_t e = cudaMemsetAsync(grad, 0, N_PARAMS * sizeof(float), st);
        if (!e) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
        return e;
    }
    static_assert(sizeof(BwSmem) <= 227 * 1024 / BT_BLOCKS_PER_SM, "backward shared memory");
    cudaError_t e = cudaFuncSetAttribute(mlp_backward_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(BwSmem));
    if (e) return e;
    int64_t tiles = (n + BT_ROWS - 1) / BT_ROWS;
    int64_t cap = bt_blocks();
    int64_t blocks = tiles < cap ? tiles : cap;
    mlp_backward_tc_kernel<<<(unsigned)blocks, BT_THREADS, sizeof(BwSmem), st>>>(
        prm, feat, rows, labels, n, h1s, h2s, raw, part);
    note_launch();
    grad_reduce_kernel<<<(N_PARAMS + 1 + 255) / 256, 256, 0, st>>>(part, (int)blocks, grad, loss);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_adam(float* prm, float* m, float* v, const float* grad, int t, float lr,
                        cudaStream_t st) {
    adam_kernel<<<(N_PARAMS + 255) / 256, 256, 0, st>>>(prm, m, v, grad, t, lr, 0.9f, 0.999f,
                                                        1e-8f);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_init(float* prm, u64 seed, cudaStream_t st) {
    mlp_init_kernel<<<(N_PARAMS + 255) / 256, 256, 0, st>>>(prm, seed);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sample_rows(const int* pool, int64_t npool, u64 seed, long long t, int b,
                               int* rows, cudaStream_t st) {
    if (b <= 0) return cudaSuccess;
    sample_rows_kernel<<<(b + 255) / 256, 256, 0, st>>>(pool, npool, seed, t, b, rows);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_normal_fallback(const float* mlp, const float* onorm, const float* pca,
                                   int64_t n, float min_norm, float* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    fallback_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mlp, onorm, pca, n, min_norm,
                                                                out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace pd

// ============================================================ C ABI (pd_normals.h)
using namespace pd;

#define NCK(x)                                                        \
    do {                                                              \
        cudaError_t e_ = (x);                                         \
        if (e_ != cudaSuccess) {                                      \
            if (ctx) api_error(ctx, "CUDA error at " #x, (long long)e_); \
            rc = e_ == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA; \
            goto done;                                                \
        }                                                             \
    } while (0)
#define NALLOC(ptr, type, count)                                                   \
    do {                                                                           \
        ptr = (type*)api_alloc(ctx, sizeof(type) * (size_t)(count), st);           \
        if (!ptr) {                                                                \
            api_error(ctx, "allocation failed: " #ptr, (long long)(count));       \
            rc = PD_ENOMEM;                                                        \
            goto done;                                                             \
        }                                                                          \
    } while (0)

extern "C" int pd_normals_pca(pd_grid* g, uint16_t* feat_dev, float* pca_dev, uint8_t* valid_dev,
                              void* stream) {
    if (!g || !feat_dev || !pca_dev) return PD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    GridNbrs nb;
    int rc = grid_knn16(g, st, &nb);
    if (rc) return rc;
    pd_ctx* ctx = nb.ctx;
    NCK(launch_features(nb.pos, nb.nbr, nb.S, nb.n, feat_dev, pca_dev, valid_dev, st));
    NCK(cudaStreamSynchronize(st));
done:
    return rc;
}

extern "C" int pd_mlp_init(float* params_dev, uint64_t seed, void* stream) {
    if (!params_dev) return PD_EINVAL;
    if (launch_mlp_init(params_dev, seed, (cudaStream_t)stream) != cudaSuccess) return PD_ECUDA;
    return PD_OK;
}

extern "C" int pd_mlp_forward(const float* params_dev, const uint16_t* feat_dev, int64_t n,
                              float* normals_dev, float* norm_dev, void* stream) {
    if (!params_dev || !feat_dev || n < 0 || (!normals_dev && !norm_dev)) return PD_EINVAL;
    cudaError_t e = launch_mlp_forward(params_dev, feat_dev, nullptr, n, normals_dev, norm_dev,
                                       nullptr, nullptr, nullptr, (cudaStream_t)stream);
    return e == cudaSuccess ? PD_OK : PD_ECUDA;
}

// Forward with stored activations and backward over `rows` (NULL = 0..n-1).
static int grad_pass(pd_ctx* ctx, const float* prm, const uint16_t* feat, const int* rows,
                     const float* labels, int64_t n, float* h1s, float* h2s, float* raw,
                     float* grad, float* loss, float* part, cudaStream_t st) {
    int rc = PD_OK;
    NCK(launch_mlp_forward(prm, feat, rows, n, nullptr, nullptr, h1s, h2s, raw, st));
    NCK(launch_mlp_backward(prm, feat, rows, labels, n, h1s, h2s, raw, grad, loss, part, st));
done:
    return rc;
}

extern "C" int pd_mlp_grad(pd_ctx* ctx, const float* params_dev, const uint16_t* feat_dev,
                           const float* labels_dev, int64_t n, float* grad_dev, float* loss_dev,
                           void* stream) {
    if (!ctx || !params_dev || !feat_dev || !labels_dev || !grad_dev || !loss_dev || n < 1)
        return PD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = PD_OK;
    float *h1s = nullptr, *h2s = nullptr, *raw = nullptr, *part = nullptr;
    NALLOC(h1s, float, n * NH);
    NALLOC(h2s, float, n * NH);
    NALLOC(raw, float, n * 3);
    NALLOC(part, float, mlp_backward_part_floats());
    rc = grad_pass(ctx, params_dev, feat_dev, nullptr, labels_dev, n, h1s, h2s, raw, grad_dev,
                   loss_dev, part, st);
    if (!rc) NCK(cudaStreamSynchronize(st));
done:
    api_free(ctx, h1s, st);
    api_free(ctx, h2s, st);
    api_free(ctx, raw, st);
    api_free(ctx, part, st);
    return rc;
}

extern "C" int pd_mlp_train(pd_ctx* ctx, float* params_dev, float* adam_dev, int step0,
                            const uint16_t* feat_dev, const float* labels_dev,
                            const uint8_t* valid_dev, int64_t n, const pd_train_params* tp,
                            float* loss_dev, void* stream) {
    if (!ctx || !params_dev || !adam_dev || !feat_dev || !labels_dev || !tp || n < 1 ||
        n >= (1ll << 31) || tp->steps < 0 || tp->batch < 1 || step0 < 0 || !(tp->lr > 0.f))
        return PD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = PD_OK;
    int b = tp->batch;
    int *pool = nullptr, *cnt = nullptr, *rows = nullptr;
    float *h1s = nullptr, *h2s = nullptr, *raw = nullptr, *grad = nullptr, *lossbuf = nullptr;
    float* part = nullptr;
    int npool = 0;
    NALLOC(pool, int, n);
    NALLOC(cnt, int, 1);
    NALLOC(rows, int, b);
    NALLOC(h1s, float, (int64_t)b * NH);
    NALLOC(h2s, float, (int64_t)b * NH);
    NALLOC(raw, float, (int64_t)b * 3);
    NALLOC(grad, float, N_PARAMS);
    NALLOC(lossbuf, float, 1);
    NALLOC(part, float, mlp_backward_part_floats());
    if (valid_dev) {
        Scratch s;
        struct Ctx {
            pd_ctx* c;
            cudaStream_t st;
        } cs = {ctx, st};
        s.alloc = [](void* self, size_t bytes) -> void* {
            Ctx* c = (Ctx*)self;
            return api_alloc(c->c, bytes, c->st);
        };
        s.free = [](void* self, void* p) {
            Ctx* c = (Ctx*)self;
            api_free(c->c, p, c->st);
        };
        s.self = &cs;
        NCK(stable_compact(valid_dev, n, pool, cnt, s, st));
        NCK(cudaMemcpyAsync(&npool, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
        NCK(cudaStreamSynchronize(st));
    } else {
        NCK(launch_iota(pool, n, st));
        npool = (int)n;
    }
    if (npool < 1) {
        api_error(ctx, "pd_mlp_train: no valid rows", 0);
        rc = PD_EINVAL;
        goto done;
    }
    for (int i = 0; i < tp->steps; i++) {
        int t = step0 + i + 1;
        NCK(launch_sample_rows(pool, npool, tp->seed, t, b, rows, st));
        float* lp = loss_dev ? loss_dev + i : lossbuf;
        rc = grad_pass(ctx, params_dev, feat_dev, rows, labels_dev, b, h1s, h2s, raw, grad, lp,
                       part, st);
        if (rc) goto done;
        NCK(launch_adam(params_dev, adam_dev, adam_dev + N_PARAMS, grad, t, tp->lr, st));
    }
    NCK(cudaStreamSynchronize(st));
done:
    void* bufs[] = {pool, cnt, rows, h1s, h2s, raw, grad, lossbuf, part};
    for (void* p : bufs) api_free(ctx, p, st);
    return rc;
}

extern "C" int pd_normals_mlp(pd_ctx* ctx, const float* params_dev, const uint16_t* feat_dev,
                              const float* pca_dev, int64_t n, float min_norm, float* normals_dev,
                              void* stream) {
    if (!ctx || !pca_dev || !normals_dev || n < 0 || (params_dev && !feat_dev)) return PD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = PD_OK;
    float *mlp = nullptr, *onorm = nullptr;
    if (min_norm <= 0.f) min_norm = 1e-3f;
    if (params_dev && n > 0) {
        NALLOC(mlp, float, n * 3);
        NALLOC(onorm, float, n);
        NCK(launch_mlp_forward(params_dev, feat_dev, nullptr, n, mlp, onorm, nullptr, nullptr,
                               nullptr, st));
    }
    NCK(launch_normal_fallback(mlp, onorm, pca_dev, n, min_norm, normals_dev, st));
done:
    api_free(ctx, mlp, st);
    api_free(ctx, onorm, st);
    return rc;
}
