// quality.cu -- kernels of the quality report of a decimated cloud.
//
// Section "Results and Discussion" (the cube experiment) judges a decimated
// cloud by the number of its points that fall within a growing neighbourhood
// of each retained point: with an even 2-D distribution the count grows
// linearly with the neighbourhood's area pi r^2, the regression slope is the
// density estimate, and R^2, RMSE and the spread of the fractile bands
// measure how even it is.  Eq. 2's quantity, the smallest nearest-neighbour
// spacing, is the Poisson-disk radius of the result.
//
//   radius_counts_kernel  one thread per retained point (Morton order): every
//                         point of the 3x3x3 cells around it at the level
//                         whose cell edge reaches the largest radius, binned
//                         by the first radius its squared distance fits in
//                         (exact int64); prefix sums give N_j(p) =
//                         #{q != p : d^2(p,q) <= r_j^2}.  Per radius: exact
//                         integer sums of N and N^2 and a histogram of N.
//   spacing_kernel        per-block minimum and sum of sqrt of the nearest
//                         squared distance (the k = 1 search's result), block
//                         partials added in block order on the host.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_internal.cuh"
#include "pd_kernels.h"

namespace pd {

#define QB 128  // threads per block of the counting kernel

__global__ void __launch_bounds__(QB) radius_counts_kernel(GridView g, int64_t n, int L,
                                                           const u64* __restrict__ r2, int nr,
                                                           u64* __restrict__ sum_n,
                                                           u64* __restrict__ sum_n2,
                                                           uint32_t* __restrict__ hist, int H) {
    __shared__ uint32_t s_bin[PD_QUALITY_MAXR][QB];
    __shared__ u64 s_sum[PD_QUALITY_MAXR], s_sum2[PD_QUALITY_MAXR];
    const int t = threadIdx.x;
    for (int j = t; j < PD_QUALITY_MAXR; j += QB) s_sum[j] = s_sum2[j] = 0;
    for (int j = 0; j < nr; j++) s_bin[j][t] = 0;
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)QB + t;
    if (s < n) {
        const int4 p = g.pos[s];
        const u64 rmax2 = r2[nr - 1];
        int cx = 0, cy = 0, cz = 0;
        if (L < g.B) {
            const u64 c0 = g.code[s];
            cx = (int)compact3(c0 >> (3 * L));
            cy = (int)compact3(c0 >> (3 * L + 1));
            cz = (int)compact3(c0 >> (3 * L + 2));
        }
        uint32_t seen_b[27];
        int nseen = 0;
        for (int o = 0; o < 27; o++) {
            uint32_t b, e;
            int lvl;
            int rt = resolve_cell(g, L, cx + o % 3 - 1, cy + (o / 3) % 3 - 1, cz + o / 9 - 1, b, e,
                                  &lvl);
            if (!rt) continue;
            if (rt == 2) {  // a coarser leaf reached from several cells is counted once
                bool dup = false;
                for (int i = 0; i < nseen; i++) dup |= seen_b[i] == b;
                if (dup) continue;
                seen_b[nseen++] = b;
            }
            for (uint32_t j = b; j < e; j++) {
                if ((int64_t)j == s) continue;
                const int4 q = g.pos[j];
                const long long dx = (long long)q.x - p.x, dy = (long long)q.y - p.y,
                                dz = (long long)q.z - p.z;
                const u64 d2 = (u64)(dx * dx + dy * dy + dz * dz);
                if (d2 > rmax2) continue;
                int lo = 0, hi = nr - 1;  // first radius with d^2 <= r_j^2
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (d2 <= r2[mid]) hi = mid;
                    else lo = mid + 1;
                }
                s_bin[lo][t]++;
            }
        }
        uint32_t run = 0;
        for (int j = 0; j < nr; j++) {
            run += s_bin[j][t];
            atomicAdd(&s_sum[j], (u64)run);
            atomicAdd(&s_sum2[j], (u64)run * (u64)run);
            atomicAdd(&hist[(int64_t)j * H + (run < (uint32_t)H ? run : (uint32_t)(H - 1))], 1u);
        }
    }
    __syncthreads();
    for (int j = t; j < nr; j += QB) {
        if (s_sum[j]) atomicAdd(&sum_n[j], s_sum[j]);
        if (s_sum2[j]) atomicAdd(&sum_n2[j], s_sum2[j]);
    }
}

cudaError_t launch_radius_counts(const GridView& g, int64_t n, int L, const u64* r2, int nr,
                                 u64* sum_n, u64* sum_n2, uint32_t* hist, int H,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (nr < 1 || nr > PD_QUALITY_MAXR) return cudaErrorInvalidValue;
    radius_counts_kernel<<<(unsigned)((n + QB - 1) / QB), QB, 0, st>>>(g, n, L, r2, nr, sum_n,
                                                                       sum_n2, hist, H);
    note_launch();
    return cudaGetLastError();
}

// Per block: the least nearest squared distance and the sum of the nearest
// distances (binary64, in a fixed order within the block).  ~0 = no neighbour.
__global__ void spacing_kernel(const u64* __restrict__ rk2, int64_t n, u64* __restrict__ bmin,
                               double* __restrict__ bsum) {
    __shared__ u64 s_min[256];
    __shared__ double s_sum[256];
    const int t = threadIdx.x;
    const int64_t s = blockIdx.x * (int64_t)256 + t;
    u64 v = s < n ? rk2[s] : ~0ull;
    s_min[t] = v;
    s_sum[t] = v == ~0ull ? 0.0 : __dsqrt_rn((double)v);
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (t < o) {
            s_min[t] = s_min[t + o] < s_min[t] ? s_min[t + o] : s_min[t];
            s_sum[t] = __dadd_rn(s_sum[t], s_sum[t + o]);
        }
        __syncthreads();
    }
    if (t == 0) {
        bmin[blockIdx.x] = s_min[0];
        bsum[blockIdx.x] = s_sum[0];
    }
}

cudaError_t launch_spacing(const u64* rk2, int64_t n, u64* bmin, double* bsum, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    spacing_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rk2, n, bmin, bsum);
    note_launch();
    return cudaGetLastError();
}

// Rows of an n x 3 int32 array at the listed positions (ascending input order).
__global__ void take_xyz_kernel(const int* __restrict__ list, const int* __restrict__ count,
                                const int32_t* __restrict__ xyz, int32_t* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= *count) return;
    const int64_t i = list[t];
    out[3 * t] = xyz[3 * i];
    out[3 * t + 1] = xyz[3 * i + 1];
    out[3 * t + 2] = xyz[3 * i + 2];
}

cudaError_t launch_take_xyz(const int* list, const int* count, int64_t cap, const int32_t* xyz,
                            int32_t* out, cudaStream_t st) {
    if (cap <= 0) return cudaSuccess;
    take_xyz_kernel<<<(unsigned)((cap + 255) / 256), 256, 0, st>>>(list, count, xyz, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace pd
