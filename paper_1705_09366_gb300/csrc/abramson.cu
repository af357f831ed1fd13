// Per-event bandwidths that follow the population density (the adaptive
// bandwidth the conclusion, Section 8, names as future work), by Abramson's
// square-root law: a pilot density f~ computed with a fixed pair (hs, ht) is
// read at each event's voxel, floored at 1e-6 of the largest such value, and
// event i gets lambda_i = clamp((f~_i / g)^(-alpha), lam_min, lam_max) with g
// the geometric mean of the f~_i; hs_i = hs lambda_i, ht_i = ht lambda_i.
//
// All reductions are block trees of fixed shape followed by one single-block
// pass, so the result does not depend on scheduling.
#include "internal.cuh"

namespace stkde {

namespace {

constexpr int AB_THREADS = 256;
constexpr double AB_FLOOR = 1e-6;

// Block-wide tree reduction of v in shared memory (sum or max); thread 0 gets it.
__device__ __forceinline__ double block_reduce(double v, bool sum) {
    __shared__ double sm[AB_THREADS];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int s = AB_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] = sum ? sm[threadIdx.x] + sm[threadIdx.x + s]
                                                        : fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    return sm[0];
}

__device__ __forceinline__ int64_t voxel_of(double c, double c0, double res, int64_t g) {
    const double v = floor((c - c0) / res);
    if (!(v >= 0.0)) return 0;            // below the grid, or not finite
    if (v >= (double)(g - 1)) return g - 1;
    return (int64_t)v;
}

// f[i] = pilot at event i's voxel (clamped into the grid); bmax[block] = block max.
__global__ void k_pilot_sample(const double* __restrict__ pts, int n, double x0, double y0,
                               double t0, double sres, double tres, int64_t gx, int64_t gy,
                               int64_t gt, const float* __restrict__ pilot, double* __restrict__ f,
                               double* __restrict__ bmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < n) {
        const int64_t X = voxel_of(pts[3 * (size_t)i], x0, sres, gx);
        const int64_t Y = voxel_of(pts[3 * (size_t)i + 1], y0, sres, gy);
        const int64_t T = voxel_of(pts[3 * (size_t)i + 2], t0, tres, gt);
        v = (double)pilot[(X * gy + Y) * gt + T];
        f[i] = v;
    }
    const double m = block_reduce(v, false);
    if (threadIdx.x == 0) bmax[blockIdx.x] = m;
}

// out[0] = sum or max of a[0..m), one block, fixed order.
__global__ void k_reduce_one(const double* __restrict__ a, int m, int sum, double* __restrict__ out) {
    double v = 0.0;  // identity of both (the values are >= 0 for max)
    for (int j = threadIdx.x; j < m; j += AB_THREADS) v = sum ? v + a[j] : fmax(v, a[j]);
    const double r = block_reduce(v, sum != 0);
    if (threadIdx.x == 0) out[0] = r;
}

// bsum[block] = sum of log(max(f_i, floor)) over the block's events.
__global__ void k_log_partial(const double* __restrict__ f, int n, const double* __restrict__ fmx,
                              double* __restrict__ bsum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double fm = fmx[0];
    double v = 0.0;
    if (i < n && fm > 0.0) v = log(fmax(f[i], AB_FLOOR * fm));
    const double s = block_reduce(v, true);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

__global__ void k_lambda(const double* __restrict__ f, int n, const double* __restrict__ fmx,
                         const double* __restrict__ slog, double alpha, double lam_min,
                         double lam_max, double hs, double ht, double* __restrict__ hs_out,
                         double* __restrict__ ht_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double fm = fmx[0];
    double lam = 1.0;
    if (fm > 0.0) {
        const double g = exp(slog[0] / (double)n);
        lam = pow(fmax(f[i], AB_FLOOR * fm) / g, -alpha);
    }
    lam = lam < lam_min ? lam_min : lam > lam_max ? lam_max : lam;
    hs_out[i] = hs * lam;
    ht_out[i] = ht * lam;
}

}  // namespace

size_t abramson_scratch_bytes(int n) {
    const size_t nb = (size_t)((n + AB_THREADS - 1) / AB_THREADS);
    return sizeof(double) * ((size_t)n + 2 * nb + 4);
}

int launch_abramson(const double* pts, int n, double x0, double y0, double t0, double sres,
                    double tres, int64_t gx, int64_t gy, int64_t gt, const float* pilot,
                    double alpha, double lam_min, double lam_max, double hs, double ht,
                    double* hs_out, double* ht_out, void* scratch, cudaStream_t st) {
    if (n <= 0) return 0;
    const int nb = (n + AB_THREADS - 1) / AB_THREADS;
    double* f = static_cast<double*>(scratch);
    double* bmax = f + n;
    double* bsum = bmax + nb;
    double* scal = bsum + nb;  // [0] max, [1] sum of logs
    k_pilot_sample<<<nb, AB_THREADS, 0, st>>>(pts, n, x0, y0, t0, sres, tres, gx, gy, gt, pilot, f,
                                              bmax);
    k_reduce_one<<<1, AB_THREADS, 0, st>>>(bmax, nb, 0, scal);
    k_log_partial<<<nb, AB_THREADS, 0, st>>>(f, n, scal, bsum);
    k_reduce_one<<<1, AB_THREADS, 0, st>>>(bsum, nb, 1, scal + 1);
    k_lambda<<<nb, AB_THREADS, 0, st>>>(f, n, scal, scal + 1, alpha, lam_min, lam_max, hs, ht,
                                        hs_out, ht_out);
    return 5;
}

}  // namespace stkde
