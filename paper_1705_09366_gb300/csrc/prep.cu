// Event preparation: re-centre and cast (K0), bin by (T slab, xy cell) with a
// stable LSD radix sort (K1-K3), bin boundaries and the sorted event array.
//
// The binning realises the subdomain assignment of PB-SYM-DD (Section 4.2,
// Algorithm 5): an xy tile must see every event whose cylinder box intersects
// it.  Instead of replicating each event into every subdomain it touches, each
// event is stored once, in the bin of its own (slab, cell); a tile then reads
// the contiguous runs of bins around it.  Bins are ordered (slab, cell x,
// cell y), so for one slab and one cell row x the cells y_lo..y_hi form a
// single contiguous run of events.
#include "internal.cuh"

#include <string.h>

namespace stkde {

// ------------------------------------------------------------------- K0 ---

// Bandwidth class of an event with record r = (hsv_i, htv_i, 1/hsv_i, 1/htv_i):
// the largest (a, b) with hsv_i <= hsv / 2^a and htv_i <= htv / 2^b (a 10^-6
// margin absorbs the rounding of the ratio), capped at the plan's class counts.
__device__ __forceinline__ uint32_t bandwidth_class(const Plan& pl, float4 r) {
    int a = 0, b = 0;
    if (pl.ncls_s > 1) a = min(max(ilogbf(pl.hsv / r.x * (1.0f - 1.0e-6f)), 0), pl.ncls_s - 1);
    if (pl.ncls_t > 1) b = min(max(ilogbf(pl.htv / r.y * (1.0f - 1.0e-6f)), 0), pl.ncls_t - 1);
    return (uint32_t)(a * pl.ncls_t + b);
}

// Re-centres event i (row `row` of its problem's n x 3 array) and computes its
// bin key, offset by the problem's first key; with per-event bandwidth records
// (evp, input order) the event's bandwidth class leads the key.
__device__ __forceinline__ void recentre_one(const double* __restrict__ row, double x0, double y0,
                                             double t0, double sres, double tres, int by_recip,
                                             double isres, double itres, const Plan& pl,
                                             uint32_t key_base, int i, float4* __restrict__ ev,
                                             uint32_t* __restrict__ keys, uint32_t* __restrict__ idx,
                                             int* __restrict__ err,
                                             const float4* __restrict__ evp = nullptr) {
    const double x = row[0];
    const double y = row[1];
    const double t = row[2];
    // Re-centre on the grid origin in FP64 (the only FP64 step of the path), then
    // round to binary32.  Division unless the resolution is a power of two, where
    // multiplying by the exact reciprocal gives the same bits.
    double px, py, pt;
    if (by_recip) {
        px = (x - x0) * isres;
        py = (y - y0) * isres;
        pt = (t - t0) * itres;
    } else {
        px = (x - x0) / sres;
        py = (y - y0) / sres;
        pt = (t - t0) / tres;
    }
    const float fx = __double2float_rn(px);
    const float fy = __double2float_rn(py);
    const float ft = __double2float_rn(pt);
    uint32_t key = pl.nkeys;  // reaches no voxel
    if (!(isfinite(x) && isfinite(y) && isfinite(t))) {
        atomicOr(err, ERRBIT_NONFINITE);
    } else if (fx > -pl.hsv - 1.0f && fx < (float)pl.gx + pl.hsv + 1.0f &&
               fy > -pl.hsv - 1.0f && fy < (float)pl.gy + pl.hsv + 1.0f &&
               ft > -pl.htv - 1.0f && ft < (float)pl.gt + pl.htv + 1.0f) {
        // Clamping moves an event outside the grid into the nearest edge cell or
        // slab, which is no farther from any in-grid tile than the event is.
        const int cx = min(max((int)floorf(fx * (1.0f / TX)), 0), pl.ntx - 1);
        const int cy = min(max((int)floorf(fy * (1.0f / TY)), 0), pl.nty - 1);
        const int s = min(max((int)floorf(ft / (float)pl.slab), 0), pl.nslab - 1);
        const uint32_t cls = evp ? bandwidth_class(pl, evp[i]) : 0u;
        key = (((cls * (uint32_t)pl.nslab + (uint32_t)s) * (uint32_t)pl.ntx + (uint32_t)cx) *
               (uint32_t)pl.nty) + (uint32_t)cy;
    }
    ev[i] = make_float4(fx, fy, ft, __int_as_float(i));
    keys[i] = key_base + key;
    idx[i] = (uint32_t)i;
}

__global__ void k_recentre(const double* __restrict__ pts, int n, double x0, double y0,
                           double t0, double sres, double tres, int by_recip, double isres,
                           double itres, Plan pl, float4* __restrict__ ev,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ idx,
                           int* __restrict__ err, const float4* __restrict__ evp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    recentre_one(pts + 3 * (size_t)i, x0, y0, t0, sres, tres, by_recip, isres, itres, pl, 0u, i,
                 ev, keys, idx, err, evp);
}

void launch_recentre(const double* pts, int n, double x0, double y0, double t0, double sres,
                     double tres, const Plan& pl, float4* ev, uint32_t* keys, uint32_t* idx,
                     int* err, cudaStream_t st, const float4* evp) {
    if (n <= 0) return;
    int e;
    const bool p2 = (frexp(sres, &e) == 0.5) && (frexp(tres, &e) == 0.5);
    k_recentre<<<(n + 255) / 256, 256, 0, st>>>(pts, n, x0, y0, t0, sres, tres, p2 ? 1 : 0,
                                               1.0 / sres, 1.0 / tres, pl, ev, keys, idx, err, evp);
}

// The same over a batch: event i belongs to the last problem whose ev_base <= i.
__global__ void k_recentre_batch(const ProblemDev* __restrict__ table, int nprob, int ntotal,
                                 float4* __restrict__ ev, uint32_t* __restrict__ keys,
                                 uint32_t* __restrict__ idx, int* __restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntotal) return;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (table[mid].ev_base <= i) lo = mid; else hi = mid - 1;
    }
    const ProblemDev& P = table[lo];
    recentre_one(P.pts + 3 * (size_t)(i - P.ev_base), P.x0, P.y0, P.t0, P.sres, P.tres, P.by_recip,
                 P.isres, P.itres, P.pl, P.key_base, i, ev, keys, idx, err);
}

void launch_recentre_batch(const ProblemDev* table, int nprob, int ntotal, float4* ev,
                           uint32_t* keys, uint32_t* idx, int* err, cudaStream_t st) {
    if (ntotal <= 0 || nprob <= 0) return;
    k_recentre_batch<<<(ntotal + 255) / 256, 256, 0, st>>>(table, nprob, ntotal, ev, keys, idx, err);
}

// ------------------------------------------------------- table upload ---
// The batch's problem table travels as kernel parameters: the launch copies the
// argument values at enqueue time, so no host buffer has to outlive the call and
// the copy can be captured into a graph (a captured cudaMemcpyAsync would read
// its host source at every replay instead).
constexpr int UPLOAD_CHUNK = 64;  // entries per launch (about 14 KB of parameters)

struct TableChunk {
    ProblemDev p[UPLOAD_CHUNK];
};

__global__ void k_table_upload(TableChunk chunk, int count, ProblemDev* __restrict__ dst) {
    constexpr int WORDS = sizeof(ProblemDev) / sizeof(uint32_t);
    static_assert(sizeof(ProblemDev) % sizeof(uint32_t) == 0, "table entries are whole words");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(chunk.p);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (int w = threadIdx.x; w < count * WORDS; w += blockDim.x) d[w] = src[w];
}

int launch_table_upload(const ProblemDev* host, int count, ProblemDev* dev, cudaStream_t st) {
    int launches = 0;
    for (int i = 0; i < count; i += UPLOAD_CHUNK) {
        const int m = count - i < UPLOAD_CHUNK ? count - i : UPLOAD_CHUNK;
        TableChunk c;
        memcpy(c.p, host + i, sizeof(ProblemDev) * (size_t)m);
        k_table_upload<<<1, 256, 0, st>>>(c, m, dev + i);
        ++launches;
    }
    return launches;
}

// ---------------------------------------------------------- radix sort ---
// LSD radix sort, 8-bit digits.  Each pass: per-block digit histograms, an
// exclusive scan over the blocks per digit (one CTA per digit) plus the digit
// totals, then a stable scatter in which a block
// ranks its keys round by round (256 keys a round, warp-level match for equal
// digits, warps combined in order), so equal digits keep their input order.

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_BINS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS)
k_rs_hist(const uint32_t* __restrict__ keys, int n, int shift, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[RS_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_TILE;
#pragma unroll
    for (int j = 0; j < RS_ROUNDS; ++j) {
        const int p = base + j * RS_THREADS + threadIdx.x;
        if (p < n) atomicAdd(&h[(keys[p] >> shift) & (RS_BINS - 1)], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of one digit's counts over the blocks, in place: one CTA per
// digit, block-wide scan in tiles of RS_THREADS; the digit's total goes to
// totals[digit].
__global__ void __launch_bounds__(RS_THREADS)
k_rs_scan_digit(uint32_t* __restrict__ hist, int nb, uint32_t* __restrict__ totals) {
    __shared__ uint32_t wsum[RS_WARPS];
    __shared__ uint32_t carry;
    uint32_t* a = hist + (size_t)blockIdx.x * nb;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += RS_THREADS) {
        const int i = base + tid;
        const uint32_t v = i < nb ? a[i] : 0u;
        uint32_t x = v;  // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t pre = carry;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) pre += w < warp ? wsum[w] : 0u;
        if (i < nb) a[i] = pre + x - v;
        __syncthreads();
        if (tid == RS_THREADS - 1) carry = pre + x;
        __syncthreads();
    }
    if (tid == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ iin,
             uint32_t* __restrict__ kout, uint32_t* __restrict__ iout, int n, int shift,
             const uint32_t* __restrict__ offs, const uint32_t* __restrict__ totals) {
    __shared__ uint32_t run[RS_BINS];
    __shared__ uint32_t wc[RS_WARPS][RS_BINS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        // base of this thread's digit = sum of the totals of smaller digits
        const uint32_t t = totals[tid];
        uint32_t x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wc[0][warp] = x;
        __syncthreads();
        uint32_t pre = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) pre += w < warp ? wc[0][w] : 0u;
        run[tid] = pre + x - t + offs[(size_t)tid * gridDim.x + blockIdx.x];
        __syncthreads();
    }
    const int base = blockIdx.x * RS_TILE;
    const uint32_t lt = (1u << lane) - 1u;
    for (int j = 0; j < RS_ROUNDS; ++j) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) wc[w][tid] = 0;
        __syncthreads();
        const int p = base + j * RS_THREADS + tid;
        const bool valid = p < n;
        const uint32_t k = valid ? kin[p] : 0u;
        const uint32_t d = valid ? ((k >> shift) & (RS_BINS - 1)) : (uint32_t)RS_BINS;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wc[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t r = run[tid];
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                const uint32_t c = wc[w][tid];
                wc[w][tid] = r;
                r += c;
            }
            run[tid] = r;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wc[warp][d] + rank;
            kout[pos] = k;
            iout[pos] = iin[p];
        }
        __syncthreads();
    }
}

size_t radix_sort_temp_bytes(int n) {
    const int nb = (n + RS_TILE - 1) / RS_TILE;
    return ((size_t)RS_BINS * (size_t)(nb > 0 ? nb : 1) + RS_BINS) * sizeof(uint32_t);
}

void launch_radix_sort(uint32_t* keys, uint32_t* idx, uint32_t* keys_tmp, uint32_t* idx_tmp,
                       uint32_t* block_hist, int n, int key_bits, cudaStream_t st) {
    if (n <= 1) return;
    const int nb = (n + RS_TILE - 1) / RS_TILE;
    const int passes = (key_bits + 7) / 8;
    uint32_t *ka = keys, *ia = idx, *kb = keys_tmp, *ib = idx_tmp;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = 8 * ps;
        uint32_t* totals = block_hist + (size_t)RS_BINS * nb;
        k_rs_hist<<<nb, RS_THREADS, 0, st>>>(ka, n, shift, block_hist);
        k_rs_scan_digit<<<RS_BINS, RS_THREADS, 0, st>>>(block_hist, nb, totals);
        k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(ka, ia, kb, ib, n, shift, block_hist, totals);
        uint32_t* t = ka; ka = kb; kb = t;
        t = ia; ia = ib; ib = t;
    }
    if (ka != keys) {
        cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(idx, ia, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    }
}

// ------------------------------------------------ bounds and gather ---

__global__ void k_bounds(const uint32_t* __restrict__ keys, int n, uint32_t nkeys,
                         uint32_t* __restrict__ start) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nkeys) return;
    int lo = 0, hi = n;  // first position with keys[pos] >= k
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    start[k] = (uint32_t)lo;
}

__global__ void k_gather(const uint32_t* __restrict__ idx, const float4* __restrict__ ev, int n,
                         float4* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) out[p] = ev[idx[p]];
}

void launch_bounds_gather(const uint32_t* sorted_keys, const uint32_t* sorted_idx,
                          const float4* ev, int n, uint32_t nkeys, uint32_t* start,
                          float4* ev_sorted, cudaStream_t st) {
    const uint32_t nk = nkeys + 1;
    k_bounds<<<(nk + 255) / 256, 256, 0, st>>>(sorted_keys, n, nkeys, start);
    if (n > 0) k_gather<<<(n + 255) / 256, 256, 0, st>>>(sorted_idx, ev, n, ev_sorted);
}

void launch_gather(const uint32_t* sorted_idx, const float4* ev, int n, float4* ev_sorted,
                   cudaStream_t st) {
    if (n > 0) k_gather<<<(n + 255) / 256, 256, 0, st>>>(sorted_idx, ev, n, ev_sorted);
}

// ----------------------------------------------- per-event bandwidths ---
// Adaptive bandwidths (the density-dependent bandwidth the conclusion names as
// future work): event i carries its own hs_i, ht_i.  Converted once to voxels in
// FP64 as the plan converts the fixed ones, then rounded.

__global__ void k_bandwidths(const double* __restrict__ hs, const double* __restrict__ ht, int n,
                             double sres, double tres, float4* __restrict__ evp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h = hs[i], k = ht[i];
    evp[i] = make_float4(__double2float_rn(h / sres), __double2float_rn(k / tres),
                         __double2float_rn(sres / h), __double2float_rn(tres / k));
}

void launch_bandwidths(const double* hs, const double* ht, int n, double sres, double tres,
                       float4* evp, cudaStream_t st) {
    if (n > 0) k_bandwidths<<<(n + 255) / 256, 256, 0, st>>>(hs, ht, n, sres, tres, evp);
}

// Positive finite doubles order as their bit patterns, so the extrema are
// unsigned integer min/max of the bits.
__global__ void k_bandwidth_range(const double* __restrict__ h, int n,
                                  unsigned long long* __restrict__ range) {
    unsigned long long lo = ~0ull, hi = 0, bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = h[i];
        if (!(isfinite(v) && v > 0.0)) { bad = 1; continue; }
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        lo = min(lo, b);
        hi = max(hi, b);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&range[0], lo);
        atomicMax(&range[1], hi);
        if (bad) atomicOr(&range[2], bad);
    }
}

void launch_bandwidth_range(const double* h, int n, unsigned long long* range, cudaStream_t st) {
    if (n <= 0) return;
    int blocks = (n + 255) / 256;
    blocks = blocks < 1024 ? blocks : 1024;
    k_bandwidth_range<<<blocks, 256, 0, st>>>(h, n, range);
}

// --------------------------------------------------------- update count ---
// Exact count of (event, in-grid voxel) pairs inside the cylinder, FP64 on the
// binary32 events.  Per event: the T count times the xy count; along each X row
// the inside set is an interval in Y (the disk is convex), located by a square
// root estimate and then settled by exact tests at both ends.

__device__ __forceinline__ bool inside_xy(double du, double py, int Y, double hs) {
    const double dv = ((double)Y + 0.5 - py) / hs;
    return du * du + dv * dv < 1.0;
}

__global__ void k_count(const float4* __restrict__ ev, int n, int gx, int gy, int gt, double hs0,
                        double ht0, const double* __restrict__ hs_i, const double* __restrict__ ht_i,
                        double sres, double tres, unsigned long long* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (i < n) {
        const float4 e = ev[i];
        // per-event bandwidths in voxels (events are in input order here)
        const double hs = hs_i ? hs_i[i] / sres : hs0;
        const double ht = ht_i ? ht_i[i] / tres : ht0;
        const double px = e.x, py = e.y, pt = e.z;
        if (isfinite(px) && isfinite(py) && isfinite(pt) && fabs(px) < 1e9 && fabs(py) < 1e9 &&
            fabs(pt) < 1e9) {
            const long long Ht = (long long)ceil(ht), Hs = (long long)ceil(hs);
            const long long Ti = (long long)floor(pt), Xi = (long long)floor(px);
            const long long Yi = (long long)floor(py);
            long long nt = 0;
            for (long long T = max(0LL, Ti - Ht); T <= min((long long)gt - 1, Ti + Ht); ++T) {
                const double w = ((double)T + 0.5 - pt) / ht;
                nt += fabs(w) <= 1.0;
            }
            long long nxy = 0;
            if (nt > 0) {
                const long long ylo0 = max(0LL, Yi - Hs), yhi0 = min((long long)gy - 1, Yi + Hs);
                for (long long X = max(0LL, Xi - Hs); X <= min((long long)gx - 1, Xi + Hs); ++X) {
                    const double du = ((double)X + 0.5 - px) / hs;
                    const double r2 = 1.0 - du * du;
                    if (r2 <= 0.0 || ylo0 > yhi0) continue;
                    const double hw = sqrt(r2) * hs;
                    long long lo = max(ylo0, (long long)floor(py - 0.5 - hw) - 1);
                    long long hi = min(yhi0, (long long)ceil(py - 0.5 + hw) + 1);
                    while (lo <= hi && !inside_xy(du, py, (int)lo, hs)) ++lo;
                    while (hi >= lo && !inside_xy(du, py, (int)hi, hs)) --hi;
                    if (hi >= lo) nxy += hi - lo + 1;
                }
            }
            c = (unsigned long long)(nxy * nt);
        }
    }
    // warp reduce then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

void launch_count_updates(const float4* ev, int n, const Plan& pl, double hsv, double htv,
                          const double* hs, const double* ht, double sres, double tres,
                          unsigned long long* count, cudaStream_t st) {
    if (n <= 0) return;
    k_count<<<(n + 255) / 256, 256, 0, st>>>(ev, n, pl.gx, pl.gy, pl.gt, hsv, htv, hs, ht, sres,
                                             tres, count);
}

}  // namespace stkde
