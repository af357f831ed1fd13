// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stkde {

// Tile footprint in the plane: TX rows of X by TY columns of Y = 128 voxels,
// one tensor-memory lane (one accumulator row) per voxel.
constexpr int TX = 16;
constexpr int TY = 8;
constexpr int TILE_XY = TX * TY;

// Device error word bits.
constexpr int ERRBIT_NONFINITE = 1;
constexpr int ERRBIT_TIMEOUT = 2;
constexpr int ERRBIT_BOUNDS = 4;

// Everything a launch needs about one problem.  Host computes it in FP64 and
// rounds the kernel's FP32 constants once.
struct Plan {
    // grid
    int gx, gy, gt;
    // bandwidths in voxels (FP32) and their reciprocals
    float hsv, htv, inv_hs, inv_ht;
    // kernel constants and normalisation 1/(n hs^2 ht) in domain units
    float cs, ct, norm;
    // event binning: cells = xy tiles, slabs of `slab` voxels in T
    int ntx, nty, slab, nslab;
    // bandwidth classes (per-event bandwidths only, else 1 x 1): class (a, b)
    // holds the events with hsv_i <= hsv / 2^a and htv_i <= htv / 2^b, binned apart
    // so that each class is read only around the tiles its own reach covers
    int ncls_s, ncls_t;
    uint32_t nkeys;          // classes*nslab*ntx*nty; key value nkeys marks an event that reaches no voxel
    int key_bits;
    // T blocks of the tile kernels
    int tblock, ntb;
    int64_t nitems;          // ntx * nty * ntb
    int n;                   // events
};

// One problem of a batched launch (a single problem is a batch of one): its
// plan, its inputs and output, and its offsets in the batch's concatenated event,
// bin-key and tile numberings.  Built on the host; the batch's table lives in
// device memory.
struct ProblemDev {
    Plan pl;
    const double* pts;        // n x 3 doubles, device memory
    double x0, y0, t0, sres, tres, isres, itres;
    int by_recip;             // both resolutions are powers of two: multiply by the exact reciprocal
    uint32_t key_base;        // first bin key of the problem (its keys: key_base .. key_base + nkeys)
    int64_t ev_base;          // first event of the problem in the batch's event numbering
    int64_t item_base;        // first tile of the problem in the batch's tile numbering
    int64_t fitem_base;       // the same in the fp32 tile kernel's numbering (64-voxel T blocks)
    const float4* ev;         // the batch's events sorted by key
    const uint32_t* start;    // the problem's bin boundaries start[0 .. nkeys]
    float* out;               // the problem's output grid, device memory
    const float4* evp;        // per-event bandwidths in sorted order (NULL: the plan's)
    int tx0, ntxg;            // the launch's tiles cover tile columns tx0 .. tx0 + ntxg - 1 (ntxg 0: all)
};

// Per-problem device buffers (views into the context's workspace).
struct Bins {
    const float4* ev;        // re-centred events sorted by key: (x', y', t', bits(original index))
    const uint32_t* start;   // start[k] = first sorted position with key >= k, k in [0, nkeys]
    // Per-event bandwidths in the same sorted order, (hsv_i, htv_i, 1/hsv_i,
    // 1/htv_i) in voxels, or NULL when every event takes the plan's.  With
    // per-event bandwidths the plan holds the largest ones (binning, tile reach
    // and the normalisation 1/(n hs_max^2 ht_max)); event i's terms are weighted
    // by (hs_max/hs_i)^2 (ht_max/ht_i).
    const float4* evp = nullptr;
};

// ----------------------------------------------------------------- prep.cu
// K0: re-centre (FP64) and cast to FP32, compute each event's bin key.
// evp: per-event bandwidth records in input order (their class joins the key), or NULL.
void launch_recentre(const double* pts, int n, double x0, double y0, double t0, double sres,
                     double tres, const Plan& pl, float4* ev, uint32_t* keys, uint32_t* idx,
                     int* err, cudaStream_t st, const float4* evp = nullptr);
// Stable LSD radix sort of (key, idx) pairs; result lands in keys/idx (tmp buffers used).
size_t radix_sort_temp_bytes(int n);
void launch_radix_sort(uint32_t* keys, uint32_t* idx, uint32_t* keys_tmp, uint32_t* idx_tmp,
                       uint32_t* block_hist, int n, int key_bits, cudaStream_t st);
// start[k] = lower_bound(sorted keys, k) for k in [0, nkeys]; gather events in sorted order.
void launch_bounds_gather(const uint32_t* sorted_keys, const uint32_t* sorted_idx,
                          const float4* ev, int n, uint32_t nkeys, uint32_t* start,
                          float4* ev_sorted, cudaStream_t st);
// Per-event bandwidths (domain units, n doubles each, device memory) to the
// (hsv, htv, 1/hsv, 1/htv) records of Bins::evp, in input order (FP64, rounded once).
void launch_bandwidths(const double* hs, const double* ht, int n, double sres, double tres,
                       float4* evp, cudaStream_t st);
// range[0..2] = bits of the smallest and largest of h[0..n) (n doubles, device
// memory), and a nonzero word if one is not finite and positive.  range must be
// preset to {~0, 0, 0}.
void launch_bandwidth_range(const double* h, int n, unsigned long long* range, cudaStream_t st);
// ev_sorted[p] = ev[idx[p]] (the gather of launch_bounds_gather, for a second array).
void launch_gather(const uint32_t* sorted_idx, const float4* ev, int n, float4* ev_sorted,
                   cudaStream_t st);
// ---------------------------------------------------------- abramson.cu
// Per-event bandwidths hs_i = hs lambda_i, ht_i = ht lambda_i from a pilot grid
// (device, gx*gy*gt floats) by Abramson's square-root law (see abramson.cu);
// events (device, n x 3) are read in input order.  scratch: abramson_scratch_bytes(n)
// of device memory.  Returns the number of kernels launched.
size_t abramson_scratch_bytes(int n);
int launch_abramson(const double* pts, int n, double x0, double y0, double t0, double sres,
                    double tres, int64_t gx, int64_t gy, int64_t gt, const float* pilot,
                    double alpha, double lam_min, double lam_max, double hs, double ht,
                    double* hs_out, double* ht_out, void* scratch, cudaStream_t st);

// Exact update count (FP64 on the binary32 re-centred events, in input order).
// hsv, htv: FP64 bandwidths in voxels; or per-event bandwidths hs, ht (domain
// units, device memory, n each; NULL for the fixed pair) divided by sres, tres.
void launch_count_updates(const float4* ev, int n, const Plan& pl, double hsv, double htv,
                          const double* hs, const double* ht, double sres, double tres,
                          unsigned long long* count, cudaStream_t st);

// ------------------------------------------------------------ tile_fp32.cu
// Returns false if the grid has 2^31 tiles or more or the kernel cannot be set up.
bool launch_tile_fp32(const Plan& pl, const Bins& b, float* out, int* err, cudaStream_t st);
// Tiles of the fp32 tile kernel for one problem.
int64_t tile_fp32_items(const Plan& pl);
// The fp32 tile kernel over every problem of a batch in one launch: `table` in
// device memory with fitem_base set to the running sum of tile_fp32_items;
// problems with n = 0 get zeros.  Returns false for 2^31 tiles or more.
bool launch_tile_fp32_batch(const ProblemDev* table, int nprob, int64_t total_items, cudaStream_t st);

// -------------------------------------------------------------- scatter.cu
void launch_scatter(const Plan& pl, const float4* ev, float* out, cudaStream_t st);

// -------------------------------------------------------------- tile_tc.cu
// Tiles of the tensor tile kernel, and the bytes of its tile-ordering scratch.
int64_t tile_tc_items(const Plan& pl);
size_t tile_order_bytes(const Plan& pl);
size_t tile_order_bytes_items(int64_t items);
// Returns false if the form is not compiled into the library (or the problem has
// 2^31 tiles or more).  tile_ctr: one device int, the launch's tile queue (zeroed
// here on the stream before the kernel).  order_ws: tile_order_bytes(pl) of device
// scratch for the heaviest-first tile order (two extra launches), or NULL to take
// the tiles in index order.
// tx0, ntxg: only the tiles of tile columns tx0 .. tx0 + ntxg - 1 (ntxg 0: all), so
// that a grid can be computed in slabs of X whose copies overlap later slabs.
// form: 0 bf16x3, 1 fp16x3, 2 tf32x3, 3 tf32x1 (the last two with fixed bandwidths only).
// wait: the bound of the kernel's waits in ns (0: the default of 2 s) and, for
// tests of the timeout path only, whether block 0 withholds the arrival of its
// first staging page (no copy is issued into that page).
struct TcWait {
    uint64_t wait_ns = 0;
    int withhold_page = 0;
};
bool launch_tile_tc(const Plan& pl, const Bins& b, float* out, int* err, int* tile_ctr,
                    uint32_t* order_ws, int form, cudaStream_t st, int tx0 = 0, int ntxg = 0,
                    TcWait wait = TcWait{});
// The same over the tiles of all problems of a batch in one launch: `table` is
// the batch's problem table in device memory (nprob entries, item_base set to
// the running sum of tile_tc_items), total_items the sum; order_ws holds
// tile_order_bytes_items(total_items).
bool launch_tile_tc_batch(const ProblemDev* table, int nprob, int64_t total_items, int* err,
                          int* tile_ctr, uint32_t* order_ws, int form, cudaStream_t st,
                          TcWait wait = TcWait{});
// Copies a host problem table into device memory through kernel parameters (up
// to 64 entries per launch), so that the copy needs no host buffer that outlives
// the call (and can be captured into a CUDA graph).  Returns the launches.
int launch_table_upload(const ProblemDev* host, int count, ProblemDev* dev, cudaStream_t st);
// K0 over all events of a batch: event i belongs to the problem whose ev_base
// range holds it; keys are offset by the problem's key_base.
void launch_recentre_batch(const ProblemDev* table, int nprob, int ntotal, float4* ev,
                           uint32_t* keys, uint32_t* idx, int* err, cudaStream_t st);

}  // namespace stkde
