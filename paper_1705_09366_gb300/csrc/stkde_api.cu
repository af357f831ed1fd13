// C ABI of the library (include/stkde.h): argument checking, the per-problem
// plan, the context-owned workspace and the launch sequence
//   K0 re-centre -> binning sort -> bin bounds + gather -> tile kernel.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include <nvtx3/nvToolsExt.h>

#include "../../include/stkde.h"
#include "../../include/stkde_testing.h"
#include "internal.cuh"

using namespace stkde;

namespace {

constexpr int MAX_PHASES = 5;
constexpr uint32_t MAX_KEYS = 1u << 25;
// Host outputs of the tensor forms: the tile kernel runs in up to MAX_SLABS slabs
// of X, each at least SLAB_MIN_BYTES of output, and each slab's copy to the host
// overlaps the later slabs' kernels.
constexpr int MAX_SLABS = 16;
constexpr size_t SLAB_MIN_BYTES = (size_t)64 << 20;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Each entry point's host-side work (checks, planning, enqueueing) is an NVTX range
// named after it, so profilers (Nsight Systems, Nsight Compute's --nvtx filters)
// can attribute launches to calls; without an attached tool a range costs a
// function-pointer check.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

struct stkde_ctx {
    stkde_options opt;
    cudaStream_t stream;
    int device;
    int sm_count;
    void* ws = nullptr;        // workspace
    size_t ws_bytes = 0;
    float* out_tmp = nullptr;  // device result buffer for host outputs
    size_t out_tmp_bytes = 0;
    int* d_err = nullptr;
    int* d_ctr = nullptr;  // tile queue of the tensor tile kernel
    unsigned long long* d_count = nullptr;
    unsigned long long* d_range = nullptr;  // bandwidth range of stkde_compute_adaptive (2 x 3 words)
    double* bw_stage = nullptr;             // device copies of host bandwidth arrays
    size_t bw_stage_bytes = 0;
    cudaEvent_t ev[MAX_PHASES + 1];
    int nphase = 0;
    bool events_ok = false;
    cudaStream_t copy_stream = nullptr;  // host-output copies of slabs
    cudaEvent_t slab_ev[MAX_SLABS] = {};
    cudaEvent_t copy_done = nullptr;
    bool slabs_ok = false;
    int launches = 0;          // kernels enqueued by the last compute call
    // test hooks (stkde_inject_fault): the allocation that fails (countdown, 0 =
    // none) and the next tensor tile launch's wait bound and withheld page
    int fail_alloc = 0;
    TcWait tc_wait{};
};

namespace {

struct Workspace {
    double* pts;
    float4* ev;
    float4* ev_sorted;
    uint32_t *keys, *idx, *keys_tmp, *idx_tmp, *hist, *start;
    uint32_t* order;  // tile-ordering scratch of the tensor tile kernel
};

// Carves the workspace for n events, nkeys bins and order_bytes of tile-ordering
// scratch; returns the bytes needed.
size_t carve(void* base, int n, uint32_t nkeys, bool host_points, size_t order_bytes, Workspace* w) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? static_cast<char*>(base) + off : nullptr;
        off = align_up(off + bytes, 256);
        return p;
    };
    const size_t nn = (size_t)(n > 0 ? n : 1);
    Workspace t;
    t.pts = reinterpret_cast<double*>(take(host_points ? 24 * nn : 0));
    t.ev = reinterpret_cast<float4*>(take(16 * nn));
    t.ev_sorted = reinterpret_cast<float4*>(take(16 * nn));
    t.keys = reinterpret_cast<uint32_t*>(take(4 * nn));
    t.idx = reinterpret_cast<uint32_t*>(take(4 * nn));
    t.keys_tmp = reinterpret_cast<uint32_t*>(take(4 * nn));
    t.idx_tmp = reinterpret_cast<uint32_t*>(take(4 * nn));
    t.hist = reinterpret_cast<uint32_t*>(take(radix_sort_temp_bytes(n)));
    t.start = reinterpret_cast<uint32_t*>(take(4 * ((size_t)nkeys + 1)));
    t.order = reinterpret_cast<uint32_t*>(take(order_bytes));
    if (w) *w = t;
    return off;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// The tensor tile kernel's form code of an API form (0 bf16x3, 1 fp16x3,
// 2 tf32x3, 3 tf32x1), or -1 for the forms that do not use it.
int tc_form(int form) {
    switch (form) {
        case STKDE_FORM_TENSOR_BF16X3: return 0;
        case STKDE_FORM_TENSOR_FP16X3: return 1;
        case STKDE_FORM_TENSOR_TF32X3: return 2;
        case STKDE_FORM_TENSOR_TF32X1: return 3;
        default: return -1;
    }
}

stkde_status check_problem(const double* points, int64_t n, const stkde_grid* g, double hs,
                           double ht) {
    if (!g) return STKDE_ERR_INVALID_ARGUMENT;
    if (n < 0 || n >= (int64_t)1 << 31) return STKDE_ERR_INVALID_ARGUMENT;
    if (n > 0 && !points) return STKDE_ERR_INVALID_ARGUMENT;
    if (!finite_pos(hs) || !finite_pos(ht) || !finite_pos(g->sres) || !finite_pos(g->tres))
        return STKDE_ERR_INVALID_ARGUMENT;
    if (!isfinite(g->x0) || !isfinite(g->y0) || !isfinite(g->t0)) return STKDE_ERR_INVALID_ARGUMENT;
    const int64_t lim = (int64_t)1 << 31;
    if (g->gx < 1 || g->gy < 1 || g->gt < 1 || g->gx >= lim || g->gy >= lim || g->gt >= lim)
        return STKDE_ERR_INVALID_ARGUMENT;
    // the grid must be addressable: gx*gy*gt < 2^60 voxels
    const double vox = (double)g->gx * (double)g->gy * (double)g->gt;
    if (vox >= 1.0e18) return STKDE_ERR_INVALID_ARGUMENT;
    const double hsv = hs / g->sres, htv = ht / g->tres;
    if (!(hsv < 1.0e6) || !(htv < 1.0e6)) return STKDE_ERR_INVALID_ARGUMENT;
    return STKDE_OK;
}

// The T extent of an event bin when the caller leaves it to the library. Shorter
// slabs mean more bin runs per tile for the loader to walk, longer ones more staged
// events that the tile filter rejects; measured on GB300 (small, medium and large
// workloads, slabs 2 to 64), the kind::f16 forms do best with the smallest power of
// two from 4 to 16 that puts at least 3.5 events in an average bin, the kind::tf32
// forms (twice the MMA entries per event, so staged events that the filter rejects
// cost them more) with at least 1.8, and the fp32 form, whose block-synchronous bin
// walk pays more per run, with 64.
int default_slab(int64_t n, int ntx, int nty, int gt, int form) {
    if (form == STKDE_FORM_FP32) return 64;
    const double per_bin =
        (form == STKDE_FORM_TENSOR_TF32X3 || form == STKDE_FORM_TENSOR_TF32X1) ? 1.8 : 3.5;
    int slab = 4;
    while (slab < 16) {
        const double bins = (double)ntx * (double)nty * (double)((gt + slab - 1) / slab);
        if ((double)n >= per_bin * bins) break;
        slab *= 2;
    }
    return slab;
}

// ncls_s x ncls_t bandwidth classes (per-event bandwidths; 1 x 1 otherwise).
// form: the stkde_form the plan is for (only the default slab depends on it).
Plan make_plan(int kernel_constants, int64_t n, const stkde_grid* g, double hs, double ht,
               int slab_opt, int form, int ncls_s = 1, int ncls_t = 1) {
    Plan p{};
    p.gx = (int)g->gx; p.gy = (int)g->gy; p.gt = (int)g->gt;
    const double hsv = hs / g->sres, htv = ht / g->tres;
    p.hsv = (float)hsv; p.htv = (float)htv;
    p.inv_hs = (float)(g->sres / hs);
    p.inv_ht = (float)(g->tres / ht);
    const double pi = 3.14159265358979323846;
    p.cs = (float)(kernel_constants == STKDE_KERNEL_UNIT_MASS ? 24.0 / (13.0 * pi) : pi / 2.0);
    p.ct = 0.75f;
    p.norm = n > 0 ? (float)(1.0 / ((double)n * hs * hs * ht)) : 0.0f;
    p.ntx = (p.gx + TX - 1) / TX;
    p.nty = (p.gy + TY - 1) / TY;
    p.ncls_s = ncls_s;
    p.ncls_t = ncls_t;
    const uint64_t ncls = (uint64_t)ncls_s * (uint64_t)ncls_t;
    int slab = slab_opt > 0 ? slab_opt : default_slab(n, p.ntx, p.nty, p.gt, form);
    slab = slab < p.gt ? slab : p.gt;
    while (true) {
        const uint64_t ns = (uint64_t)((p.gt + slab - 1) / slab);
        const uint64_t nk = ncls * ns * (uint64_t)p.ntx * (uint64_t)p.nty;
        if (nk <= MAX_KEYS || slab >= p.gt) break;
        slab *= 2;
    }
    p.slab = slab;
    p.nslab = (p.gt + slab - 1) / slab;
    const uint64_t nk = ncls * (uint64_t)p.nslab * (uint64_t)p.ntx * (uint64_t)p.nty;
    p.nkeys = (uint32_t)(nk < 0xffffffffull ? nk : 0xffffffffull);
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) <= (uint64_t)p.nkeys) ++bits;
    p.key_bits = bits;
    p.n = (int)n;
    p.tblock = 0; p.ntb = 0; p.nitems = 0;
    return p;
}

stkde_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return STKDE_OK;
    if (e == cudaErrorMemoryAllocation) return STKDE_ERR_OOM;
    return STKDE_ERR_CUDA;
}

// True while the context's stream is being captured into a CUDA graph: nothing
// may then allocate, wait for the stream or copy from pageable host memory.
bool capturing(const stkde_ctx* c) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Every device buffer a context grows is allocated here.  The test hook of
// stkde_inject_fault makes the k-th allocation from now on fail as it would on
// a device out of memory.
cudaError_t ctx_malloc(stkde_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (c->fail_alloc > 0 && --c->fail_alloc == 0) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
    }
    return e;
}

// Grows the context buffer *buf (of *have bytes) to hold `bytes`, allocating
// `want` >= bytes.  The old buffer is freed first (after the stream drains), so
// a failed growth leaves the buffer empty: nothing leaks and a later call
// starts over.  Under stream capture a buffer cannot grow: UNSUPPORTED.
stkde_status grow(stkde_ctx* c, void** buf, size_t* have, size_t bytes, size_t want) {
    if (bytes <= *have) return STKDE_OK;
    if (capturing(c)) return STKDE_ERR_UNSUPPORTED;
    cudaStreamSynchronize(c->stream);
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (ctx_malloc(c, buf, want) != cudaSuccess) return STKDE_ERR_OOM;
    *have = want;
    return STKDE_OK;
}

stkde_status ensure_ws(stkde_ctx* c, size_t bytes) {
    return grow(c, &c->ws, &c->ws_bytes, bytes, align_up(bytes + bytes / 8, 1 << 20));
}

// The context's device result buffer (host outputs, the pilot of
// stkde_abramson_bandwidths).
stkde_status ensure_out_tmp(stkde_ctx* c, size_t bytes) {
    return grow(c, reinterpret_cast<void**>(&c->out_tmp), &c->out_tmp_bytes, bytes, bytes);
}

// Is p a pointer the device can use directly?  Host (pageable or pinned) memory
// is copied instead.  -1: device memory of another device.
int pointer_kind(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return 0; }
    if (a.type == cudaMemoryTypeDevice) return a.device == device ? 1 : -1;
    if (a.type == cudaMemoryTypeManaged) return 1;
    return 0;
}

void mark(stkde_ctx* c) {
    if (c->opt.profile && c->events_ok && c->nphase <= MAX_PHASES)
        cudaEventRecord(c->ev[c->nphase++], c->stream);
}

// Enqueues one problem whose events are already on the device.  The result goes
// to the device buffer `out`.  With per-event bandwidths, evp holds their
// records in input order and evp_sorted receives them in bin order.  With
// host_out (a host buffer for the grid), a tensor-form grid of at least two slabs
// is computed slab by slab along X and each slab is copied to host_out on the
// context's copy stream while the next slabs compute; *copied tells the caller
// that the copy is enqueued (the context's stream waits for it).
stkde_status enqueue(stkde_ctx* c, const double* dpts, const Plan& pl, const stkde_grid* g,
                     const Workspace& w, float* out, const float4* evp = nullptr,
                     float4* evp_sorted = nullptr, float* host_out = nullptr,
                     bool* copied = nullptr) {
    if (copied) *copied = false;
    cudaStream_t st = c->stream;
    const int form = c->opt.form;
    const int n = pl.n;
    mark(c);
    launch_recentre(dpts, n, g->x0, g->y0, g->t0, g->sres, g->tres, pl, w.ev, w.keys, w.idx,
                    c->d_err, st, evp);
    c->launches += 1;
    if (form == STKDE_FORM_SCATTER) {
        mark(c);
        cudaMemsetAsync(out, 0, sizeof(float) * (size_t)pl.gx * pl.gy * pl.gt, st);
        mark(c);
        mark(c);
        launch_scatter(pl, w.ev, out, st);
        c->launches += 1;
        mark(c);
        return cuda_status(cudaGetLastError());
    }
    mark(c);
    launch_radix_sort(w.keys, w.idx, w.keys_tmp, w.idx_tmp, w.hist, n, pl.key_bits, st);
    c->launches += n > 1 ? 3 * ((pl.key_bits + 7) / 8) : 0;
    mark(c);
    launch_bounds_gather(w.keys, w.idx, w.ev, n, pl.nkeys, w.start, w.ev_sorted, st);
    c->launches += 2;
    if (evp) {
        launch_gather(w.idx, evp, n, evp_sorted, st);
        c->launches += 1;
    }
    mark(c);
    Bins b{w.ev_sorted, w.start, evp ? evp_sorted : nullptr};
    if (form == STKDE_FORM_FP32) {
        if (!launch_tile_fp32(pl, b, out, c->d_err, st)) return STKDE_ERR_UNSUPPORTED;
    } else {
        const int tcf = tc_form(form);
        const size_t row_bytes = sizeof(float) * (size_t)pl.gy * (size_t)pl.gt;  // one X row
        const size_t grid_bytes = row_bytes * (size_t)pl.gx;
        int nslab = 1;
        if (host_out && c->slabs_ok) {
            nslab = (int)(grid_bytes / SLAB_MIN_BYTES);
            nslab = nslab < MAX_SLABS ? nslab : MAX_SLABS;
            nslab = nslab < pl.ntx ? nslab : pl.ntx;
        }
        const TcWait tw = c->tc_wait;  // a test hook applies to one launch
        c->tc_wait = TcWait{};
        if (nslab < 2) {
            // heaviest tiles first (two small launches), then the tile kernel
            if (!launch_tile_tc(pl, b, out, c->d_err, c->d_ctr, w.order, tcf, st, 0, 0, tw))
                return STKDE_ERR_UNSUPPORTED;
            c->launches += 2;
        } else {
            // every kernel first, then every copy: a copy into pageable memory
            // may hold the calling thread until it is done
            int lo[MAX_SLABS + 1];
            for (int k = 0; k <= nslab; ++k) lo[k] = (int)((int64_t)pl.ntx * k / nslab);
            for (int k = 0; k < nslab; ++k) {
                if (!launch_tile_tc(pl, b, out, c->d_err, c->d_ctr, w.order, tcf, st, lo[k],
                                    lo[k + 1] - lo[k], k == 0 ? tw : TcWait{}))
                    return STKDE_ERR_UNSUPPORTED;
                cudaEventRecord(c->slab_ev[k], st);
            }
            c->launches += 3 * nslab - 1;
            for (int k = 0; k < nslab; ++k) {
                const size_t x0 = (size_t)lo[k] * TX;
                const size_t x1 = (size_t)(lo[k + 1] * TX < pl.gx ? lo[k + 1] * TX : pl.gx);
                cudaStreamWaitEvent(c->copy_stream, c->slab_ev[k], 0);
                cudaError_t e = cudaMemcpyAsync(host_out + x0 * (row_bytes / sizeof(float)),
                                                out + x0 * (row_bytes / sizeof(float)),
                                                (x1 - x0) * row_bytes, cudaMemcpyDeviceToHost,
                                                c->copy_stream);
                if (e != cudaSuccess) return cuda_status(e);
            }
            cudaEventRecord(c->copy_done, c->copy_stream);
            cudaStreamWaitEvent(st, c->copy_done, 0);
            if (copied) *copied = true;
        }
    }
    c->launches += 1;
    mark(c);
    return cuda_status(cudaGetLastError());
}

// Device copies of the per-event bandwidth arrays: device arrays are used in
// place, host arrays (kind 0) are copied on the stream into the context's staging
// buffer, which grows on demand.
stkde_status stage_bandwidths(stkde_ctx* c, int64_t n, const double*& hs, const double*& ht,
                              int hkind, int tkind) {
    const size_t nn = (size_t)n;
    const size_t need = sizeof(double) * ((hkind == 0 ? nn : 0) + (tkind == 0 ? nn : 0));
    if (need == 0) return STKDE_OK;
    const stkde_status s = grow(c, reinterpret_cast<void**>(&c->bw_stage), &c->bw_stage_bytes, need, need);
    if (s != STKDE_OK) return s;
    double* dst = c->bw_stage;
    cudaError_t e = cudaSuccess;
    if (hkind == 0) {
        e = cudaMemcpyAsync(dst, hs, sizeof(double) * nn, cudaMemcpyHostToDevice, c->stream);
        hs = dst;
        dst += nn;
    }
    if (e == cudaSuccess && tkind == 0) {
        e = cudaMemcpyAsync(dst, ht, sizeof(double) * nn, cudaMemcpyHostToDevice, c->stream);
        ht = dst;
    }
    return cuda_status(e);
}

// Smallest and largest of the per-event bandwidth arrays hs, ht (device memory):
// a reduction kernel per array and one wait for the stream; INVALID_ARGUMENT if
// one is not finite and positive.
stkde_status bandwidth_range(stkde_ctx* c, int64_t n, const double* hs, const double* ht,
                             double lo[2], double hi[2]) {
    const double* arr[2] = {hs, ht};
    unsigned long long init[6] = {~0ull, 0ull, 0ull, ~0ull, 0ull, 0ull};
    cudaError_t e = cudaMemcpyAsync(c->d_range, init, sizeof(init), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (int a = 0; a < 2; ++a) launch_bandwidth_range(arr[a], (int)n, c->d_range + 3 * a, c->stream);
    unsigned long long got[6];
    e = cudaMemcpyAsync(got, c->d_range, sizeof(got), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    bool bad = false;
    for (int a = 0; a < 2; ++a) {
        bad = bad || got[3 * a + 2] != 0;
        memcpy(&lo[a], &got[3 * a], sizeof(double));
        memcpy(&hi[a], &got[3 * a + 1], sizeof(double));
    }
    return bad ? STKDE_ERR_INVALID_ARGUMENT : STKDE_OK;
}

}  // namespace

namespace stkde {
stkde_status check_problem_args(const double* points, int64_t n, const stkde_grid* g, double hs,
                                double ht) {
    return check_problem(points, n, g, hs, ht);
}
Plan plan_problem(int kernel_constants, int64_t n, const stkde_grid* g, double hs, double ht, int form) {
    return make_plan(kernel_constants, n, g, hs, ht, 0, form);
}
}  // namespace stkde

extern "C" {

void stkde_default_options(stkde_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->device = 0;
    opt->stream = nullptr;
    opt->form = STKDE_FORM_TENSOR_BF16X3;
    opt->kernel_constants = STKDE_KERNEL_PRINTED;
}

const char* stkde_status_string(stkde_status s) {
    switch (s) {
        case STKDE_OK: return "ok";
        case STKDE_ERR_INVALID_ARGUMENT: return "invalid argument";
        case STKDE_ERR_OOM: return "out of device memory";
        case STKDE_ERR_CUDA: return "CUDA runtime error";
        case STKDE_ERR_TIMEOUT: return "device-side wait timed out";
        case STKDE_ERR_UNSUPPORTED: return "unsupported device or form";
        case STKDE_ERR_NONFINITE: return "non-finite event coordinate";
        case STKDE_ERR_INTERNAL: return "device-side consistency check failed";
    }
    return "unknown status";
}

stkde_status stkde_create(stkde_ctx** out, const stkde_options* opt) {
    if (!out) return STKDE_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    stkde_options o;
    if (opt) o = *opt; else stkde_default_options(&o);
    if (o.form < STKDE_FORM_TENSOR_BF16X3 || o.form > STKDE_FORM_TENSOR_TF32X1)
        return STKDE_ERR_INVALID_ARGUMENT;
    if (o.kernel_constants != STKDE_KERNEL_PRINTED && o.kernel_constants != STKDE_KERNEL_UNIT_MASS)
        return STKDE_ERR_INVALID_ARGUMENT;
    if (o.t_block != 0) return STKDE_ERR_INVALID_ARGUMENT;  // reserved
    if (o.slab < 0) return STKDE_ERR_INVALID_ARGUMENT;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return STKDE_ERR_UNSUPPORTED; }
    if (o.device < 0 || o.device >= ndev) return STKDE_ERR_INVALID_ARGUMENT;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, o.device) != cudaSuccess) return STKDE_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return STKDE_ERR_UNSUPPORTED;
    if (cudaSetDevice(o.device) != cudaSuccess) return STKDE_ERR_CUDA;
    stkde_ctx* c = new (std::nothrow) stkde_ctx;
    if (!c) return STKDE_ERR_OOM;
    c->opt = o;
    c->stream = static_cast<cudaStream_t>(o.stream);
    c->device = o.device;
    c->sm_count = prop.multiProcessorCount;
    if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_ctr, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_count, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_range, 6 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        if (c->d_err) cudaFree(c->d_err);
        if (c->d_ctr) cudaFree(c->d_ctr);
        if (c->d_count) cudaFree(c->d_count);
        delete c;
        return STKDE_ERR_OOM;
    }
    cudaMemset(c->d_err, 0, sizeof(int));
    c->events_ok = true;
    for (int i = 0; i <= MAX_PHASES; ++i)
        if (cudaEventCreate(&c->ev[i]) != cudaSuccess) c->events_ok = false;
    c->slabs_ok = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c->copy_done, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < MAX_SLABS && c->slabs_ok; ++i)
        c->slabs_ok = cudaEventCreateWithFlags(&c->slab_ev[i], cudaEventDisableTiming) == cudaSuccess;
    cudaGetLastError();
    cudaDeviceSynchronize();
    *out = c;
    return STKDE_OK;
}

void stkde_destroy(stkde_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->ws) cudaFree(c->ws);
    if (c->out_tmp) cudaFree(c->out_tmp);
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_ctr) cudaFree(c->d_ctr);
    if (c->d_count) cudaFree(c->d_count);
    if (c->d_range) cudaFree(c->d_range);
    if (c->bw_stage) cudaFree(c->bw_stage);
    for (int i = 0; i <= MAX_PHASES; ++i)
        if (c->events_ok) cudaEventDestroy(c->ev[i]);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->copy_done) cudaEventDestroy(c->copy_done);
    for (int i = 0; i < MAX_SLABS; ++i)
        if (c->slab_ev[i]) cudaEventDestroy(c->slab_ev[i]);
    delete c;
}

stkde_status stkde_synchronize(stkde_ctx* c) {
    const NvtxRange nvtx_range("stkde_synchronize");
    if (!c) return STKDE_ERR_INVALID_ARGUMENT;
    cudaSetDevice(c->device);
    if (capturing(c)) return STKDE_ERR_UNSUPPORTED;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    int h = 0;
    e = cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    if (h) cudaMemset(c->d_err, 0, sizeof(int));
    if (h & ERRBIT_NONFINITE) return STKDE_ERR_NONFINITE;
    if (h & ERRBIT_TIMEOUT) return STKDE_ERR_TIMEOUT;
    if (h & ERRBIT_BOUNDS) return STKDE_ERR_INTERNAL;
    return STKDE_OK;
}

stkde_status stkde_compute(stkde_ctx* c, const double* points, int64_t n, const stkde_grid* g,
                           double hs, double ht, float* out) {
    const NvtxRange nvtx_range("stkde_compute");
    if (!c || !out) return STKDE_ERR_INVALID_ARGUMENT;
    stkde_status s = check_problem(points, n, g, hs, ht);
    if (s != STKDE_OK) return s;
    if (cudaSetDevice(c->device) != cudaSuccess) return STKDE_ERR_CUDA;
    const int okind = pointer_kind(out, c->device);
    if (okind < 0) return STKDE_ERR_INVALID_ARGUMENT;
    const bool cap = capturing(c);
    if (cap && (okind == 0 || (n > 0 && pointer_kind(points, c->device) == 0)))
        return STKDE_ERR_UNSUPPORTED;  // host buffers cannot be part of a graph
    const size_t grid_bytes = sizeof(float) * (size_t)g->gx * (size_t)g->gy * (size_t)g->gt;
    float* dout = out;
    if (okind == 0) {  // host output: compute into the context's buffer, copy back
        const stkde_status so = ensure_out_tmp(c, grid_bytes);
        if (so != STKDE_OK) return so;
        dout = c->out_tmp;
    }
    c->nphase = 0;
    c->launches = 0;
    bool copied = false;
    if (n == 0) {
        cudaMemsetAsync(dout, 0, grid_bytes, c->stream);
    } else {
        if (c->opt.form == STKDE_FORM_SCATTER) {
            const double htv = ht / g->tres;
            if (2.0 * ceil(htv) + 1.0 > 12000.0) return STKDE_ERR_UNSUPPORTED;
        }
        const int pkind = pointer_kind(points, c->device);
        if (pkind < 0) return STKDE_ERR_INVALID_ARGUMENT;
        const Plan pl = make_plan(c->opt.kernel_constants, n, g, hs, ht, c->opt.slab, c->opt.form);
        Workspace w;
        const bool tensor = tc_form(c->opt.form) >= 0;
        const size_t order_bytes = tensor ? tile_order_bytes(pl) : 0;
        const size_t need = carve(nullptr, (int)n, pl.nkeys, pkind == 0, order_bytes, nullptr);
        s = ensure_ws(c, need);
        if (s != STKDE_OK) return s;
        carve(c->ws, (int)n, pl.nkeys, pkind == 0, order_bytes, &w);
        const double* dpts = points;
        if (pkind == 0) {
            cudaError_t e = cudaMemcpyAsync(w.pts, points, 24 * (size_t)n, cudaMemcpyHostToDevice,
                                            c->stream);
            if (e != cudaSuccess) return cuda_status(e);
            dpts = w.pts;
        }
        s = enqueue(c, dpts, pl, g, w, dout, nullptr, nullptr, okind == 0 ? out : nullptr, &copied);
        if (s != STKDE_OK) return s;
    }
    if (okind == 0 && !copied) {
        cudaError_t e = cudaMemcpyAsync(out, dout, grid_bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(cudaGetLastError());
}

// Per-event bandwidths: the range of both arrays is read first (on the host, or
// by a reduction kernel and one wait for the stream), the plan takes the largest
// pair, the arrays are converted to voxel records next to the re-centred events
// and gathered into bin order with them; the tile kernels weight each event by
// (hs_max/hs_i)^2 (ht_max/ht_i).
stkde_status stkde_compute_adaptive(stkde_ctx* c, const double* points, int64_t n,
                                    const stkde_grid* g, const double* hs, const double* ht,
                                    float* out) {
    const NvtxRange nvtx_range("stkde_compute_adaptive");
    if (!c || !out || !g) return STKDE_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!hs || !ht)) return STKDE_ERR_INVALID_ARGUMENT;
    // grid and event checks (the bandwidths are checked below)
    stkde_status s = check_problem(points, n, g, g->sres, g->tres);
    if (s != STKDE_OK) return s;
    if (c->opt.form == STKDE_FORM_SCATTER || c->opt.form == STKDE_FORM_TENSOR_TF32X3 ||
        c->opt.form == STKDE_FORM_TENSOR_TF32X1)
        return STKDE_ERR_UNSUPPORTED;
    if (n == 0) return stkde_compute(c, points, 0, g, g->sres, g->tres, out);
    if (cudaSetDevice(c->device) != cudaSuccess) return STKDE_ERR_CUDA;
    if (capturing(c)) return STKDE_ERR_UNSUPPORTED;  // waits for the stream
    const int okind = pointer_kind(out, c->device);
    const int pkind = pointer_kind(points, c->device);
    const int hkind = pointer_kind(hs, c->device), tkind = pointer_kind(ht, c->device);
    if (okind < 0 || pkind < 0 || hkind < 0 || tkind < 0) return STKDE_ERR_INVALID_ARGUMENT;

    const double* dhs = hs;
    const double* dht = ht;
    s = stage_bandwidths(c, n, dhs, dht, hkind, tkind);
    if (s != STKDE_OK) return s;
    double lo[2], hi[2];
    s = bandwidth_range(c, n, dhs, dht, lo, hi);
    if (s != STKDE_OK) return s;
    s = check_problem(points, n, g, hi[0], hi[1]);
    if (s != STKDE_OK) return s;
    if (c->opt.form == STKDE_FORM_TENSOR_FP16X3) {
        const double r = hi[0] / lo[0];
        if (r * r * (hi[1] / lo[1]) > 16384.0) return STKDE_ERR_UNSUPPORTED;
    }

    const size_t grid_bytes = sizeof(float) * (size_t)g->gx * (size_t)g->gy * (size_t)g->gt;
    float* dout = out;
    if (okind == 0) {
        const stkde_status so = ensure_out_tmp(c, grid_bytes);
        if (so != STKDE_OK) return so;
        dout = c->out_tmp;
    }
    // Bandwidth classes for the tensor forms: halvings of the largest spatial
    // bandwidth down to the smallest, at most 3, with 8-voxel T slabs (fewer,
    // longer bin runs per tile).  Temporal classes are not used: a 256-voxel T
    // block dwarfs the temporal reach, and each class multiplies the bin runs a
    // tile walks.  The fp32 form walks its bins in block-synchronous batches, so
    // more runs cost it more than the smaller reach saves: one class there.
    const bool tensor = c->opt.form != STKDE_FORM_FP32;
    int ncls_s = 1;
    if (tensor)
        while (ncls_s < 3 && hi[0] / lo[0] > (double)(1 << ncls_s)) ++ncls_s;
    const Plan pl = make_plan(c->opt.kernel_constants, n, g, hi[0], hi[1],
                              c->opt.slab > 0 ? c->opt.slab : (ncls_s > 1 ? 8 : 0), c->opt.form, ncls_s, 1);
    const size_t order_bytes = tensor ? tile_order_bytes(pl) : 0;
    const size_t nn = (size_t)n;
    // the problem's workspace, then the two bandwidth record arrays
    const size_t base = carve(nullptr, (int)n, pl.nkeys, pkind == 0, order_bytes, nullptr);
    const size_t o_evp = align_up(base, 256);
    const size_t o_evps = align_up(o_evp + 16 * nn, 256);
    s = ensure_ws(c, align_up(o_evps + 16 * nn, 256));
    if (s != STKDE_OK) return s;
    Workspace w;
    carve(c->ws, (int)n, pl.nkeys, pkind == 0, order_bytes, &w);
    char* wb = static_cast<char*>(c->ws);
    cudaError_t e = cudaSuccess;
    c->nphase = 0;
    c->launches = 0;
    const double* dpts = points;
    if (pkind == 0) {
        e = cudaMemcpyAsync(w.pts, points, 24 * nn, cudaMemcpyHostToDevice, c->stream);
        dpts = w.pts;
    }
    if (e != cudaSuccess) return cuda_status(e);
    float4* evp = reinterpret_cast<float4*>(wb + o_evp);
    float4* evps = reinterpret_cast<float4*>(wb + o_evps);
    launch_bandwidths(dhs, dht, (int)n, g->sres, g->tres, evp, c->stream);
    bool copied = false;
    s = enqueue(c, dpts, pl, g, w, dout, evp, evps, okind == 0 ? out : nullptr, &copied);
    c->launches += 3;  // two range reductions and the record conversion
    if (s != STKDE_OK) return s;
    if (okind == 0 && !copied) {
        e = cudaMemcpyAsync(out, dout, grid_bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(cudaGetLastError());
}

// Bandwidths from a pilot density: the pilot is stkde_compute with the fixed pair
// into `pilot` (or the context's result buffer), then five small kernels sample it
// at the events, reduce, and write hs_i, ht_i.
stkde_status stkde_abramson_bandwidths(stkde_ctx* c, const double* points, int64_t n,
                                       const stkde_grid* g, double hs, double ht, double alpha,
                                       double lam_min, double lam_max, float* pilot,
                                       double* hs_out, double* ht_out) {
    const NvtxRange nvtx_range("stkde_abramson_bandwidths");
    if (!c || !g) return STKDE_ERR_INVALID_ARGUMENT;
    stkde_status s = check_problem(points, n, g, hs, ht);
    if (s != STKDE_OK) return s;
    if (!(isfinite(alpha) && alpha >= 0.0) || !(lam_min > 0.0 && lam_min <= 1.0) ||
        !(isfinite(lam_max) && lam_max >= 1.0))
        return STKDE_ERR_INVALID_ARGUMENT;
    if (cudaSetDevice(c->device) != cudaSuccess) return STKDE_ERR_CUDA;
    if (capturing(c)) return STKDE_ERR_UNSUPPORTED;
    if (pilot && pointer_kind(pilot, c->device) != 1) return STKDE_ERR_INVALID_ARGUMENT;
    if (n == 0) return pilot ? stkde_compute(c, points, 0, g, hs, ht, pilot) : STKDE_OK;
    if (!hs_out || !ht_out || pointer_kind(hs_out, c->device) != 1 ||
        pointer_kind(ht_out, c->device) != 1)
        return STKDE_ERR_INVALID_ARGUMENT;
    const int pkind = pointer_kind(points, c->device);
    if (pkind < 0) return STKDE_ERR_INVALID_ARGUMENT;
    const size_t grid_bytes = sizeof(float) * (size_t)g->gx * (size_t)g->gy * (size_t)g->gt;
    float* dpil = pilot;
    if (!dpil) {  // the context's result buffer holds the pilot
        const stkde_status so = ensure_out_tmp(c, grid_bytes);
        if (so != STKDE_OK) return so;
        dpil = c->out_tmp;
    }
    s = stkde_compute(c, points, n, g, hs, ht, dpil);
    if (s != STKDE_OK) return s;
    const int launches = c->launches;
    // the workspace after the pilot's work (same stream): events (if host) and scratch
    const size_t o_pts = 0, o_scr = align_up(pkind == 0 ? 24 * (size_t)n : 0, 256);
    s = ensure_ws(c, o_scr + abramson_scratch_bytes((int)n));
    if (s != STKDE_OK) return s;
    char* wb = static_cast<char*>(c->ws);
    const double* dpts = points;
    if (pkind == 0) {
        cudaError_t e = cudaMemcpyAsync(wb + o_pts, points, 24 * (size_t)n, cudaMemcpyHostToDevice,
                                        c->stream);
        if (e != cudaSuccess) return cuda_status(e);
        dpts = reinterpret_cast<const double*>(wb + o_pts);
    }
    c->launches = launches + launch_abramson(dpts, (int)n, g->x0, g->y0, g->t0, g->sres, g->tres,
                                             g->gx, g->gy, g->gt, dpil, alpha, lam_min, lam_max,
                                             hs, ht, hs_out, ht_out, wb + o_scr, c->stream);
    return cuda_status(cudaGetLastError());
}

// Batched compute: one re-centre, one binning sort and one bounds + gather pass
// over the concatenated events of all problems (keys offset per problem, so the
// sort groups events by problem, then by bin), then one tile-kernel launch whose
// tile queue holds the tiles of every problem (heaviest first with the tensor
// forms; the fp32 form's grid numbers the tiles problem after problem).  Each
// problem's result equals its own stkde_compute with the same form: the same
// kernels see the same events in the same order.  The problem table reaches the
// device as kernel parameters, so with device events and a workspace that
// already fits, the call allocates nothing, waits for nothing and can be
// captured into a CUDA graph.
stkde_status stkde_compute_batch(stkde_ctx* c, const stkde_problem* probs, int count) {
    const NvtxRange nvtx_range("stkde_compute_batch");
    if (!c || (count > 0 && !probs) || count < 0) return STKDE_ERR_INVALID_ARGUMENT;
    if (count == 0) return STKDE_OK;
    const int form = c->opt.form;
    if (form == STKDE_FORM_SCATTER) return STKDE_ERR_UNSUPPORTED;
    const bool tensor = tc_form(form) >= 0;
    if (cudaSetDevice(c->device) != cudaSuccess) return STKDE_ERR_CUDA;
    const bool cap = capturing(c);

    // validate everything and lay the batch out before any launch
    ProblemDev* tab = new (std::nothrow) ProblemDev[count];
    int* pkinds = new (std::nothrow) int[count];
    if (!tab || !pkinds) {
        delete[] tab;
        delete[] pkinds;
        return STKDE_ERR_OOM;
    }
    struct Guard {
        ProblemDev* t; int* k;
        ~Guard() { delete[] t; delete[] k; }
    } guard{tab, pkinds};
    int64_t ntot = 0, itot = 0, ftot = 0, host_events = 0;
    uint64_t ktot = 0;
    for (int i = 0; i < count; ++i) {
        const stkde_problem& q = probs[i];
        stkde_status s = check_problem(q.points, q.n, &q.grid, q.hs, q.ht);
        if (s != STKDE_OK) return s;
        if (!q.out || pointer_kind(q.out, c->device) != 1) return STKDE_ERR_INVALID_ARGUMENT;
        pkinds[i] = q.n > 0 ? pointer_kind(q.points, c->device) : 1;
        if (pkinds[i] < 0) return STKDE_ERR_INVALID_ARGUMENT;
        if (pkinds[i] == 0 && cap) return STKDE_ERR_UNSUPPORTED;  // host events in a graph
        ProblemDev& P = tab[i];
        P = ProblemDev{};
        P.pl = make_plan(c->opt.kernel_constants, q.n, &q.grid, q.hs, q.ht, c->opt.slab, form);
        P.x0 = q.grid.x0; P.y0 = q.grid.y0; P.t0 = q.grid.t0;
        P.sres = q.grid.sres; P.tres = q.grid.tres;
        P.isres = 1.0 / q.grid.sres; P.itres = 1.0 / q.grid.tres;
        int e2;
        P.by_recip = (frexp(q.grid.sres, &e2) == 0.5) && (frexp(q.grid.tres, &e2) == 0.5);
        P.key_base = (uint32_t)ktot;
        P.ev_base = ntot;
        P.item_base = itot;
        P.fitem_base = ftot;
        ktot += (uint64_t)P.pl.nkeys + 1;  // the problem's bins and its "reaches nothing" key
        ntot += q.n;
        if (pkinds[i] == 0) host_events += q.n;
        if (tensor) itot += tile_tc_items(P.pl);
        else ftot += tile_fp32_items(P.pl);
        if (ntot >= ((int64_t)1 << 31) || ktot >= ((uint64_t)1 << 32) || itot >= ((int64_t)1 << 31) ||
            ftot >= ((int64_t)1 << 31))
            return STKDE_ERR_UNSUPPORTED;
    }

    // workspace: staging for host events, events, keys, sort scratch, bin bounds,
    // tile-order scratch, the problem table
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    const size_t nn = (size_t)(ntot > 0 ? ntot : 1);
    const size_t o_pts = take(24 * (size_t)host_events);
    const size_t o_ev = take(16 * nn), o_evs = take(16 * nn);
    const size_t o_keys = take(4 * nn), o_idx = take(4 * nn), o_kt = take(4 * nn), o_it = take(4 * nn);
    const size_t o_hist = take(radix_sort_temp_bytes((int)ntot));
    const size_t o_start = take(4 * (size_t)ktot);
    const size_t o_order = take(tensor ? tile_order_bytes_items(itot) : 0);
    const size_t o_tab = take(sizeof(ProblemDev) * (size_t)count);
    stkde_status s = ensure_ws(c, off);
    if (s != STKDE_OK) return s;
    char* base = static_cast<char*>(c->ws);
    double* staging = reinterpret_cast<double*>(base + o_pts);
    float4* ev = reinterpret_cast<float4*>(base + o_ev);
    float4* ev_sorted = reinterpret_cast<float4*>(base + o_evs);
    uint32_t* keys = reinterpret_cast<uint32_t*>(base + o_keys);
    uint32_t* idx = reinterpret_cast<uint32_t*>(base + o_idx);
    uint32_t* keys_tmp = reinterpret_cast<uint32_t*>(base + o_kt);
    uint32_t* idx_tmp = reinterpret_cast<uint32_t*>(base + o_it);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + o_hist);
    uint32_t* start = reinterpret_cast<uint32_t*>(base + o_start);
    uint32_t* order = tensor ? reinterpret_cast<uint32_t*>(base + o_order) : nullptr;
    ProblemDev* dtab = reinterpret_cast<ProblemDev*>(base + o_tab);

    cudaStream_t st = c->stream;
    c->nphase = 0;
    c->launches = 0;
    int64_t staged = 0;
    for (int i = 0; i < count; ++i) {
        ProblemDev& P = tab[i];
        P.pts = probs[i].points;
        if (pkinds[i] == 0 && probs[i].n > 0) {  // host events: copy into the staging area
            double* dst = staging + 3 * staged;
            const cudaError_t e = cudaMemcpyAsync(dst, probs[i].points, 24 * (size_t)probs[i].n,
                                                  cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_status(e);
            P.pts = dst;
            staged += probs[i].n;
        }
        P.ev = ev_sorted;
        P.start = start + P.key_base;
        P.out = probs[i].out;
    }
    c->launches += launch_table_upload(tab, count, dtab, st);
    int key_bits = 1;
    while (key_bits < 32 && ((uint64_t)1 << key_bits) <= ktot - 1) ++key_bits;

    mark(c);
    launch_recentre_batch(dtab, count, (int)ntot, ev, keys, idx, c->d_err, st);
    c->launches += ntot > 0 ? 1 : 0;
    mark(c);
    launch_radix_sort(keys, idx, keys_tmp, idx_tmp, hist, (int)ntot, key_bits, st);
    c->launches += ntot > 1 ? 3 * ((key_bits + 7) / 8) : 0;
    mark(c);
    launch_bounds_gather(keys, idx, ev, (int)ntot, (uint32_t)(ktot - 1), start, ev_sorted, st);
    c->launches += ntot > 0 ? 2 : 1;
    mark(c);
    if (tensor) {
        const TcWait tw = c->tc_wait;
        c->tc_wait = TcWait{};
        if (!launch_tile_tc_batch(dtab, count, itot, c->d_err, c->d_ctr, order, tc_form(form), st, tw))
            return STKDE_ERR_UNSUPPORTED;
        c->launches += itot > 0 ? 3 : 0;
    } else {
        if (!launch_tile_fp32_batch(dtab, count, ftot, st)) return STKDE_ERR_UNSUPPORTED;
        c->launches += ftot > 0 ? 1 : 0;
    }
    mark(c);
    return cuda_status(cudaGetLastError());
}

// Update count of one problem; hs_i/ht_i: per-event bandwidths (device memory,
// domain units) or NULL for the fixed pair hs, ht.  Host arrays are staged first.
static stkde_status count_updates(stkde_ctx* c, const double* points, int64_t n,
                                  const stkde_grid* g, double hs, double ht, const double* hs_i,
                                  const double* ht_i, int hkind, int tkind, uint64_t* count) {
    if (capturing(c)) return STKDE_ERR_UNSUPPORTED;  // synchronous
    const int pkind = pointer_kind(points, c->device);
    if (pkind < 0) return STKDE_ERR_INVALID_ARGUMENT;
    const Plan pl = make_plan(c->opt.kernel_constants, n, g, hs, ht, c->opt.slab, c->opt.form);
    Workspace w;
    const size_t nn = (size_t)n;
    const size_t base = carve(nullptr, (int)n, pl.nkeys, pkind == 0, 0, nullptr);
    const size_t o_hs = base, o_ht = align_up(o_hs + (hs_i && hkind == 0 ? 8 * nn : 0), 256);
    stkde_status s = ensure_ws(c, align_up(o_ht + (ht_i && tkind == 0 ? 8 * nn : 0), 256));
    if (s != STKDE_OK) return s;
    carve(c->ws, (int)n, pl.nkeys, pkind == 0, 0, &w);
    char* wb = static_cast<char*>(c->ws);
    const double* dpts = points;
    if (pkind == 0) {
        cudaMemcpyAsync(w.pts, points, 24 * nn, cudaMemcpyHostToDevice, c->stream);
        dpts = w.pts;
    }
    if (hs_i && hkind == 0) {
        cudaMemcpyAsync(wb + o_hs, hs_i, 8 * nn, cudaMemcpyHostToDevice, c->stream);
        hs_i = reinterpret_cast<const double*>(wb + o_hs);
    }
    if (ht_i && tkind == 0) {
        cudaMemcpyAsync(wb + o_ht, ht_i, 8 * nn, cudaMemcpyHostToDevice, c->stream);
        ht_i = reinterpret_cast<const double*>(wb + o_ht);
    }
    launch_recentre(dpts, (int)n, g->x0, g->y0, g->t0, g->sres, g->tres, pl, w.ev, w.keys, w.idx,
                    c->d_err, c->stream);
    cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), c->stream);
    launch_count_updates(w.ev, (int)n, pl, hs / g->sres, ht / g->tres, hs_i, ht_i, g->sres, g->tres,
                         c->d_count, c->stream);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, c->d_count, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    *count = h;
    return STKDE_OK;
}

stkde_status stkde_count_updates(stkde_ctx* c, const double* points, int64_t n,
                                 const stkde_grid* g, double hs, double ht, uint64_t* count) {
    const NvtxRange nvtx_range("stkde_count_updates");
    if (!c || !count) return STKDE_ERR_INVALID_ARGUMENT;
    stkde_status s = check_problem(points, n, g, hs, ht);
    if (s != STKDE_OK) return s;
    *count = 0;
    if (n == 0) return STKDE_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return STKDE_ERR_CUDA;
    return count_updates(c, points, n, g, hs, ht, nullptr, nullptr, 0, 0, count);
}

stkde_status stkde_count_updates_adaptive(stkde_ctx* c, const double* points, int64_t n,
                                          const stkde_grid* g, const double* hs, const double* ht,
                                          uint64_t* count) {
    const NvtxRange nvtx_range("stkde_count_updates_adaptive");
    if (!c || !count || !g) return STKDE_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!hs || !ht)) return STKDE_ERR_INVALID_ARGUMENT;
    stkde_status s = check_problem(points, n, g, g->sres, g->tres);
    if (s != STKDE_OK) return s;
    *count = 0;
    if (n == 0) return STKDE_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return STKDE_ERR_CUDA;
    if (capturing(c)) return STKDE_ERR_UNSUPPORTED;  // synchronous
    const int hkind = pointer_kind(hs, c->device), tkind = pointer_kind(ht, c->device);
    if (hkind < 0 || tkind < 0) return STKDE_ERR_INVALID_ARGUMENT;
    s = stage_bandwidths(c, n, hs, ht, hkind, tkind);
    if (s != STKDE_OK) return s;
    double lo[2], hi[2];
    s = bandwidth_range(c, n, hs, ht, lo, hi);
    if (s != STKDE_OK) return s;
    s = check_problem(points, n, g, hi[0], hi[1]);
    if (s != STKDE_OK) return s;
    return count_updates(c, points, n, g, hi[0], hi[1], hs, ht, 1, 1, count);
}

int stkde_last_launch_count(stkde_ctx* c) { return c ? c->launches : 0; }

stkde_status stkde_reserve(stkde_ctx* c, size_t bytes) {
    const NvtxRange nvtx_range("stkde_reserve");
    if (!c) return STKDE_ERR_INVALID_ARGUMENT;
    if (cudaSetDevice(c->device) != cudaSuccess) return STKDE_ERR_CUDA;
    return ensure_ws(c, bytes);
}

stkde_status stkde_inject_fault(stkde_ctx* c, int fault, int64_t arg) {
    if (!c) return STKDE_ERR_INVALID_ARGUMENT;
    switch (fault) {
        case STKDE_FAULT_NONE:
            c->fail_alloc = 0;
            c->tc_wait = TcWait{};
            return STKDE_OK;
        case STKDE_FAULT_ALLOC:
            if (arg < 1 || arg > (1 << 30)) return STKDE_ERR_INVALID_ARGUMENT;
            c->fail_alloc = (int)arg;
            return STKDE_OK;
        case STKDE_FAULT_WITHHOLD_PAGE:
            if (arg < 1 || arg > 2000000) return STKDE_ERR_INVALID_ARGUMENT;
            c->tc_wait.wait_ns = (uint64_t)arg * 1000u;
            c->tc_wait.withhold_page = 1;
            return STKDE_OK;
        default:
            return STKDE_ERR_INVALID_ARGUMENT;
    }
}

int stkde_phase_times(stkde_ctx* c, float* ms, int cap) {
    if (!c || !c->opt.profile || !c->events_ok || c->nphase < 2) return 0;
    cudaSetDevice(c->device);
    cudaEventSynchronize(c->ev[c->nphase - 1]);
    int k = 0;
    for (int i = 0; i + 1 < c->nphase && k < cap; ++i, ++k) {
        float t = 0.f;
        cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]);
        ms[k] = t;
    }
    return k;
}

}  // extern "C"
