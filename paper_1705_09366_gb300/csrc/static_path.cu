// stkde_compute_static: the density of stkde_compute for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs where another
// component owns every device allocation (a host application's or framework's
// caching allocator or memory pool, an arena reserved up front), or a loop that
// must not take the implicit device-wide synchronisation of cudaMalloc/cudaFree.
// For them this entry point takes device inputs and outputs from the caller and
// keeps all of its own scratch -- re-centred events, sort keys and indices, radix
// histograms, bin boundaries, the sorted events, the device error word and the
// tensor kernel's tile queue -- in
// one file-scope __device__ array of fixed size (about 16 MB, held by every
// device that loads the library until the process exits).  It calls no
// cudaMalloc, cudaFree or other allocating routine.
//
// The array's name is only a host-side stand-in for the device memory, so its
// device address is looked up with cudaGetSymbolAddress on every call made
// outside stream capture (a context reset gives the array a new address); a
// call made during a capture uses the address the last call on that device
// found, so the first call on a device must come before any capture.  Every
// call on a device shares the one array and
// each call overwrites what the previous one left (the error word is cleared at
// the start of every call): calls whose work overlaps on the GPU -- two streams,
// two host threads -- race with each other and must be serialised by the caller.
#include <mutex>

#include "../../include/stkde.h"
#include "internal.cuh"

namespace stkde {
stkde_status check_problem_args(const double* points, int64_t n, const stkde_grid* g, double hs,
                                double ht);
Plan plan_problem(int kernel_constants, int64_t n, const stkde_grid* g, double hs, double ht, int form);
}  // namespace stkde

using namespace stkde;

namespace {

constexpr size_t kMaxEvents = STKDE_STATIC_MAX_EVENTS;
constexpr size_t kMaxBins = STKDE_STATIC_MAX_BINS;  // nkeys + 1 bin boundaries
constexpr size_t kAlign = 256;

constexpr size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
// radix histograms: 256 digits x blocks of 2048 events, plus 256 digit totals
constexpr size_t kHistBytes = (256 * ((kMaxEvents + 2047) / 2048) + 256) * 4;
constexpr size_t kOffEv = 0;
constexpr size_t kOffEvSorted = kOffEv + up(16 * kMaxEvents);
constexpr size_t kOffKeys = kOffEvSorted + up(16 * kMaxEvents);
constexpr size_t kOffIdx = kOffKeys + up(4 * kMaxEvents);
constexpr size_t kOffKeysTmp = kOffIdx + up(4 * kMaxEvents);
constexpr size_t kOffIdxTmp = kOffKeysTmp + up(4 * kMaxEvents);
constexpr size_t kOffHist = kOffIdxTmp + up(4 * kMaxEvents);
constexpr size_t kOffStart = kOffHist + up(kHistBytes);
constexpr size_t kOffErr = kOffStart + up(4 * kMaxBins);
constexpr size_t kScratchBytes = kOffErr + kAlign;

// The scratch.  Host code must not use its name as a device address.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char* g_dev_scratch[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Device address of the scratch on the current device: looked up again outside
// stream capture, the last address found on the device during a capture.
stkde_status scratch_for_device(int dev, bool capture, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return STKDE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!capture) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return STKDE_ERR_CUDA;
        }
        g_dev_scratch[dev] = static_cast<unsigned char*>(p);
    } else if (!g_dev_scratch[dev]) {
        return STKDE_ERR_UNSUPPORTED;  // no call on this device preceded the capture
    }
    *out = g_dev_scratch[dev];
    return STKDE_OK;
}

bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// The tensor tile kernel's form code of an API tensor form.
int static_tc_form(int form) {
    return form == STKDE_FORM_TENSOR_FP16X3 ? 1 : form == STKDE_FORM_TENSOR_TF32X3 ? 2
         : form == STKDE_FORM_TENSOR_TF32X1 ? 3 : 0;
}

bool is_device_pointer(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" stkde_status stkde_compute_static(const double* points, int64_t n,
                                             const stkde_grid* grid, double hs, double ht,
                                             float* out, int form, int kernel_constants,
                                             void* stream, int sync) {
    if (!out) return STKDE_ERR_INVALID_ARGUMENT;
    if (form < STKDE_FORM_TENSOR_BF16X3 || form > STKDE_FORM_TENSOR_TF32X1) return STKDE_ERR_INVALID_ARGUMENT;
    if (kernel_constants != STKDE_KERNEL_PRINTED && kernel_constants != STKDE_KERNEL_UNIT_MASS)
        return STKDE_ERR_INVALID_ARGUMENT;
    stkde_status s = check_problem_args(points, n, grid, hs, ht);
    if (s != STKDE_OK) return s;
    if ((size_t)n > kMaxEvents || radix_sort_temp_bytes((int)n) > kHistBytes)
        return STKDE_ERR_UNSUPPORTED;  // beyond the fixed scratch
    const Plan pl = plan_problem(kernel_constants, n, grid, hs, ht, form);
    if ((size_t)pl.nkeys + 1 > kMaxBins) return STKDE_ERR_UNSUPPORTED;  // too many bins
    if (form == STKDE_FORM_SCATTER && 2.0 * ceil(ht / grid->tres) + 1.0 > 12000.0)
        return STKDE_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return STKDE_ERR_CUDA; }
    if (!is_device_pointer(out, dev)) return STKDE_ERR_INVALID_ARGUMENT;
    if (n > 0 && !is_device_pointer(points, dev)) return STKDE_ERR_INVALID_ARGUMENT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool capture = stream_capturing(st);
    if (capture && sync) return STKDE_ERR_UNSUPPORTED;  // a captured call cannot wait
    unsigned char* base = nullptr;
    s = scratch_for_device(dev, capture, &base);
    if (s != STKDE_OK) return s;

    float4* ev = reinterpret_cast<float4*>(base + kOffEv);
    float4* ev_sorted = reinterpret_cast<float4*>(base + kOffEvSorted);
    uint32_t* keys = reinterpret_cast<uint32_t*>(base + kOffKeys);
    uint32_t* idx = reinterpret_cast<uint32_t*>(base + kOffIdx);
    uint32_t* keys_tmp = reinterpret_cast<uint32_t*>(base + kOffKeysTmp);
    uint32_t* idx_tmp = reinterpret_cast<uint32_t*>(base + kOffIdxTmp);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kOffHist);
    uint32_t* start = reinterpret_cast<uint32_t*>(base + kOffStart);
    int* err = reinterpret_cast<int*>(base + kOffErr);
    int* tile_ctr = reinterpret_cast<int*>(base + kOffErr + 128);
    const size_t grid_bytes = sizeof(float) * (size_t)grid->gx * (size_t)grid->gy * (size_t)grid->gt;

    cudaMemsetAsync(err, 0, sizeof(int), st);  // the previous call's error word
    if (n == 0) {
        cudaMemsetAsync(out, 0, grid_bytes, st);
    } else {
        launch_recentre(points, (int)n, grid->x0, grid->y0, grid->t0, grid->sres, grid->tres, pl,
                        ev, keys, idx, err, st);
        if (form == STKDE_FORM_SCATTER) {
            cudaMemsetAsync(out, 0, grid_bytes, st);
            launch_scatter(pl, ev, out, st);
        } else {
            launch_radix_sort(keys, idx, keys_tmp, idx_tmp, hist, (int)n, pl.key_bits, st);
            launch_bounds_gather(keys, idx, ev, (int)n, pl.nkeys, start, ev_sorted, st);
            Bins b{ev_sorted, start};
            if (form == STKDE_FORM_FP32) {
                if (!launch_tile_fp32(pl, b, out, err, st)) return STKDE_ERR_UNSUPPORTED;
            } else if (!launch_tile_tc(pl, b, out, err, tile_ctr, nullptr, static_tc_form(form), st)) {
                return STKDE_ERR_UNSUPPORTED;
            }
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? STKDE_ERR_OOM : STKDE_ERR_CUDA;
    if (!sync) return STKDE_OK;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return STKDE_ERR_CUDA;
    int h = 0;
    e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return STKDE_ERR_CUDA;
    if (h & ERRBIT_NONFINITE) return STKDE_ERR_NONFINITE;
    if (h & ERRBIT_TIMEOUT) return STKDE_ERR_TIMEOUT;
    if (h & ERRBIT_BOUNDS) return STKDE_ERR_INTERNAL;
    return STKDE_OK;
}
