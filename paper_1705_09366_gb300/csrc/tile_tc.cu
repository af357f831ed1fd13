// K5: tcgen05 tensor-core tile kernel.
//
// PB-SYM (Section 3.2, Algorithm 3) adds, for every event i, the outer product
// of its spatial invariant K_s,i[X][Y] and its temporal invariant K_t,i[T].
// Inside one output tile of 128 voxels in the plane (16 x 8) by up to 256
// voxels of T, the sum over the events that reach the tile is a rank-k
// contraction
//     C[xy][t] = sum_k A[xy][k] * B[k][t],  A = K_s (128 x k),  B = K_t (k x t),
// which runs on the tensor cores: tcgen05.mma, M = 128, K = 16 events per
// instruction, N = the T columns the 16 events' windows cover, the fp32
// accumulator in tensor memory.  For accuracy A and B are split into a 16-bit
// high part and a 16-bit remainder and three products hi*hi + hi*lo + lo*hi are
// accumulated (the dropped lo*lo term is below 2^-16 relative).
//
// The tensor cores round each accumulation step toward zero, so a long run of
// steps into one accumulator drifts low.  The MMA thread therefore closes an
// accumulator "segment" before any 16-column block of it has taken more than
// FLUSH steps; the epilogue stores the first segment of a tile and adds later
// ones to it in fp32 (round to nearest), which bounds the drift per segment.
//
// Persistent CTA per SM, warp-specialised, every hand-off through mbarriers:
//   warp 0      MMA issue (one thread), tensor-memory allocation
//   warp 1      loader: walks the tile's event bins and stages them into shared
//               memory pages with cp.async.bulk (no multicast)
//   warp 2      filter: keeps the events whose cylinder reaches the tile and
//               appends them, in bin order, to a ring of 16-event chunk slots;
//               a tile ends with a partial slot and an end-of-tile slot
//   warps 3-10  generators: chunk slot j is built by generator j mod 8, alone,
//               into its own operand stage: A = K_s and B = K_t as hi and lo
//               16-bit tiles (B in column windows of up to 128)
//   warps 11-14 epilogue: one per tensor-memory lane quarter; scales by
//               1/(n hs^2 ht), writes each voxel of the tile (vector stores),
//               adds later segments, zeroes the accumulator
// Two accumulators of 256 columns let the epilogue of one segment overlap the
// MMAs of the next.  The MMA thread consumes chunk slots in sequence order, so
// every voxel sums its events in the same order on every run (bit-reproducible,
// no global atomics).  The earliest unconsumed chunk can always be produced,
// so no wait can close a cycle.
//
// Every wait on an mbarrier is bounded (2 s of %globaltimer); on expiry the
// kernel sets the timeout bit of the error word, every role leaves its loop,
// outstanding copies and MMAs are drained with a second bounded wait, and the
// tensor memory is freed before the CTA exits.
#include "internal.cuh"
#include "ptx.cuh"
#include "tile_common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace stkde {

namespace {

constexpr int NB = 256;            // T columns per tile = accumulator width
constexpr int NACC = 2;            // accumulators (512 tensor-memory columns)
constexpr int NGEN = 8;            // generator warps
constexpr int NEPI = 4;            // epilogue warps
constexpr int WARP_MMA = 0;
constexpr int WARP_LOAD = 1;
constexpr int WARP_FILT = 2;
constexpr int WARP_GEN0 = 3;
constexpr int WARP_EPI0 = WARP_GEN0 + NGEN;
constexpr int NTHREADS = (WARP_EPI0 + NEPI) * 32;
constexpr int PAGE = 256;          // events per staging page
constexpr int NPAGES = 4;
constexpr int CHUNK = 16;          // events per MMA (K of kind::f16)
constexpr int RSLOTS = 32;         // chunk slots in the kept-event ring
constexpr int NCAP = 128;          // T columns per operand stage (one column window)
constexpr int TAB_ROW = 144;       // bytes per factor-table row (16 float2 + pad: no bank conflicts)
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr uint64_t DRAIN_NS = 200000000ull;
constexpr uint32_t A_BYTES = TILE_XY * CHUNK * 2;   // 4 KB
constexpr uint32_t B_BYTES = NCAP * CHUNK * 2;      // 4 KB
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr uint32_t TAB_BYTES = 3584;                // x table, y table, t values
constexpr uint32_t CORE_LBO = 128;  // next core matrix along K
constexpr uint32_t CORE_SBO = 256;  // next core matrix along M / N

// slot and stage header flags
constexpr int F_CHUNK = 1, F_MORE = 2, F_END = 4, F_TERM = 8;

struct L {
    static constexpr uint32_t OFF_STAGE = 0;
    static constexpr uint32_t OFF_PAGES = OFF_STAGE + NGEN * STAGE_BYTES;
    static constexpr uint32_t OFF_RING = OFF_PAGES + NPAGES * PAGE * 16;
    static constexpr uint32_t OFF_RHDR = OFF_RING + RSLOTS * CHUNK * 16;
    static constexpr uint32_t OFF_TAB = OFF_RHDR + RSLOTS * 16;
    static constexpr uint32_t OFF_SHDR = OFF_TAB + NGEN * TAB_BYTES;
    static constexpr uint32_t OFF_PMETA = OFF_SHDR + NGEN * 16;
    static constexpr uint32_t OFF_DESC = OFF_PMETA + NPAGES * 16;
    static constexpr uint32_t OFF_BAR = OFF_DESC + NACC * 16;
    static constexpr int NBARS = 2 * NPAGES + 2 * RSLOTS + 2 * NGEN + 3 * NACC + 1;
    static constexpr uint32_t OFF_MISC = OFF_BAR + NBARS * 8;
    static constexpr uint32_t TOTAL = OFF_MISC + 16;
    __host__ __device__ static constexpr int pfull(int p) { return p; }
    __host__ __device__ static constexpr int pempty(int p) { return NPAGES + p; }
    __host__ __device__ static constexpr int cfull(int s) { return 2 * NPAGES + s; }
    __host__ __device__ static constexpr int cempty(int s) { return 2 * NPAGES + RSLOTS + s; }
    __host__ __device__ static constexpr int sfull(int g) { return 2 * NPAGES + 2 * RSLOTS + g; }
    __host__ __device__ static constexpr int sempty(int g) { return 2 * NPAGES + 2 * RSLOTS + NGEN + g; }
    __host__ __device__ static constexpr int afull(int b) { return 2 * NPAGES + 2 * RSLOTS + 2 * NGEN + b; }
    __host__ __device__ static constexpr int aempty(int b) { return 2 * NPAGES + 2 * RSLOTS + 2 * NGEN + NACC + b; }
    __host__ __device__ static constexpr int dfull(int b) { return 2 * NPAGES + 2 * RSLOTS + 2 * NGEN + 2 * NACC + b; }
    __host__ __device__ static constexpr int drain() { return 2 * NPAGES + 2 * RSLOTS + 2 * NGEN + 3 * NACC; }
    static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
    static_assert(TOTAL <= 227 * 1024, "shared memory budget");
    static_assert(TAB_BYTES >= (TX + TY) * TAB_ROW + CHUNK * 4, "table size");
};

// hi + lo split of two values into packed 16-bit pairs (low half = first value).
template <bool FP16>
__device__ __forceinline__ void split2(float a0, float a1, uint32_t& hi, uint32_t& lo) {
    if constexpr (FP16) {
        const __half2 h = __floats2half2_rn(a0, a1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a0 - hf.x, a1 - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a0 - hf.x, a1 - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

struct Ctl {
    volatile int* abort;
    int* err;
};

// Bounded wait for the phase of parity `parity` of barrier `bar`.  Returns
// false (and raises the abort flag) after WAIT_NS, or as soon as another role
// has aborted.
__device__ __forceinline__ bool wait_bar(const Ctl& c, uint32_t bar, uint32_t parity) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = ptx::globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*c.abort) return false;
            if (ptx::globaltimer() - t0 > WAIT_NS) {
                *c.abort = 1;
                atomicOr(c.err, ERRBIT_TIMEOUT);
                return false;
            }
        }
    }
}

// The same for a whole warp: the warp proceeds only if all lanes saw the
// phase complete, so a timeout never splits the warp.
__device__ __forceinline__ bool wait_warp(const Ctl& c, uint32_t bar, uint32_t parity) {
    const bool r = wait_bar(c, bar, parity);
    return __all_sync(0xffffffffu, r);
}

// Bounded wait used while draining after an abort (ignores the abort flag).
__device__ __forceinline__ void drain_bar(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(bar, parity))
        if (ptx::globaltimer() - t0 > DRAIN_NS) break;
}

__device__ __forceinline__ void decode_item(const Plan& pl, int64_t item, int& tx, int& ty,
                                            int& tb) {
    ty = (int)(item % pl.nty);
    tx = (int)((item / pl.nty) % pl.ntx);
    tb = (int)(item / ((int64_t)pl.nty * pl.ntx));
}

template <bool FP16>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tile_tc(Plan pl, const float4* __restrict__ ev, const uint32_t* __restrict__ start,
          float* __restrict__ out, int* __restrict__ err, int64_t nitems, int flush_steps) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t sb = ptx::smem_addr(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ctl c{reinterpret_cast<volatile int*>(smem + L::OFF_MISC + 4), err};
    auto bar = [sb](int i) -> uint32_t { return sb + L::OFF_BAR + 8u * (uint32_t)i; };

    if (threadIdx.x == 0) {
        for (int p = 0; p < NPAGES; ++p) {
            ptx::mbar_init(bar(L::pfull(p)), 1);
            ptx::mbar_init(bar(L::pempty(p)), 1);
        }
        for (int s = 0; s < RSLOTS; ++s) {
            ptx::mbar_init(bar(L::cfull(s)), 1);
            ptx::mbar_init(bar(L::cempty(s)), 1);
        }
        for (int g = 0; g < NGEN; ++g) {
            ptx::mbar_init(bar(L::sfull(g)), 1);
            ptx::mbar_init(bar(L::sempty(g)), 1);
        }
        for (int b = 0; b < NACC; ++b) {
            ptx::mbar_init(bar(L::afull(b)), 1);
            ptx::mbar_init(bar(L::aempty(b)), NEPI);
            ptx::mbar_init(bar(L::dfull(b)), 1);
        }
        ptx::mbar_init(bar(L::drain()), 1);
        *c.abort = 0;
        ptx::fence_mbar_init();
    }
    if (warp == WARP_MMA) {
        ptx::tmem_alloc(sb + L::OFF_MISC, NB * NACC);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + L::OFF_MISC);

    if (warp == WARP_LOAD) {
        // ------------------------------------------------------------ loader
        uint32_t pg = 0, fill = 0;
        bool open = false, ok = true;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            int tx, ty, tb;
            decode_item(pl, item, tx, ty, tb);
            const TileGeom g = tile_geom(pl, tx, ty, tb, NB);
            const int ncx = g.cx_hi - g.cx_lo + 1;
            const int nr = (g.s_hi >= g.s_lo && ncx > 0) ? (g.s_hi - g.s_lo + 1) * ncx : 0;
            for (int r0 = 0; r0 <= nr && ok; r0 += 32) {
                uint32_t a = 0, b = 0;
                const int r = r0 + lane;
                if (r < nr) {
                    const int s = g.s_lo + r / ncx, cx = g.cx_lo + r % ncx;
                    const uint32_t kb =
                        ((uint32_t)s * (uint32_t)pl.ntx + (uint32_t)cx) * (uint32_t)pl.nty;
                    a = start[kb + g.cy_lo];
                    b = start[kb + g.cy_hi + 1];
                }
                const int nj = min(32, nr - r0);
                // nj <= 0 on the final pass: it only closes the tile's last page
                for (int j = 0; j <= nj && ok; ++j) {
                    uint32_t aj = 0, bj = 0;
                    if (j < nj) {
                        aj = __shfl_sync(0xffffffffu, a, j);
                        bj = __shfl_sync(0xffffffffu, b, j);
                    } else if (r0 + 32 <= nr) {
                        break;  // not the final pass
                    }
                    const bool last = (j == nj) && (r0 + 32 > nr);
                    while (aj < bj || last) {
                        if (!open) {
                            const uint32_t p = pg % NPAGES;
                            if (!(ok = wait_warp(c, bar(L::pempty(p)), ((pg / NPAGES) & 1u) ^ 1u))) break;
                            open = true;
                            fill = 0;
                        }
                        const uint32_t p = pg % NPAGES;
                        const uint32_t take = min(bj - aj, (uint32_t)PAGE - fill);
                        if (take > 0 && lane == 0) {
                            ptx::mbar_expect_tx(bar(L::pfull(p)), take * 16u);
                            ptx::bulk_g2s(sb + L::OFF_PAGES + (p * PAGE + fill) * 16u, ev + aj,
                                          take * 16u, bar(L::pfull(p)));
                        }
                        fill += take;
                        aj += take;
                        if (fill == (uint32_t)PAGE || (last && aj >= bj)) {
                            if (lane == 0) {
                                ptx::sts_i4(sb + L::OFF_PMETA + p * 16,
                                            make_int4((int)fill, last && aj >= bj ? 1 : 0, 0, 0));
                                ptx::mbar_arrive(bar(L::pfull(p)));
                            }
                            __syncwarp();
                            ++pg;
                            open = false;
                            if (last && aj >= bj) break;
                        }
                    }
                }
            }
        }
        if (!ok) {
            if (open) {
                if (lane == 0) {
                    const uint32_t p = pg % NPAGES;
                    ptx::sts_i4(sb + L::OFF_PMETA + p * 16, make_int4((int)fill, 1, 0, 0));
                    ptx::mbar_arrive(bar(L::pfull(p)));
                }
                ++pg;
            }
            for (uint32_t q = (pg > NPAGES ? pg - NPAGES : 0); q < pg; ++q)
                drain_bar(bar(L::pfull(q % NPAGES)), (q / NPAGES) & 1u);
        }
    } else if (warp == WARP_FILT) {
        // ------------------------------------------------------------ filter
        uint32_t pg = 0, kabs = 0, acq = 0, pub = 0;
        bool ok = true;
        const uint32_t lt = (1u << lane) - 1u;
        // makes ring slots [acq, upto] writable
        auto acquire = [&](uint32_t upto) -> bool {
            while (acq <= upto) {
                if (!wait_warp(c, bar(L::cempty(acq % RSLOTS)), ((acq / RSLOTS) & 1u) ^ 1u))
                    return false;
                ++acq;
            }
            return true;
        };
        // publishes slot `pub` with `count` events
        auto publish = [&](int count, int flags, int64_t item) {
            __syncwarp();
            if (lane == 0) {
                const uint32_t s = pub % RSLOTS;
                ptx::sts_i4(sb + L::OFF_RHDR + s * 16,
                            make_int4(count, flags, (int)(item & 0xffffffff), (int)(item >> 32)));
                ptx::mbar_arrive(bar(L::cfull(s)));
            }
            __syncwarp();
            ++pub;
        };
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            int tx, ty, tb;
            decode_item(pl, item, tx, ty, tb);
            const TileGeom g = tile_geom(pl, tx, ty, tb, NB);
            bool end = false;
            while (!end && ok) {
                const uint32_t p = pg % NPAGES;
                if (!(ok = wait_warp(c, bar(L::pfull(p)), (pg / NPAGES) & 1u))) break;
                const int4 meta = ptx::lds_i4(sb + L::OFF_PMETA + p * 16);
                end = meta.y != 0;
                for (int r = 0; r * 32 < meta.x && ok; ++r) {
                    const int slot = r * 32 + lane;
                    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
                    bool keep = false;
                    if (slot < meta.x) {
                        e = ptx::lds_f4(sb + L::OFF_PAGES + (p * PAGE + slot) * 16u);
                        keep = reaches(pl, g, e);
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                    const uint32_t nk = __popc(bal);
                    if (nk == 0) continue;
                    if (!(ok = acquire((kabs + nk - 1) / CHUNK))) break;
                    if (keep) {
                        const uint32_t pos = (kabs + __popc(bal & lt)) % (RSLOTS * CHUNK);
                        ptx::sts_f4(sb + L::OFF_RING + pos * 16, e);
                    }
                    kabs += nk;
                    while (pub < kabs / CHUNK) publish(CHUNK, F_CHUNK, item);
                }
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(bar(L::pempty(p)));
                ++pg;
            }
            if (!ok) break;
            if (kabs % CHUNK) {  // the tile's last, partial chunk
                publish((int)(kabs % CHUNK), F_CHUNK, item);
                kabs = pub * CHUNK;
            }
            if (!(ok = acquire(pub))) break;  // end-of-tile slot
            publish(0, F_END, item);
            kabs = pub * CHUNK;
        }
        // one termination slot per generator
        for (int gq = 0; gq < NGEN && ok; ++gq) {
            if (!(ok = acquire(pub))) break;
            publish(0, F_TERM, 0);
        }
    } else if (warp >= WARP_GEN0 && warp < WARP_EPI0) {
        // -------------------------------------------------------- generators
        const int gw = warp - WARP_GEN0;
        const uint32_t tab = sb + L::OFF_TAB + gw * TAB_BYTES;
        const uint32_t tabx = tab, taby = tab + TX * TAB_ROW, tt = tab + (TX + TY) * TAB_ROW;
        const uint32_t stg = sb + L::OFF_STAGE + gw * STAGE_BYTES;
        const uint32_t a_hi = stg, a_lo = stg + A_BYTES, b_hi = stg + 2 * A_BYTES,
                       b_lo = b_hi + B_BYTES;
        const uint32_t shdr = sb + L::OFF_SHDR + gw * 16;
        const float csct = pl.cs * pl.ct;
        uint32_t suse = 0;  // uses of this warp's stage
        bool ok = true;
        for (uint32_t j = (uint32_t)gw; ok; j += NGEN) {
            const uint32_t s = j % RSLOTS;
            if (!(ok = wait_warp(c, bar(L::cfull(s)), (j / RSLOTS) & 1u))) break;
            const int4 h = ptx::lds_i4(sb + L::OFF_RHDR + s * 16);
            const int count = h.x;
            float4 e = make_float4(1.0e30f, 1.0e30f, 1.0e30f, 0.f);
            if (lane < count) e = ptx::lds_f4(sb + L::OFF_RING + (s * CHUNK + lane) * 16u);
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(bar(L::cempty(s)));
            if (h.y & F_TERM) break;
            if (h.y & F_END) {  // forward the end of the tile to the MMA thread
                if (!(ok = wait_warp(c, bar(L::sempty(gw)), (suse & 1u) ^ 1u))) break;
                if (lane == 0) {
                    ptx::sts_i4(shdr, make_int4(0, 0, F_END, 0));
                    ptx::mbar_arrive(bar(L::sfull(gw)));
                }
                __syncwarp();
                ++suse;
                continue;
            }
            const int64_t item = (int64_t)(uint32_t)h.z | ((int64_t)h.w << 32);
            int tx, ty, tb;
            decode_item(pl, item, tx, ty, tb);
            const int X0 = tx * TX, Y0 = ty * TY, T0 = tb * NB;
            const int nbv = min(NB, pl.gt - T0);

            // columns the events' T windows cover, clipped into the block (the
            // filter's margin can keep an event whose window misses the block;
            // its K_t values are zero anyway)
            int lo = 0x7fffffff, hi = -1;
            if (lane < count) {
                lo = min(max((int)ceilf(e.z - 0.5f - pl.htv) - T0, 0), nbv - 1);
                hi = min(max((int)floorf(e.z - 0.5f + pl.htv) - T0, lo), nbv - 1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            const int c0 = lo & ~15;
            const int cend = ((hi + 1) + 15) & ~15;  // exclusive, <= roundup16(nbv) <= NB

            // factor tables of K_s: (u^2, 1-u^2) per x and (v^2, 1-v^2) per y
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = i * 32 + lane, x = q >> 4, k = q & 15;
                const float ex = __shfl_sync(0xffffffffu, e.x, k);
                const float du = ((float)(X0 + x) + 0.5f - ex) * pl.inv_hs;
                const float u2 = du * du;
                ptx::sts_f2(tabx + x * TAB_ROW + k * 8, make_float2(u2, 1.0f - u2));
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int q = i * 32 + lane, y = q >> 4, k = q & 15;
                const float ey = __shfl_sync(0xffffffffu, e.y, k);
                const float dv = ((float)(Y0 + y) + 0.5f - ey) * pl.inv_hs;
                const float v2 = dv * dv;
                ptx::sts_f2(taby + y * TAB_ROW + k * 8, make_float2(v2, 1.0f - v2));
            }
            if (lane < CHUNK) ptx::sts_f(tt + lane * 4, e.z);
            __syncwarp();

            if (!(ok = wait_warp(c, bar(L::sempty(gw)), (suse & 1u) ^ 1u))) break;
            // A = K_s without c_s: row r = voxel (x = r / 8, y = r % 8); lane owns
            // rows lane + 32 j, all with y = lane % 8
#pragma unroll
            for (int kg = 0; kg < 2; ++kg) {
                float4 fy[4];
#pragma unroll
                for (int kp = 0; kp < 4; ++kp)
                    fy[kp] = ptx::lds_f4(taby + (lane & 7) * TAB_ROW + (kg * 8 + 2 * kp) * 8);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int r = lane + 32 * jj;
                    uint32_t ah[4], al[4];
#pragma unroll
                    for (int kp = 0; kp < 4; ++kp) {
                        const float4 fx = ptx::lds_f4(tabx + (r >> 3) * TAB_ROW + (kg * 8 + 2 * kp) * 8);
                        const float a0 = (fx.x + fy[kp].x < 1.0f) ? fx.y * fy[kp].y : 0.0f;
                        const float a1 = (fx.z + fy[kp].z < 1.0f) ? fx.w * fy[kp].w : 0.0f;
                        split2<FP16>(a0, a1, ah[kp], al[kp]);
                    }
                    const uint32_t off = (uint32_t)(r >> 3) * CORE_SBO + kg * CORE_LBO + (r & 7) * 16;
                    ptx::sts_u4(a_hi + off, ah[0], ah[1], ah[2], ah[3]);
                    ptx::sts_u4(a_lo + off, al[0], al[1], al[2], al[3]);
                }
            }
            // B = c_s c_t (1 - w^2)_+ in column windows of up to NCAP
            float tk[CHUNK];
#pragma unroll
            for (int k4 = 0; k4 < CHUNK / 4; ++k4) {
                const float4 t4 = ptx::lds_f4(tt + k4 * 16);
                tk[4 * k4] = t4.x; tk[4 * k4 + 1] = t4.y; tk[4 * k4 + 2] = t4.z; tk[4 * k4 + 3] = t4.w;
            }
            for (int cw = c0; cw < cend && ok; cw += NCAP) {
                if (cw != c0 && !(ok = wait_warp(c, bar(L::sempty(gw)), (suse & 1u) ^ 1u))) break;
                const int ncols = min(NCAP, cend - cw);
                for (int n = lane; n < ncols; n += 32) {
                    const float tc = (float)(T0 + cw + n) + 0.5f;
#pragma unroll
                    for (int kg = 0; kg < 2; ++kg) {
                        uint32_t bh[4], bl[4];
#pragma unroll
                        for (int kp = 0; kp < 4; ++kp) {
                            const float w0 = (tc - tk[kg * 8 + 2 * kp]) * pl.inv_ht;
                            const float w1 = (tc - tk[kg * 8 + 2 * kp + 1]) * pl.inv_ht;
                            const float b0 = csct * fmaxf(fmaf(-w0, w0, 1.0f), 0.0f);
                            const float b1 = csct * fmaxf(fmaf(-w1, w1, 1.0f), 0.0f);
                            split2<FP16>(b0, b1, bh[kp], bl[kp]);
                        }
                        const uint32_t off = (uint32_t)(n >> 3) * CORE_SBO + kg * CORE_LBO + (n & 7) * 16;
                        ptx::sts_u4(b_hi + off, bh[0], bh[1], bh[2], bh[3]);
                        ptx::sts_u4(b_lo + off, bl[0], bl[1], bl[2], bl[3]);
                    }
                }
                const int more = (cw + NCAP < cend) ? F_MORE : 0;
                if (lane == 0) ptx::sts_i4(shdr, make_int4(cw, ncols, F_CHUNK | more, 0));
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(bar(L::sfull(gw)));
                ++suse;
            }
        }
    } else if (warp == WARP_MMA) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            uint32_t par = 0;  // bit g: parity of the next use of generator g's stage
            uint32_t seg = 0;  // accumulator segments opened so far
            uint32_t jm = 0;   // next chunk slot
            bool ok = true;
            const uint32_t fmt = FP16 ? 0u : 1u;
            for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                int b = (int)(seg & 1u);
                if (!(ok = wait_bar(c, bar(L::aempty(b)), (seg >> 1) & 1u))) break;
                ptx::tc_fence_after();
                int first = 1;
                uint32_t touched = 0;            // 32-column blocks written in this segment
                uint16_t steps[NB / 16];         // accumulation steps per 16-column block
#pragma unroll
                for (int q = 0; q < NB / 16; ++q) steps[q] = 0;
                bool done = false;
                while (!done && ok) {
                    const int gq = (int)(jm % NGEN);
                    bool more = true;
                    while (more && ok) {
                        if (!(ok = wait_bar(c, bar(L::sfull(gq)), (par >> gq) & 1u))) break;
                        par ^= 1u << gq;
                        ptx::tc_fence_after();
                        const int4 h = ptx::lds_i4(sb + L::OFF_SHDR + gq * 16);
                        more = (h.z & F_MORE) != 0;
                        if (h.z & F_END) {
                            ptx::mbar_arrive(bar(L::sempty(gq)));
                            done = true;
                            break;
                        }
                        const bool in_range = h.x >= 0 && h.y >= 16 && h.y <= NCAP &&
                                              (h.y & 15) == 0 && h.x + h.y <= NB && (h.x & 15) == 0;
                        if (!in_range) {  // never issue an MMA outside the accumulator
                            atomicOr(err, ERRBIT_BOUNDS);
                            ptx::mbar_arrive(bar(L::sempty(gq)));
                            continue;
                        }
                        const int blo = h.x >> 4, bhi = (h.x + h.y) >> 4;
                        bool full = false;
#pragma unroll
                        for (int q = 0; q < NB / 16; ++q)
                            if (q >= blo && q < bhi && steps[q] + 3 > flush_steps) full = true;
                        if (full) {
                            // close the segment: the epilogue adds it in fp32
                            ptx::sts_i4(sb + L::OFF_DESC + b * 16,
                                        make_int4((int)(item & 0xffffffff), (int)(item >> 32), first, (int)touched));
                            ptx::mbar_arrive(bar(L::dfull(b)));
                            ptx::tc_commit(bar(L::afull(b)));
                            ++seg;
                            b = (int)(seg & 1u);
                            if (!(ok = wait_bar(c, bar(L::aempty(b)), (seg >> 1) & 1u))) break;
                            ptx::tc_fence_after();
                            first = 0;
                            touched = 0;
#pragma unroll
                            for (int q = 0; q < NB / 16; ++q) steps[q] = 0;
                        }
#pragma unroll
                        for (int q = 0; q < NB / 16; ++q)
                            if (q >= blo && q < bhi) steps[q] += 3;
                        for (int q = h.x >> 5; q <= (h.x + h.y - 1) >> 5; ++q) touched |= 1u << q;
                        const uint32_t st = sb + L::OFF_STAGE + (uint32_t)gq * STAGE_BYTES;
                        const uint64_t ahi = ptx::smem_desc(st, CORE_LBO, CORE_SBO);
                        const uint64_t alo = ptx::smem_desc(st + A_BYTES, CORE_LBO, CORE_SBO);
                        const uint64_t bhi_d = ptx::smem_desc(st + 2 * A_BYTES, CORE_LBO, CORE_SBO);
                        const uint64_t blo_d = ptx::smem_desc(st + 2 * A_BYTES + B_BYTES, CORE_LBO, CORE_SBO);
                        const uint32_t idesc = ptx::idesc_f16(128, (uint32_t)h.y, fmt);
                        const uint32_t d = tmem + (uint32_t)(b * NB + h.x);
                        ptx::mma_f16_ss(d, ahi, bhi_d, idesc, 1);
                        ptx::mma_f16_ss(d, ahi, blo_d, idesc, 1);
                        ptx::mma_f16_ss(d, alo, bhi_d, idesc, 1);
                        ptx::tc_commit(bar(L::sempty(gq)));
                    }
                    ++jm;
                }
                if (!ok) break;
                ptx::sts_i4(sb + L::OFF_DESC + b * 16,
                            make_int4((int)(item & 0xffffffff), (int)(item >> 32), first | 2, (int)touched));
                ptx::mbar_arrive(bar(L::dfull(b)));
                ptx::tc_commit(bar(L::afull(b)));
                ++seg;
            }
            // every MMA issued has completed before the accumulator is released
            ptx::tc_commit(bar(L::drain()));
            drain_bar(bar(L::drain()), 0);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        for (int col = 0; col < NB * NACC; col += 32) ptx::tmem_st32_zero(trow + (uint32_t)col);
        ptx::tmem_wait_st();
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0)
            for (int b = 0; b < NACC; ++b) ptx::mbar_arrive(bar(L::aempty(b)));
        bool ok = true;
        uint32_t seg = 0;
        const bool vec = (pl.gt & 3) == 0;
        while (ok) {
            const int b = (int)(seg & 1u);
            const uint32_t par = (seg >> 1) & 1u;
            // the item of this segment is in its descriptor; stop after the CTA's last item
            if (!(ok = wait_warp(c, bar(L::dfull(b)), par))) break;
            if (!(ok = wait_warp(c, bar(L::afull(b)), par))) break;
            ptx::tc_fence_after();
            const int4 dsc = ptx::lds_i4(sb + L::OFF_DESC + b * 16);
            const int64_t item = (int64_t)(uint32_t)dsc.x | ((int64_t)dsc.y << 32);
            const bool first = (dsc.z & 1) != 0, last = (dsc.z & 2) != 0;
            const uint32_t touched = (uint32_t)dsc.w;
            int tx, ty, tb;
            decode_item(pl, item, tx, ty, tb);
            const int m = 32 * q + lane;
            const int X = tx * TX + m / TY, Y = ty * TY + m % TY, T0 = tb * NB;
            const int nbv = min(NB, pl.gt - T0);
            const bool valid = X < pl.gx && Y < pl.gy;
            float* dst = out + ((int64_t)X * pl.gy + Y) * (int64_t)pl.gt + T0;
            for (int col = 0; col < nbv; col += 32) {
                const bool hit = (touched >> (col >> 5)) & 1u;
                if (!first && !hit) continue;
                uint32_t r[32];
                const uint32_t ta = trow + (uint32_t)(b * NB + col);
                ptx::tmem_ld32(ta, r);
                ptx::tmem_wait_ld();
                if (hit) ptx::tmem_st32_zero(ta);
                if (!valid) continue;
                const int nv = min(32, nbv - col);
                if (vec && nv == 32) {
#pragma unroll
                    for (int v4 = 0; v4 < 8; ++v4) {
                        float4 o = make_float4(__uint_as_float(r[4 * v4]) * pl.norm,
                                               __uint_as_float(r[4 * v4 + 1]) * pl.norm,
                                               __uint_as_float(r[4 * v4 + 2]) * pl.norm,
                                               __uint_as_float(r[4 * v4 + 3]) * pl.norm);
                        float4* p4 = reinterpret_cast<float4*>(dst + col) + v4;
                        if (!first) {
                            const float4 pv = *p4;
                            o.x += pv.x; o.y += pv.y; o.z += pv.z; o.w += pv.w;
                        }
                        if (last) __stcs(p4, o); else *p4 = o;
                    }
                } else {
#pragma unroll
                    for (int jx = 0; jx < 32; ++jx) {
                        if (jx < nv) {
                            float o = __uint_as_float(r[jx]) * pl.norm;
                            if (!first) o += dst[col + jx];
                            dst[col + jx] = o;
                        }
                    }
                }
            }
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(bar(L::aempty(b)));
            ++seg;
            if (last && item + gridDim.x >= nitems) break;
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == WARP_MMA) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, NB * NACC);
    }
}

template <bool FP16>
bool launch_cfg(const Plan& pl, const Bins& b, float* out, int* err, cudaStream_t st) {
    auto kern = k_tile_tc<FP16>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::TOTAL) !=
            cudaSuccess)
            return false;
        attr = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntb = (pl.gt + NB - 1) / NB;
    const int64_t items = (int64_t)pl.ntx * pl.nty * ntb;
    if (items <= 0) return true;
    const int grid = (int)(items < sms ? items : sms);
    // accumulation steps per 16-column block before a segment is closed: bounds
    // the round-toward-zero drift of the tensor-core accumulation per segment
    const int flush_steps = FP16 ? 192 : 384;
    kern<<<grid, NTHREADS, L::TOTAL, st>>>(pl, b.ev, b.start, out, err, items, flush_steps);
    return true;
}

}  // namespace

bool launch_tile_tc(const Plan& pl, const Bins& b, float* out, int* err, int fp16,
                    cudaStream_t st) {
    return fp16 ? launch_cfg<true>(pl, b, out, err, st) : launch_cfg<false>(pl, b, out, err, st);
}

}  // namespace stkde
