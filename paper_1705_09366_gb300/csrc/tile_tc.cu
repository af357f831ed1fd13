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
// accumulator "segment" before any 32-column block of it has taken more than a
// fixed number of chunks; the epilogue stores the first segment of a tile and
// adds later ones to it in fp32 (round to nearest), which bounds the drift.
//
// Persistent CTA per SM, warp-specialised, every hand-off through mbarriers
// (warp w runs on scheduler w % 4; the MMA thread shares its scheduler only
// with the light loader and one epilogue warp):
//   warp 0            MMA issue (one thread), tensor-memory allocation
//   warp 4            loader: walks the tile's event bins and stages them, in
//                     bin order, into 256-event shared-memory pages with
//                     cp.async.bulk (no multicast), one copy per bin run, all
//                     lanes issuing in parallel
//   warps 1-3,5-7,9,10  generators: every generator reads every page; the
//                     page's owner (page q: generator q mod 8) keeps the events
//                     whose cylinder reaches the tile, compacting the page in
//                     place, and chunk c of the page -- kept events 16c..16c+15
//                     -- is built by generator (q + c) mod 8 in its own operand
//                     stage: A = K_s and B = K_t as hi and lo 16-bit tiles (B in
//                     column windows of up to 128)
//   warps 12-15       epilogue: one per tensor-memory lane quarter; scales by
//                     1/(n hs^2 ht), writes each voxel of the tile (vector
//                     stores), adds later segments, zeroes the accumulator
// Two accumulators of 256 columns let the epilogue of one segment overlap the
// MMAs of the next.  The MMA thread consumes pages, and the chunks of a page, in
// order, so every voxel sums its events in the same order on every run
// (bit-reproducible, no global atomics).  The generator of the earliest
// unconsumed chunk can always build it, so no wait can close a cycle.
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
constexpr int WARP_LOAD = 4;
constexpr int WARP_EPI0 = 12;
constexpr int NTHREADS = 16 * 32;
constexpr int PAGE = 256;          // events per staging page
constexpr int NPAGES = 12;
constexpr int CHUNK = 16;          // events per MMA (K of kind::f16)
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

// page and stage header flags
constexpr int F_MMA = 1;        // stage holds operands for the MMA
constexpr int F_PAGE_END = 2;   // last stage of a page
constexpr int F_ITEM_END = 4;   // last page / stage of a tile
constexpr int F_TERM = 8;       // page: no more tiles
constexpr int F_MORE = 16;      // stage: another column window of the same chunk follows

// generator index of a warp (-1: not a generator)
__device__ __forceinline__ int gen_index(int warp) {
    return (warp >= 1 && warp <= 3) ? warp - 1 : (warp >= 5 && warp <= 7) ? warp - 2
         : (warp == 9 || warp == 10) ? warp - 3 : -1;
}

struct L {
    static constexpr uint32_t OFF_STAGE = 0;
    static constexpr uint32_t OFF_PAGES = OFF_STAGE + NGEN * STAGE_BYTES;
    static constexpr uint32_t OFF_TAB = OFF_PAGES + NPAGES * PAGE * 16;
    static constexpr uint32_t OFF_SHDR = OFF_TAB + NGEN * TAB_BYTES;
    static constexpr uint32_t OFF_PMETA = OFF_SHDR + NGEN * 32;
    static constexpr uint32_t OFF_KEPT = OFF_PMETA + NPAGES * 16;
    static constexpr uint32_t OFF_DESC = OFF_KEPT + NPAGES * 16;
    static constexpr uint32_t OFF_BAR = OFF_DESC + NACC * 16;
    static constexpr int NBARS = 3 * NPAGES + 2 * NGEN + 3 * NACC + 1;
    static constexpr uint32_t OFF_MISC = OFF_BAR + NBARS * 8;
    static constexpr uint32_t TOTAL = OFF_MISC + 16;
    __host__ __device__ static constexpr int pfull(int p) { return p; }
    __host__ __device__ static constexpr int pempty(int p) { return NPAGES + p; }
    __host__ __device__ static constexpr int pfilt(int p) { return 2 * NPAGES + p; }
    __host__ __device__ static constexpr int sfull(int g) { return 3 * NPAGES + g; }
    __host__ __device__ static constexpr int sempty(int g) { return 3 * NPAGES + NGEN + g; }
    __host__ __device__ static constexpr int afull(int b) { return 3 * NPAGES + 2 * NGEN + b; }
    __host__ __device__ static constexpr int aempty(int b) { return 3 * NPAGES + 2 * NGEN + NACC + b; }
    __host__ __device__ static constexpr int dfull(int b) { return 3 * NPAGES + 2 * NGEN + 2 * NACC + b; }
    __host__ __device__ static constexpr int drain() { return 3 * NPAGES + 2 * NGEN + 3 * NACC; }
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
          float* __restrict__ out, int* __restrict__ err, int64_t nitems, int flush_chunks) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t sb = ptx::smem_addr(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ctl c{reinterpret_cast<volatile int*>(smem + L::OFF_MISC + 4), err};
    auto bar = [sb](int i) -> uint32_t { return sb + L::OFF_BAR + 8u * (uint32_t)i; };

    if (threadIdx.x == 0) {
        for (int p = 0; p < NPAGES; ++p) {
            ptx::mbar_init(bar(L::pfull(p)), 1);
            ptx::mbar_init(bar(L::pempty(p)), NGEN);
            ptx::mbar_init(bar(L::pfilt(p)), 1);
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
    const int gi = gen_index(warp);

    if (warp == WARP_LOAD) {
        // ------------------------------------------------------------ loader
        uint32_t pg = 0, fill = 0;
        bool open = false, ok = true;
        auto open_page = [&]() -> bool {
            if (!wait_warp(c, bar(L::pempty(pg % NPAGES)), ((pg / NPAGES) & 1u) ^ 1u)) return false;
            open = true;
            fill = 0;
            return true;
        };
        auto close_page = [&](int flags, int64_t item) {
            __syncwarp();
            if (lane == 0) {
                const uint32_t p = pg % NPAGES;
                ptx::sts_i4(sb + L::OFF_PMETA + p * 16,
                            make_int4((int)fill, flags, (int)(item & 0xffffffff), (int)(item >> 32)));
                ptx::mbar_arrive(bar(L::pfull(p)));
            }
            __syncwarp();
            ++pg;
            open = false;
        };
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            int tx, ty, tb;
            decode_item(pl, item, tx, ty, tb);
            const TileGeom g = tile_geom(pl, tx, ty, tb, NB);
            const int ncx = g.cx_hi - g.cx_lo + 1;
            const int nr = (g.s_hi >= g.s_lo && ncx > 0) ? (g.s_hi - g.s_lo + 1) * ncx : 0;
            for (int r0 = 0; r0 < nr && ok; r0 += 32) {
                // 32 bin runs at a time: lane-parallel lengths, offsets by a warp scan
                uint32_t a = 0, len = 0;
                const int r = r0 + lane;
                if (r < nr) {
                    const int s = g.s_lo + r / ncx, cx = g.cx_lo + r % ncx;
                    const uint32_t kb =
                        ((uint32_t)s * (uint32_t)pl.ntx + (uint32_t)cx) * (uint32_t)pl.nty;
                    a = start[kb + g.cy_lo];
                    len = start[kb + g.cy_hi + 1] - a;
                }
                uint32_t incl = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const uint32_t off = incl - len, tot = __shfl_sync(0xffffffffu, incl, 31);
                uint32_t done = 0;
                while (done < tot) {
                    if (!open && !(ok = open_page())) break;
                    const uint32_t p = pg % NPAGES;
                    const uint32_t take = min((uint32_t)PAGE - fill, tot - done);
                    // this page takes pass positions [done, done + take); each lane copies
                    // the part of its own run that falls there
                    const uint32_t lo = max(off, done), hi = min(off + len, done + take);
                    if (hi > lo) {
                        ptx::mbar_expect_tx(bar(L::pfull(p)), (hi - lo) * 16u);
                        ptx::bulk_g2s(sb + L::OFF_PAGES + (p * PAGE + fill + (lo - done)) * 16u,
                                      ev + a + (lo - off), (hi - lo) * 16u, bar(L::pfull(p)));
                    }
                    fill += take;
                    done += take;
                    if (fill == (uint32_t)PAGE) close_page(0, item);
                }
            }
            if (!ok) break;
            if (!open && !(ok = open_page())) break;
            close_page(F_ITEM_END, item);  // the tile's last page, possibly empty
        }
        // termination page (every generator reads every page)
        if (ok && (ok = open_page())) close_page(F_TERM, 0);
        if (!ok) {
            if (open) close_page(F_TERM, 0);
            for (uint32_t q = (pg > NPAGES ? pg - NPAGES : 0); q < pg; ++q)
                drain_bar(bar(L::pfull(q % NPAGES)), (q / NPAGES) & 1u);
        }
    } else if (gi >= 0) {
        // -------------------------------------------------------- generators
        // Every generator reads every page.  The page's owner (page q: generator
        // q mod 8) keeps the events whose cylinder reaches the tile, compacting
        // them in place; chunk c of page q (events 16c .. 16c+15 of the kept list)
        // is then built by generator (q + c) mod 8 into its own stage.
        const uint32_t tab = sb + L::OFF_TAB + gi * TAB_BYTES;
        const uint32_t tabx = tab, taby = tab + TX * TAB_ROW, tt = tab + (TX + TY) * TAB_ROW;
        const uint32_t stg = sb + L::OFF_STAGE + gi * STAGE_BYTES;
        const uint32_t a_hi = stg, a_lo = stg + A_BYTES, b_hi = stg + 2 * A_BYTES,
                       b_lo = b_hi + B_BYTES;
        const uint32_t shdr = sb + L::OFF_SHDR + gi * 32;
        const uint32_t lt = (1u << lane) - 1u;
        const float csct = pl.cs * pl.ct;
        uint32_t suse = 0;  // uses of this warp's stage
        bool ok = true;
        // hands the stage to the MMA thread, with what it needs precomputed: the
        // instruction descriptor, the 32-column blocks the MMAs touch and the
        // per-block chunk-count increments (bytes, four blocks per word)
        const uint32_t fmt = FP16 ? 0u : 1u;
        auto publish = [&](int c0, int ncols, int flags) {
            if (lane == 0) {
                uint32_t idesc = 0, mask = 0, inc_lo = 0, inc_hi = 0;
                if (flags & F_MMA) {
                    idesc = ptx::idesc_f16(128, (uint32_t)ncols, fmt);
                    const uint32_t b0 = (uint32_t)c0 >> 5, b1 = (uint32_t)(c0 + ncols - 1) >> 5;
                    mask = ((2u << b1) - 1u) & ~((1u << b0) - 1u);
                    inc_lo = ((mask & 15u) * 0x204081u) & 0x01010101u;
                    inc_hi = ((mask >> 4) * 0x204081u) & 0x01010101u;
                }
                ptx::sts_i4(shdr, make_int4(c0, ncols, flags, 0));
                ptx::sts_i4(shdr + 16, make_int4((int)idesc, (int)mask, (int)inc_lo, (int)inc_hi));
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(bar(L::sfull(gi)));
            ++suse;
        };
        // Keeps the events of page fq (staged, owned by this generator) whose
        // cylinder reaches their tile, compacted in place, and publishes the count.
        uint32_t filt_next = (uint32_t)gi;  // next owned page not yet filtered
        auto filter_page = [&](uint32_t fq) {
            const uint32_t fp = fq % NPAGES;
            const uint32_t fb = sb + L::OFF_PAGES + fp * PAGE * 16;
            const int4 fm = ptx::lds_i4(sb + L::OFF_PMETA + fp * 16);
            uint32_t kept = 0;
            if (!(fm.y & F_TERM)) {
                const int64_t fitem = (int64_t)(uint32_t)fm.z | ((int64_t)fm.w << 32);
                int ftx, fty, ftb;
                decode_item(pl, fitem, ftx, fty, ftb);
                const TileGeom fg = tile_geom(pl, ftx, fty, ftb, NB);
                for (int r = 0; r * 32 < fm.x; ++r) {
                    const int slot = r * 32 + lane;
                    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
                    bool keep = false;
                    if (slot < fm.x) {
                        e = ptx::lds_f4(fb + slot * 16u);
                        keep = reaches(pl, fg, e);
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                    __syncwarp();
                    if (keep) ptx::sts_f4(fb + (kept + __popc(bal & lt)) * 16u, e);
                    kept += __popc(bal);
                    __syncwarp();
                }
            }
            if (lane == 0) {
                ptx::sts_i4(sb + L::OFF_KEPT + fp * 16, make_int4((int)kept, 0, 0, 0));
                ptx::mbar_arrive(bar(L::pfilt(fp)));
            }
            __syncwarp();
            filt_next = fq + NGEN;
        };
        // filters the next owned page ahead of time if it is already staged
        auto filter_ahead = [&](uint32_t q) {
            if (filt_next > q && filt_next < q + NPAGES) {
                const uint32_t fp = filt_next % NPAGES;
                const bool ready = __all_sync(0xffffffffu,
                    ptx::mbar_try_wait(bar(L::pfull(fp)), (filt_next / NPAGES) & 1u));
                if (ready) filter_page(filt_next);
            }
        };
        for (uint32_t q = 0; ok; ++q) {
            const uint32_t p = q % NPAGES;
            const uint32_t ph = (q / NPAGES) & 1u;
            const uint32_t pgb = sb + L::OFF_PAGES + p * PAGE * 16;
            if (!(ok = wait_warp(c, bar(L::pfull(p)), ph))) break;
            const int4 meta = ptx::lds_i4(sb + L::OFF_PMETA + p * 16);
            if (meta.y & F_TERM) break;
            const int64_t item = (int64_t)(uint32_t)meta.z | ((int64_t)meta.w << 32);
            const int end = meta.y & F_ITEM_END;
            int tx, ty, tb;
            decode_item(pl, item, tx, ty, tb);
            const TileGeom g = tile_geom(pl, tx, ty, tb, NB);
            const int X0 = g.X0, Y0 = g.Y0, T0 = g.T0, nbv = g.T1 - g.T0;
            if ((int)(q % NGEN) == gi && q >= filt_next) {
                // this generator owns page q and has not filtered it ahead: do it now
                filter_page(q);
            } else if (!(ok = wait_warp(c, bar(L::pfilt(p)), ph))) {
                break;
            }
            const int kept = ptx::lds_i4(sb + L::OFF_KEPT + p * 16).x;
            const int nch = (kept + CHUNK - 1) / CHUNK;
            if (nch == 0 && (int)(q % NGEN) == gi) {  // nothing to add: just mark the page's end
                if (!(ok = wait_warp(c, bar(L::sempty(gi)), (suse & 1u) ^ 1u))) break;
                publish(0, 0, F_PAGE_END | end);
            }
            for (int ch = (int)((gi - (int)(q % NGEN) + NGEN) % NGEN); ch < nch && ok; ch += NGEN) {
                filter_ahead(q);
                const int count = min(CHUNK, kept - ch * CHUNK);
                float4 e = make_float4(1.0e30f, 1.0e30f, 1.0e30f, 0.f);
                if (lane < count) e = ptx::lds_f4(pgb + (ch * CHUNK + lane) * 16u);
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
                    const int qq = i * 32 + lane, x = qq >> 4, k = qq & 15;
                    const float ex = __shfl_sync(0xffffffffu, e.x, k);
                    const float du = ((float)(X0 + x) + 0.5f - ex) * pl.inv_hs;
                    const float u2 = du * du;
                    ptx::sts_f2(tabx + x * TAB_ROW + k * 8, make_float2(u2, 1.0f - u2));
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int qq = i * 32 + lane, y = qq >> 4, k = qq & 15;
                    const float ey = __shfl_sync(0xffffffffu, e.y, k);
                    const float dv = ((float)(Y0 + y) + 0.5f - ey) * pl.inv_hs;
                    const float v2 = dv * dv;
                    ptx::sts_f2(taby + y * TAB_ROW + k * 8, make_float2(v2, 1.0f - v2));
                }
                if (lane < CHUNK) ptx::sts_f(tt + lane * 4, e.z);
                __syncwarp();

                if (!(ok = wait_warp(c, bar(L::sempty(gi)), (suse & 1u) ^ 1u))) break;
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
                    if (cw != c0 && !(ok = wait_warp(c, bar(L::sempty(gi)), (suse & 1u) ^ 1u))) break;
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
                    const bool more = cw + NCAP < cend;
                    const int fl = F_MMA | (more ? F_MORE : 0) |
                                   ((!more && ch == nch - 1) ? (F_PAGE_END | end) : 0);
                    publish(cw, ncols, fl);
                }
            }
            if (!ok) break;
            // done with the page: order these generic accesses before the loader's
            // next bulk copy into it, then release it
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(bar(L::pempty(p)));
        }
    } else if (warp == WARP_MMA) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            uint32_t par = 0;  // bit g: parity of the next use of generator g's stage
            uint32_t seg = 0;  // accumulator segments opened so far
            uint32_t qm = 0;   // next page
            bool ok = true;
            // descriptors of stage 0; stage g adds g * STAGE_BYTES / 16 to the address field
            const uint64_t d_ahi = ptx::smem_desc(sb + L::OFF_STAGE, CORE_LBO, CORE_SBO);
            const uint64_t d_alo = d_ahi + (A_BYTES >> 4);
            const uint64_t d_bhi = d_ahi + ((2 * A_BYTES) >> 4);
            const uint64_t d_blo = d_ahi + ((2 * A_BYTES + B_BYTES) >> 4);
            // chunks per 32-column block before a segment is closed, four blocks per word
            const uint32_t thr4 = (uint32_t)flush_chunks * 0x01010101u;
            for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                int b = (int)(seg & 1u);
                if (!(ok = wait_bar(c, bar(L::aempty(b)), (seg >> 1) & 1u))) break;
                ptx::tc_fence_after();
                int first = 1;
                uint32_t touched = 0;             // 32-column blocks written in this segment
                uint32_t cnt_lo = 0, cnt_hi = 0;  // chunks per 32-column block (bytes)
                int flags = 0;
                while (!(flags & F_ITEM_END) && ok) {
                    flags = 0;
                    for (uint32_t ch = 0; !(flags & F_PAGE_END) && ok; ++ch) {
                        const int gq = (int)((qm + ch) % NGEN);
                        flags = F_MORE;
                        while ((flags & F_MORE) && ok) {
                            if (!(ok = wait_bar(c, bar(L::sfull(gq)), (par >> gq) & 1u))) break;
                            par ^= 1u << gq;
                            const int4 h = ptx::lds_i4(sb + L::OFF_SHDR + gq * 32);
                            const int4 h1 = ptx::lds_i4(sb + L::OFF_SHDR + gq * 32 + 16);
                            flags = h.z;
                            // never issue an MMA outside the accumulator
                            const bool in_range = (uint32_t)h.x + (uint32_t)h.y <= (uint32_t)NB &&
                                                  (uint32_t)(h.y - 16) <= (uint32_t)(NCAP - 16) &&
                                                  ((h.x | h.y) & 15) == 0;
                            if (!(flags & F_MMA) || !in_range) {
                                if ((flags & F_MMA) && !in_range) atomicOr(err, ERRBIT_BOUNDS);
                                ptx::mbar_arrive(bar(L::sempty(gq)));
                                continue;
                            }
                            const uint32_t mask = (uint32_t)h1.y;
                            const uint32_t inc_lo = (uint32_t)h1.z, inc_hi = (uint32_t)h1.w;
                            uint32_t n_lo = cnt_lo + inc_lo, n_hi = cnt_hi + inc_hi;
                            if (__vcmpgtu4(n_lo, thr4) | __vcmpgtu4(n_hi, thr4)) {
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
                                n_lo = inc_lo;
                                n_hi = inc_hi;
                            }
                            cnt_lo = n_lo;
                            cnt_hi = n_hi;
                            touched |= mask;
                            const uint64_t so = (uint64_t)gq * (STAGE_BYTES >> 4);
                            const uint32_t idesc = (uint32_t)h1.x;
                            const uint32_t d = tmem + (uint32_t)(b * NB + h.x);
                            ptx::mma_f16_ss(d, d_ahi + so, d_bhi + so, idesc, 1);
                            ptx::mma_f16_ss(d, d_ahi + so, d_blo + so, idesc, 1);
                            ptx::mma_f16_ss(d, d_alo + so, d_bhi + so, idesc, 1);
                            ptx::tc_commit(bar(L::sempty(gq)));
                        }
                    }
                    ++qm;
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
    } else if (warp >= WARP_EPI0) {
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
                    float4* p4 = reinterpret_cast<float4*>(dst + col);
                    float4 pv[8];
                    if (!first) {  // earlier segments of this tile: load all, then add
#pragma unroll
                        for (int v4 = 0; v4 < 8; ++v4) pv[v4] = p4[v4];
                    }
#pragma unroll
                    for (int v4 = 0; v4 < 8; ++v4) {
                        float4 o = make_float4(__uint_as_float(r[4 * v4]) * pl.norm,
                                               __uint_as_float(r[4 * v4 + 1]) * pl.norm,
                                               __uint_as_float(r[4 * v4 + 2]) * pl.norm,
                                               __uint_as_float(r[4 * v4 + 3]) * pl.norm);
                        if (!first) {
                            o.x += pv[v4].x; o.y += pv[v4].y; o.z += pv[v4].z; o.w += pv[v4].w;
                        }
                        if (last) __stcs(p4 + v4, o); else p4[v4] = o;
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
    // chunks (three accumulation steps each) per 32-column block before a segment
    // is closed: bounds the round-toward-zero drift of the tensor-core
    // accumulation per segment
    const int flush_chunks = FP16 ? 64 : 128;
    kern<<<grid, NTHREADS, L::TOTAL, st>>>(pl, b.ev, b.start, out, err, items, flush_chunks);
    return true;
}

}  // namespace

bool launch_tile_tc(const Plan& pl, const Bins& b, float* out, int* err, int fp16,
                    cudaStream_t st) {
    return fp16 ? launch_cfg<true>(pl, b, out, err, st) : launch_cfg<false>(pl, b, out, err, st);
}

}  // namespace stkde
