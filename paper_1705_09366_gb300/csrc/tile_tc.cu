// K5: tcgen05 tensor-core tile kernel.
//
// PB-SYM (Section 3.2, Algorithm 3) adds, for every event i, the outer product
// of its spatial invariant K_s,i[X][Y] and its temporal invariant K_t,i[T].
// Inside one output tile of 128 voxels in the plane (16 x 8) by up to 256
// voxels of T, the sum over the events that reach the tile is a rank-k
// contraction
//     C[xy][t] = sum_k A[xy][k] * B[k][t],  A = K_s (128 x k),  B = K_t (k x t),
// which runs on the tensor cores: tcgen05.mma, M = 128, K = 16 events per
// instruction, N = the T columns the 16 events' windows cover (16..NCAP), the
// fp32 accumulator in tensor memory.  For accuracy A and B are split into a
// 16-bit high part and a 16-bit remainder, and three products hi*hi + hi*lo +
// lo*hi are accumulated (the dropped lo*lo term is below 2^-16 relative).
//
// Persistent CTA per SM, warp-specialised:
//   warp 0      MMA issue (one thread) and tensor-memory allocation
//   warp 1      loader: walks the tile's event bins and stages them into shared
//               memory pages with cp.async.bulk (no multicast), one mbarrier per page
//   warps 2-9   generator group (256 threads): filters each page jointly, appends
//               the events whose cylinder reaches the tile to a ring in bin order,
//               and turns every run of (up to) 16 kept events into one chunk --
//               A = K_s and B = K_t as hi and lo operand tiles -- in a ring of
//               operand stages
//   warps 10-13 epilogue: one per tensor-memory lane quarter; reads the
//               accumulator, scales by 1/(n hs^2 ht), writes every voxel of the
//               tile once with vector stores, and zeroes the accumulator
// Two accumulators of 256 columns let the epilogue of one tile overlap the MMAs
// of the next.  Chunks are formed from the kept-event stream in order and the
// MMA thread consumes them in that order, so every voxel sums its events in the
// same order on every run: the result is bit-reproducible, and no global
// atomics are used.  With a single producer group and a single consumer no
// wait can close a cycle.
//
// Every wait on an mbarrier is bounded (2 s of %globaltimer); on expiry the
// kernel sets the timeout bit of the error word, every role leaves its loop
// (the generator group decides together, through a reducing named barrier),
// outstanding copies and MMAs are drained with a second bounded wait, and the
// tensor memory is freed before the CTA exits.
#include "internal.cuh"
#include "ptx.cuh"
#include "tile_common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace stkde {

namespace {

constexpr int NB = 256;           // T columns per tile = accumulator width
constexpr int NACC = 2;           // accumulators (512 tensor-memory columns)
constexpr int NGEN = 8;           // generator warps
constexpr int NEPI = 4;           // epilogue warps
constexpr int WARP_MMA = 0;
constexpr int WARP_LOAD = 1;
constexpr int WARP_GEN0 = 2;
constexpr int WARP_EPI0 = WARP_GEN0 + NGEN;
constexpr int GEN_THREADS = 32 * NGEN;
constexpr int NTHREADS = (WARP_EPI0 + NEPI) * 32;
constexpr int PAGE = GEN_THREADS; // events per staging page: one per generator thread
constexpr int NPAGES = 4;
constexpr int CHUNK = 16;         // events per MMA (K of kind::f16)
constexpr int KRING = 512;        // kept-event ring (>= PAGE + CHUNK)
constexpr int GEN_BAR = 1;        // named barrier of the generator group
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr uint64_t DRAIN_NS = 200000000ull;
constexpr uint32_t A_BYTES = TILE_XY * CHUNK * 2;
constexpr uint32_t CORE_LBO = 128;  // next core matrix along K
constexpr uint32_t CORE_SBO = 256;  // next core matrix along M / N

template <int NCAP, int S>
struct Layout {
    static constexpr uint32_t B_BYTES = NCAP * CHUNK * 2;
    static constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr uint32_t OFF_STAGES = 0;
    static constexpr uint32_t OFF_PAGES = OFF_STAGES + S * STAGE_BYTES;
    static constexpr uint32_t OFF_KRING = OFF_PAGES + NPAGES * PAGE * 16;
    static constexpr uint32_t OFF_TABX = OFF_KRING + KRING * 16;   // [16 x][16 k] float2
    static constexpr uint32_t OFF_TABY = OFF_TABX + TX * CHUNK * 8; // [8 y][16 k] float2
    static constexpr uint32_t OFF_TT = OFF_TABY + TY * CHUNK * 8;   // [16 k] float
    static constexpr uint32_t OFF_HDR = OFF_TT + CHUNK * 4;
    static constexpr uint32_t OFF_PMETA = OFF_HDR + S * 16;
    static constexpr uint32_t OFF_WCNT = OFF_PMETA + NPAGES * 16;
    static constexpr uint32_t OFF_BAR = OFF_WCNT + 64;
    static constexpr int NBARS = 2 * NPAGES + 2 * S + 2 * NACC + 1;
    static constexpr uint32_t OFF_MISC = OFF_BAR + NBARS * 8;
    static constexpr uint32_t TOTAL = OFF_MISC + 16;
    __device__ static constexpr int pfull(int p) { return p; }
    __device__ static constexpr int pempty(int p) { return NPAGES + p; }
    __device__ static constexpr int sfull(int s) { return 2 * NPAGES + s; }
    __device__ static constexpr int sempty(int s) { return 2 * NPAGES + S + s; }
    __device__ static constexpr int afull(int b) { return 2 * NPAGES + 2 * S + b; }
    __device__ static constexpr int aempty(int b) { return 2 * NPAGES + 2 * S + NACC + b; }
    __device__ static constexpr int drain() { return 2 * NPAGES + 2 * S + 2 * NACC; }
    static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
    static_assert(TOTAL <= 227 * 1024, "shared memory budget");
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

__device__ __forceinline__ void sts128(uint8_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    *reinterpret_cast<uint4*>(p) = make_uint4(a, b, c, d);
}

// Named barrier of the generator group that also ORs a predicate over it.
__device__ __forceinline__ bool gen_bar_or(bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "n"(GEN_BAR), "n"(GEN_THREADS)
        : "memory");
    return r != 0;
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

// The same for a whole warp: every lane waits, and the warp proceeds only if
// all lanes saw the phase complete, so a timeout never splits the warp.
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

template <int NCAP, int S, bool FP16>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tile_tc(Plan pl, const float4* __restrict__ ev, const uint32_t* __restrict__ start,
          float* __restrict__ out, int* __restrict__ err, int64_t nitems) {
    using L = Layout<NCAP, S>;
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t sbase = ptx::smem_addr(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::OFF_MISC);
    Ctl c{reinterpret_cast<volatile int*>(smem + L::OFF_MISC + 4), err};
    auto bar = [&](int i) -> uint32_t { return sbase + L::OFF_BAR + 8u * (uint32_t)i; };
    int4* hdr = reinterpret_cast<int4*>(smem + L::OFF_HDR);

    if (threadIdx.x == 0) {
        for (int p = 0; p < NPAGES; ++p) {
            ptx::mbar_init(bar(L::pfull(p)), 1);
            ptx::mbar_init(bar(L::pempty(p)), NGEN);
        }
        for (int s = 0; s < S; ++s) {
            ptx::mbar_init(bar(L::sfull(s)), 1);
            ptx::mbar_init(bar(L::sempty(s)), 1);
        }
        for (int b = 0; b < NACC; ++b) {
            ptx::mbar_init(bar(L::afull(b)), 1);
            ptx::mbar_init(bar(L::aempty(b)), NEPI);
        }
        ptx::mbar_init(bar(L::drain()), 1);
        *c.abort = 0;
        ptx::fence_mbar_init();
    }
    if (warp == WARP_MMA) {
        ptx::tmem_alloc(ptx::smem_addr(tmem_slot), NB * NACC);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == WARP_LOAD) {
        // ------------------------------------------------------------ loader
        uint32_t pg = 0, fill = 0;
        bool open = false, ok = true;
        auto pages = [&](uint32_t p) -> uint32_t { return sbase + L::OFF_PAGES + p * PAGE * 16; };
        auto close_page = [&](uint32_t count, int end) {
            const uint32_t p = pg % NPAGES;
            if (lane == 0) {
                int4* meta = reinterpret_cast<int4*>(smem + L::OFF_PMETA) + p;
                *meta = make_int4((int)count, end, 0, 0);
                ptx::mbar_arrive(bar(L::pfull(p)));
            }
            __syncwarp();
            ++pg;
            open = false;
        };
        auto open_page = [&]() -> bool {
            const uint32_t p = pg % NPAGES;
            if (!wait_warp(c, bar(L::pempty(p)), ((pg / NPAGES) & 1u) ^ 1u)) return false;
            open = true;
            fill = 0;
            return true;
        };
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            int tx, ty, tb;
            decode_item(pl, item, tx, ty, tb);
            const TileGeom g = tile_geom(pl, tx, ty, tb, NB);
            const int ncx = g.cx_hi - g.cx_lo + 1;
            const int nr = (g.s_hi >= g.s_lo && ncx > 0) ? (g.s_hi - g.s_lo + 1) * ncx : 0;
            for (int r0 = 0; r0 < nr && ok; r0 += 32) {
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
                for (int j = 0; j < nj && ok; ++j) {
                    uint32_t aj = __shfl_sync(0xffffffffu, a, j);
                    const uint32_t bj = __shfl_sync(0xffffffffu, b, j);
                    while (aj < bj) {
                        if (!open && !(ok = open_page())) break;
                        const uint32_t take = min(bj - aj, (uint32_t)PAGE - fill);
                        const uint32_t p = pg % NPAGES;
                        if (lane == 0) {
                            ptx::mbar_expect_tx(bar(L::pfull(p)), take * 16u);
                            ptx::bulk_g2s(pages(p) + fill * 16u, ev + aj, take * 16u,
                                          bar(L::pfull(p)));
                        }
                        fill += take;
                        aj += take;
                        if (fill == (uint32_t)PAGE) close_page(PAGE, 0);
                    }
                }
            }
            if (!ok) break;
            if (!open && !(ok = open_page())) break;
            close_page(fill, 1);
        }
        if (!ok) {
            // drain: close an open page so its copies can complete, then wait for
            // the most recent fill of every page
            if (open) close_page(fill, 1);
            for (uint32_t q = (pg > NPAGES ? pg - NPAGES : 0); q < pg; ++q)
                drain_bar(bar(L::pfull(q % NPAGES)), (q / NPAGES) & 1u);
        }
    } else if (warp >= WARP_GEN0 && warp < WARP_EPI0) {
        // --------------------------------------------------- generator group
        const int gt = threadIdx.x - WARP_GEN0 * 32;  // 0..255
        const int gwi = gt >> 5;
        const uint32_t lt = (1u << lane) - 1u;
        const float4* pagesp = reinterpret_cast<const float4*>(smem + L::OFF_PAGES);
        float4* kring = reinterpret_cast<float4*>(smem + L::OFF_KRING);
        float2* tabx = reinterpret_cast<float2*>(smem + L::OFF_TABX);
        float2* taby = reinterpret_cast<float2*>(smem + L::OFF_TABY);
        float* tt = reinterpret_cast<float*>(smem + L::OFF_TT);
        volatile int* wcnt = reinterpret_cast<volatile int*>(smem + L::OFF_WCNT);
        const float4 far = make_float4(1.0e30f, 1.0e30f, 1.0e30f, 0.0f);
        const float csct = pl.cs * pl.ct;
        uint32_t pg = 0, sc = 0;
        uint32_t kabs = 0, jabs = 0;  // kept events appended / consumed (ring positions)
        bool ok = true;

        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            int tx, ty, tb;
            decode_item(pl, item, tx, ty, tb);
            const TileGeom g = tile_geom(pl, tx, ty, tb, NB);
            const int nbv = g.T1 - g.T0;

            // One chunk from kring[jabs, jabs + take): every warp derives the same
            // take / column range, then the group builds the operand tiles.
            auto chunk = [&]() -> bool {
                const int avail = (int)min(kabs - jabs, (uint32_t)CHUNK);
                int lo = 0x7fffffff, hi = -0x7fffffff;
                if (lane < avail) {
                    // the event's T window clipped into the block; the filter's margin
                    // can keep an event whose window misses the block, so both ends are
                    // clamped into [0, nbv-1] (its K_t values there are zero anyway)
                    const float pt = kring[(jabs + lane) % KRING].z;
                    lo = min(max((int)ceilf(pt - 0.5f - pl.htv) - g.T0, 0), nbv - 1);
                    hi = min(max((int)floorf(pt - 0.5f + pl.htv) - g.T0, lo), nbv - 1);
                }
                int pmin = lo, pmax = hi;
#pragma unroll
                for (int off = 1; off < 16; off <<= 1) {
                    const int vmin = __shfl_up_sync(0xffffffffu, pmin, off);
                    const int vmax = __shfl_up_sync(0xffffffffu, pmax, off);
                    if (lane >= off) { pmin = min(pmin, vmin); pmax = max(pmax, vmax); }
                }
                const int c0k = pmin & ~15;
                const bool fits = lane < avail && (pmax - c0k + 1) <= NCAP;
                const uint32_t fm = __ballot_sync(0xffffffffu, fits) & 0xffffu;
                int take = __ffs(~fm) - 1;  // length of the leading run of fitting prefixes
                take = max(1, min(take, avail));
                const int c0 = __shfl_sync(0xffffffffu, c0k, take - 1);
                const int cmax = __shfl_sync(0xffffffffu, pmax, take - 1);
                const int ncols = min(NCAP, ((cmax - c0 + 1) + 15) & ~15);

                const int s = (int)(sc % S);
                const bool wok = wait_warp(c, bar(L::sempty(s)), ((sc / S) & 1u) ^ 1u);
                // factor tables of K_s: (u^2, 1-u^2) per x and (v^2, 1-v^2) per y, per event
                {
                    const int k = gt & 15;
                    const float4 e = k < take ? kring[(jabs + k) % KRING] : far;
                    const int x = gt >> 4;  // 0..15
                    const float du = ((float)(g.X0 + x) + 0.5f - e.x) * pl.inv_hs;
                    const float u2 = du * du;
                    tabx[x * CHUNK + k] = make_float2(u2, 1.0f - u2);
                    if (gt < TY * CHUNK) {
                        const int y = gt >> 4;  // 0..7
                        const float dv = ((float)(g.Y0 + y) + 0.5f - e.y) * pl.inv_hs;
                        const float v2 = dv * dv;
                        taby[y * CHUNK + k] = make_float2(v2, 1.0f - v2);
                    }
                    if (gt < CHUNK) tt[gt] = e.z;
                }
                if (gen_bar_or(!wok)) return false;  // tables visible; all agree on aborting

                uint8_t* st = smem + L::OFF_STAGES + (uint32_t)s * L::STAGE_BYTES;
                uint8_t* a_hi = st;
                uint8_t* a_lo = st + A_BYTES;
                uint8_t* b_hi = st + 2 * A_BYTES;
                uint8_t* b_lo = b_hi + L::B_BYTES;
                const int kg = gt >> 7;       // events kg*8 .. kg*8+7
                {
                    // A = K_s without c_s: row r = voxel (x = r / 8, y = r % 8)
                    const int r = gt & 127;
                    const float4* txp = reinterpret_cast<const float4*>(tabx + (r >> 3) * CHUNK + kg * 8);
                    const float4* typ = reinterpret_cast<const float4*>(taby + (r & 7) * CHUNK + kg * 8);
                    uint32_t ah[4], al[4];
#pragma unroll
                    for (int kp = 0; kp < 4; ++kp) {
                        const float4 fx = txp[kp];  // (u2, 1-u2) of events 2kp, 2kp+1
                        const float4 fy = typ[kp];
                        const float a0 = (fx.x + fy.x < 1.0f) ? fx.y * fy.y : 0.0f;
                        const float a1 = (fx.z + fy.z < 1.0f) ? fx.w * fy.w : 0.0f;
                        split2<FP16>(a0, a1, ah[kp], al[kp]);
                    }
                    const uint32_t off = (uint32_t)(r >> 3) * CORE_SBO + kg * CORE_LBO + (r & 7) * 16;
                    sts128(a_hi + off, ah[0], ah[1], ah[2], ah[3]);
                    sts128(a_lo + off, al[0], al[1], al[2], al[3]);
                }
                // B = c_s c_t (1 - w^2)_+: row n = T column (T0 + c0 + n)
                for (int n = gt & 127; n < ncols; n += 128) {
                    const float tc = (float)(g.T0 + c0 + n) + 0.5f;
                    uint32_t bh[4], bl[4];
#pragma unroll
                    for (int kp = 0; kp < 4; ++kp) {
                        const float w0 = (tc - tt[kg * 8 + 2 * kp]) * pl.inv_ht;
                        const float w1 = (tc - tt[kg * 8 + 2 * kp + 1]) * pl.inv_ht;
                        const float b0 = csct * fmaxf(fmaf(-w0, w0, 1.0f), 0.0f);
                        const float b1 = csct * fmaxf(fmaf(-w1, w1, 1.0f), 0.0f);
                        split2<FP16>(b0, b1, bh[kp], bl[kp]);
                    }
                    const uint32_t off = (uint32_t)(n >> 3) * CORE_SBO + kg * CORE_LBO + (n & 7) * 16;
                    sts128(b_hi + off, bh[0], bh[1], bh[2], bh[3]);
                    sts128(b_lo + off, bl[0], bl[1], bl[2], bl[3]);
                }
                if (gt == 0) hdr[s] = make_int4(c0, ncols, 1, 0);
                ptx::fence_proxy_async_smem();
                gen_bar_or(false);  // stage complete; tables free for the next chunk
                if (gt == 0) ptx::mbar_arrive(bar(L::sfull(s)));
                ++sc;
                jabs += (uint32_t)take;
                return true;
            };

            bool end = false;
            while (!end && ok) {
                const uint32_t p = pg % NPAGES;
                const bool wok = wait_warp(c, bar(L::pfull(p)), (pg / NPAGES) & 1u);
                int4 meta = make_int4(0, 1, 0, 0);
                float4 e = far;
                bool keep = false;
                if (wok) {
                    meta = reinterpret_cast<const int4*>(smem + L::OFF_PMETA)[p];
                    if (gt < meta.x) {
                        e = pagesp[p * PAGE + gt];
                        keep = reaches(pl, g, e);
                    }
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(bar(L::pempty(p)));
                }
                ++pg;
                const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) wcnt[gwi] = __popc(bal);
                if (gen_bar_or(!wok)) { ok = false; break; }  // counts visible
                end = meta.y != 0;
                int pre = 0, tot = 0;
#pragma unroll
                for (int w = 0; w < NGEN; ++w) {
                    const int cw = wcnt[w];
                    pre += w < gwi ? cw : 0;
                    tot += cw;
                }
                if (keep) kring[(kabs + (uint32_t)pre + __popc(bal & lt)) % KRING] = e;
                kabs += (uint32_t)tot;
                gen_bar_or(false);  // ring writes visible; wcnt free
                while (ok && (kabs - jabs >= (uint32_t)CHUNK || (end && kabs > jabs))) ok = chunk();
            }
            if (!ok) break;
            // end-of-tile marker
            const int s = (int)(sc % S);
            bool wok = true;
            if (gwi == 0) {
                wok = wait_warp(c, bar(L::sempty(s)), ((sc / S) & 1u) ^ 1u);
                if (wok && lane == 0) {
                    hdr[s] = make_int4(0, 0, 0, 0);
                    ptx::mbar_arrive(bar(L::sfull(s)));
                }
            }
            if (gen_bar_or(!wok)) break;
            ++sc;
        }
    } else if (warp == WARP_MMA) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            uint32_t sc = 0;
            bool ok = true;
            int64_t it = 0;
            const uint32_t fmt = FP16 ? 0u : 1u;
            for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++it) {
                const int b = (int)(it & 1);
                const uint32_t use = (uint32_t)(it >> 1);
                if (!(ok = wait_bar(c, bar(L::aempty(b)), use & 1u))) break;
                ptx::tc_fence_after();
                while (true) {
                    const int s = (int)(sc % S);
                    if (!(ok = wait_bar(c, bar(L::sfull(s)), (sc / S) & 1u))) break;
                    ptx::tc_fence_after();
                    const int4 h = hdr[s];
                    ++sc;
                    if (h.z == 0) {
                        ptx::mbar_arrive(bar(L::sempty(s)));
                        break;
                    }
                    const bool in_range = h.x >= 0 && h.y >= 16 && h.y <= NCAP &&
                                          (h.y & 15) == 0 && h.x + h.y <= NB;
                    if (!in_range) {  // never issue an MMA outside the accumulator
                        atomicOr(err, ERRBIT_BOUNDS);
                        ptx::mbar_arrive(bar(L::sempty(s)));
                        continue;
                    }
                    const uint32_t stg = sbase + L::OFF_STAGES + (uint32_t)s * L::STAGE_BYTES;
                    const uint64_t ahi = ptx::smem_desc(stg, CORE_LBO, CORE_SBO);
                    const uint64_t alo = ptx::smem_desc(stg + A_BYTES, CORE_LBO, CORE_SBO);
                    const uint64_t bhi = ptx::smem_desc(stg + 2 * A_BYTES, CORE_LBO, CORE_SBO);
                    const uint64_t blo =
                        ptx::smem_desc(stg + 2 * A_BYTES + L::B_BYTES, CORE_LBO, CORE_SBO);
                    const uint32_t idesc = ptx::idesc_f16(128, (uint32_t)h.y, fmt);
                    const uint32_t d = tmem + (uint32_t)(b * NB + h.x);
                    ptx::mma_f16_ss(d, ahi, bhi, idesc, 1);
                    ptx::mma_f16_ss(d, ahi, blo, idesc, 1);
                    ptx::mma_f16_ss(d, alo, bhi, idesc, 1);
                    ptx::tc_commit(bar(L::sempty(s)));
                }
                if (!ok) break;
                ptx::tc_commit(bar(L::afull(b)));
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
        if (lane == 0) {
            for (int b = 0; b < NACC; ++b) ptx::mbar_arrive(bar(L::aempty(b)));
        }
        bool ok = true;
        int64_t it = 0;
        const bool vec = (pl.gt & 3) == 0;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++it) {
            const int b = (int)(it & 1);
            const uint32_t use = (uint32_t)(it >> 1);
            if (!(ok = wait_warp(c, bar(L::afull(b)), use & 1u))) break;
            ptx::tc_fence_after();
            int tx, ty, tb;
            decode_item(pl, item, tx, ty, tb);
            const int m = 32 * q + lane;
            const int X = tx * TX + m / TY, Y = ty * TY + m % TY, T0 = tb * NB;
            const int nbv = min(NB, pl.gt - T0);
            const bool valid = X < pl.gx && Y < pl.gy;
            float* dst = out + ((int64_t)X * pl.gy + Y) * (int64_t)pl.gt + T0;
            for (int col = 0; col < nbv; col += 32) {
                uint32_t r[32];
                const uint32_t ta = trow + (uint32_t)(b * NB + col);
                ptx::tmem_ld32(ta, r);
                ptx::tmem_wait_ld();
                ptx::tmem_st32_zero(ta);
                if (valid) {
                    const int nv = min(32, nbv - col);
                    if (vec && nv == 32) {
#pragma unroll
                        for (int v4 = 0; v4 < 8; ++v4) {
                            const float4 o = make_float4(__uint_as_float(r[4 * v4]) * pl.norm,
                                                         __uint_as_float(r[4 * v4 + 1]) * pl.norm,
                                                         __uint_as_float(r[4 * v4 + 2]) * pl.norm,
                                                         __uint_as_float(r[4 * v4 + 3]) * pl.norm);
                            __stcs(reinterpret_cast<float4*>(dst + col) + v4, o);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < nv) __stcs(dst + col + j, __uint_as_float(r[j]) * pl.norm);
                    }
                }
            }
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(bar(L::aempty(b)));
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == WARP_MMA) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, NB * NACC);
    }
}

template <int NCAP, int S, bool FP16>
bool launch_cfg(const Plan& pl, const Bins& b, float* out, int* err, cudaStream_t st) {
    using L = Layout<NCAP, S>;
    auto kern = k_tile_tc<NCAP, S, FP16>;
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
    kern<<<grid, NTHREADS, L::TOTAL, st>>>(pl, b.ev, b.start, out, err, items);
    return true;
}

}  // namespace

bool launch_tile_tc(const Plan& pl, const Bins& b, float* out, int* err, int fp16,
                    cudaStream_t st) {
    // A chunk spans at most NCAP columns: one event's window (2 ceil(ht) + 1
    // voxels), the 16-column alignment of its start, and room for the spread of
    // the 16 events' times.
    const int win = 2 * (int)ceilf(pl.htv) + 1;
    if (win + 15 + 8 <= 64)
        return fp16 ? launch_cfg<64, 12, true>(pl, b, out, err, st)
                    : launch_cfg<64, 12, false>(pl, b, out, err, st);
    if (win + 15 + 8 <= 128)
        return fp16 ? launch_cfg<128, 10, true>(pl, b, out, err, st)
                    : launch_cfg<128, 10, false>(pl, b, out, err, st);
    return fp16 ? launch_cfg<256, 7, true>(pl, b, out, err, st)
                : launch_cfg<256, 7, false>(pl, b, out, err, st);
}

}  // namespace stkde
