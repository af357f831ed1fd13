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
// accumulated (the dropped lo*lo term is below 2^-15 relative).
//
// The tensor cores round each accumulation step toward zero, so a long run of
// steps into one accumulator drifts low.  The MMA warp therefore counts the
// chunks each 32-column block of the accumulator has taken and, before a block
// would reach a fixed count, hands just the blocks at the limit to the epilogue
// (a "flush"): the first drain of a block stores it, later drains add to the
// stored values in fp32 (round to nearest), which bounds the drift.  The tile's
// last drain writes every block, zeros included, so each voxel is stored once.
//
// Persistent CTA per SM holding two independent pipelines ("streams"), each
// with its own loader, four generators, stage ring, MMA warp and 256-column
// accumulator; the four epilogue warps serve both.  One MMA warp issues at most
// one entry every few hundred cycles (stage wait, header, three MMAs, commit),
// so two streams double the issue rate.  Tiles are handed out on demand from one
// global counter (zeroed before the launch) to whichever stream of whichever CTA
// is free, which evens out the clustered workloads' uneven tiles; each tile is
// computed by one stream in a fixed order, so the result does not depend on
// which stream or CTA computes it.  Roles (warp w runs on scheduler w % 4):
//   warps 0, 8        MMA issue for streams 0, 1 (the whole warp runs the loop,
//                     one elected lane issues); warp 0 allocates tensor memory
//   warps 4, 11       loaders: walk a tile's event bins and stage them, in bin
//                     order, into 256-event shared-memory pages with
//                     cp.async.bulk (no multicast), one copy per bin run, all
//                     lanes issuing in parallel; then, one page behind, keep the
//                     events whose cylinder reaches the tile (compacting the page
//                     in place) and record per chunk of 16 kept events the T
//                     columns their windows cover, and the page's entry table
//   warps 1-3,5       generators of stream 0; warps 6,7,9,10 of stream 1.
//                     Every generator of a stream reads every page of it.  Each
//                     chunk becomes one "entry" per column window of up to 80
//                     columns; entry e of a stream is built by generator e mod 4
//                     into stage e mod 6 of the stream's ring: A = K_s and
//                     B = K_t as hi and lo 16-bit tiles in the tensor cores'
//                     shared memory layout.
//   warps 12-15       epilogue: one per tensor-memory lane quarter; scales by
//                     c_s c_t / (n hs^2 ht), writes each voxel of the tile
//                     (vector stores), adds later drains of a block, zeroes
//                     the drained blocks.  It serves whichever stream has a
//                     drain ready.
// The builder of a stream's earliest unbuilt entry only waits on that stream's
// earlier entries, and the streams share only the epilogue, which never waits on
// a stream's producers, so no wait can close a cycle.
//
// A launch covers all tiles of its problems, or (host outputs computed in slabs
// along X) the tiles of a range of tile columns.  With per-event bandwidths the
// events are binned by bandwidth class as well, and the loader walks each class's
// bins within that class's own reach.
//
// With per-event bandwidths (ADAPT) a page holds 128 events followed by their
// (hsv_i, htv_i, 1/hsv_i, 1/htv_i) records, both staged by the loader; the
// filter and the column windows use each event's own bandwidths, the factor
// tables its own 1/hsv_i (A) and 1/htv_i (B), and A carries the event's weight
// (hs_max/hs_i)^2 (ht_max/ht_i) (the plan holds the largest bandwidths and the
// normalisation 1/(n hs_max^2 ht_max)).  The weight scales both the product and
// the disk-test difference of A, so the mask is unchanged.
//
// Every wait on an mbarrier is bounded (2 s of %globaltimer, or the launch's
// own bound); on expiry the kernel sets the timeout bit of the error word, every
// role leaves its loop, outstanding copies and MMAs are drained with a second
// bounded wait, and the tensor memory is freed before the CTA exits.  A test
// hook makes block 0 withhold the arrival of its first staging page (issuing no
// copy into it), so that this path can be exercised without a fault.
#include "internal.cuh"
#include "ptx.cuh"
#include "tile_common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>

namespace stkde {

namespace {

constexpr int NSTREAM = 2;
constexpr int NB = 256;            // T columns per tile = accumulator width per stream
constexpr int NGEN = 4;            // generator warps per stream
constexpr int NEPI = 4;            // epilogue warps
constexpr int WARP_EPI0 = 12;
constexpr int NTHREADS = 16 * 32;
constexpr int PAGE = 256;          // events per staging page (128 with per-event bandwidths)
constexpr uint32_t PAGE_BYTES = PAGE * 16;
constexpr int NPAGES = 5;          // pages per stream
constexpr int MAXCH = PAGE / 8;    // chunk records per page (8-event chunks of the tf32 forms)
constexpr int MAXENT = 128;        // entries per page: chunks x their column windows
constexpr int NCAP = 80;           // T columns per entry (one column window)
constexpr int NSTAGE = 6;          // stages per stream, handed over one at a time
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr uint64_t DRAIN_NS = 200000000ull;
constexpr uint32_t A_BYTES = TILE_XY * 32;          // one A part: 128 rows x 32 bytes (4 KB)
constexpr uint32_t B_BYTES = NCAP * 32;             // one B part: NCAP rows x 32 bytes (2.5 KB)
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr uint32_t CORE_LBO = 128;  // next core matrix along K
constexpr uint32_t CORE_SBO = 256;  // next core matrix along M / N
enum { FORM_BF16X3 = 0, FORM_FP16X3 = 1, FORM_TF32X3 = 2, FORM_TF32X1 = 3 };

// A chunk is the K of one MMA: 16 events of 16-bit parts (kind::f16) or 8 events
// of 32-bit parts (kind::tf32); either way a row of one A or B part is 32 bytes.
template <int FORM>
struct Cfg {
    static constexpr bool TF32 = FORM >= FORM_TF32X3;
    static constexpr bool FP16 = FORM == FORM_FP16X3;
    static constexpr int CHUNK = TF32 ? 8 : 16;
    static constexpr uint32_t ABFMT = TF32 ? 2u : FP16 ? 0u : 1u;
};

// per-generator factor tables (rows padded so the A loop's reads hit distinct banks)
constexpr int XA_STRIDE = 20;       // floats per x row: 1 - u^2 for 16 events
constexpr int YB_STRIDE = 36;       // floats per y row: 1 - v^2, then v^2, for 16 events
constexpr uint32_t TAB_XA = 0;
constexpr uint32_t TAB_YB = TX * XA_STRIDE * 4;
constexpr uint32_t TAB_TK = TAB_YB + TY * YB_STRIDE * 4;
constexpr uint32_t TAB_BYTES = TAB_TK + 128;

// entry header flags
constexpr int F_MMA = 1;        // the stage holds operands for the MMA
constexpr int F_ITEM_END = 4;   // last entry of a tile
constexpr int F_TERM = 8;       // end of the stream's sequence
// page meta flags (written by the loader)
constexpr int P_ITEM_END = 4;
constexpr int P_TERM = 8;
// drain descriptor flags (MMA warp -> epilogue); the descriptor's fourth word
// holds the blocks touched since their last drain (bits 0-7), the blocks to
// drain (bits 8-15, all of them with D_LAST) and the blocks already stored
// (bits 16-23)
constexpr int D_LAST = 2, D_TERM = 4;

// roles
__device__ __forceinline__ int mma_stream(int w) { return w == 0 ? 0 : w == 8 ? 1 : -1; }
__device__ __forceinline__ int load_stream(int w) { return w == 4 ? 0 : w == 11 ? 1 : -1; }
// generator id: stream * NGEN + index within the stream (-1: not a generator)
__device__ __forceinline__ int gen_id(int w) {
    return (w >= 1 && w <= 3) ? w - 1 : w == 5 ? 3 : (w == 6 || w == 7) ? w - 2
         : (w == 9 || w == 10) ? w - 3 : -1;
}

struct L {
    static constexpr uint32_t OFF_STAGE = 0;
    static constexpr uint32_t OFF_PAGES = OFF_STAGE + NSTREAM * NSTAGE * STAGE_BYTES;
    static constexpr uint32_t OFF_TAB = OFF_PAGES + NSTREAM * NPAGES * PAGE * 16;
    static constexpr uint32_t OFF_HDR = OFF_TAB + NSTREAM * NGEN * TAB_BYTES;
    static constexpr uint32_t OFF_PMETA = OFF_HDR + NSTREAM * NSTAGE * 32;
    static constexpr uint32_t OFF_KEPT = OFF_PMETA + NSTREAM * NPAGES * 48;
    static constexpr uint32_t OFF_CTAB = OFF_KEPT + NSTREAM * NPAGES * 16;
    static constexpr uint32_t OFF_ENT = OFF_CTAB + NSTREAM * NPAGES * MAXCH * 8;
    static constexpr uint32_t OFF_DESC = OFF_ENT + NSTREAM * NPAGES * MAXENT * 2;
    static constexpr uint32_t OFF_BAR = OFF_DESC + NSTREAM * 16;
    static constexpr int BARS_PER_STREAM = 3 * NPAGES + 2 * NSTAGE + 4;
    static constexpr int NBARS = NSTREAM * BARS_PER_STREAM;
    static constexpr uint32_t OFF_MISC = OFF_BAR + NBARS * 8;  // tmem base, abort flag, wait bound
    static constexpr uint32_t TOTAL = OFF_MISC + 16;
    // barrier indices of stream p
    __host__ __device__ static constexpr int pfull(int p, int q) { return p * BARS_PER_STREAM + q; }
    __host__ __device__ static constexpr int pempty(int p, int q) { return p * BARS_PER_STREAM + NPAGES + q; }
    __host__ __device__ static constexpr int pfilt(int p, int q) { return p * BARS_PER_STREAM + 2 * NPAGES + q; }
    __host__ __device__ static constexpr int sfull(int p, int s) { return p * BARS_PER_STREAM + 3 * NPAGES + s; }
    __host__ __device__ static constexpr int sempty(int p, int s) {
        return p * BARS_PER_STREAM + 3 * NPAGES + NSTAGE + s;
    }
    __host__ __device__ static constexpr int afull(int p) { return p * BARS_PER_STREAM + 3 * NPAGES + 2 * NSTAGE; }
    __host__ __device__ static constexpr int aempty(int p) { return afull(p) + 1; }
    __host__ __device__ static constexpr int dfull(int p) { return afull(p) + 2; }
    __host__ __device__ static constexpr int drain(int p) { return afull(p) + 3; }
    static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
    static_assert(TAB_BYTES % 16 == 0 && OFF_PAGES % 16 == 0 && OFF_BAR % 8 == 0, "alignment");
    static_assert(TOTAL <= 227 * 1024, "shared memory budget");
    static_assert(NCAP % 16 == 0 && NCAP <= NB, "column window");
    static_assert(NSTREAM * NB <= 512, "tensor memory");
    // a generator's consecutive entries are NGEN apart; its stage waits stay at
    // most one barrier phase behind when NGEN <= NSTAGE
    static_assert(NGEN <= NSTAGE, "stage ring too short for the generators");
};

__device__ __forceinline__ float2 fneg2(float2 a) { return make_float2(-a.x, -a.y); }

template <typename T>
__device__ __forceinline__ uint32_t bits32(const T& v) {
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Two sign masks as one word: low 16 bits all ones if a < 0 (or -0), high 16
// bits all ones if b < 0 (prmt's sign-replicating byte select).
__device__ __forceinline__ uint32_t sign_mask2(float a, float b) {
    uint32_t m;
    asm("prmt.b32 %0, %1, %2, 0xFFBB;" : "=r"(m) : "r"(__float_as_uint(a)), "r"(__float_as_uint(b)));
    return m;
}

// hi = round-to-nearest 16-bit value of v, lo = rounded remainder, both packed
// (low half = v.x).
template <bool FP16>
__device__ __forceinline__ void split_rn(float2 v, uint32_t& hi, uint32_t& lo) {
    if constexpr (FP16) {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        const float2 r = __fadd2_rn(v, fneg2(__half22float2(h)));
        hi = bits32(h);
        lo = bits32(__floats2half2_rn(r.x, r.y));
    } else {
        const uint32_t h = bits32(__floats2bfloat162_rn(v.x, v.y));
        const float2 hf = make_float2(__uint_as_float(h << 16), __uint_as_float(h & 0xffff0000u));
        const float2 r = __fadd2_rn(v, fneg2(hf));
        hi = h;
        lo = bits32(__floats2bfloat162_rn(r.x, r.y));
    }
}

// hi = the value with its low 13 significand bits cleared (exact in tf32), lo =
// the remainder (exact in fp32), for a pair v; elements whose disk-test
// difference d is negative (or -0) give 0.
__device__ __forceinline__ void split_tf32(float2 v, float2 d, uint32_t& h0, uint32_t& h1, uint32_t& l0,
                                           uint32_t& l1) {
    const uint32_t m0 = (uint32_t)(__float_as_int(d.x) >> 31), m1 = (uint32_t)(__float_as_int(d.y) >> 31);
    const uint32_t a0 = __float_as_uint(v.x) & ~m0, a1 = __float_as_uint(v.y) & ~m1;
    h0 = a0 & 0xffffe000u;
    h1 = a1 & 0xffffe000u;
    const float2 r = __fadd2_rn(make_float2(__uint_as_float(a0), __uint_as_float(a1)),
                                make_float2(-__uint_as_float(h0), -__uint_as_float(h1)));
    l0 = __float_as_uint(r.x);
    l1 = __float_as_uint(r.y);
}

// The products of one entry, issued by one elected lane of a converged warp:
// D += Ahi*Bhi, D += Ahi*Blo, D += Alo*Bhi (kind::f16 or kind::tf32), or only
// D += Ahi*Bhi for the one-product form.
template <int FORM>
__device__ __forceinline__ void mma3_elect(uint32_t d, uint64_t ahi, uint64_t alo, uint64_t bhi,
                                           uint64_t blo, uint32_t idesc) {
    if constexpr (FORM == FORM_TF32X1) {
        asm volatile(
            "{\n\t.reg .pred e, acc;\n\t"
            "setp.ne.b32 acc, 1, 0;\n\t"
            "elect.sync _|e, 0xffffffff;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, acc;\n\t}"
            ::"r"(d), "l"(ahi), "l"(bhi), "r"(idesc)
            : "memory");
    } else if constexpr (FORM == FORM_TF32X3) {
        asm volatile(
            "{\n\t.reg .pred e, acc;\n\t"
            "setp.ne.b32 acc, 1, 0;\n\t"
            "elect.sync _|e, 0xffffffff;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %3, %5, acc;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %4, %5, acc;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %2, %3, %5, acc;\n\t}"
            ::"r"(d), "l"(ahi), "l"(alo), "l"(bhi), "l"(blo), "r"(idesc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred e, acc;\n\t"
            "setp.ne.b32 acc, 1, 0;\n\t"
            "elect.sync _|e, 0xffffffff;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %3, %5, acc;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %4, %5, acc;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %3, %5, acc;\n\t}"
            ::"r"(d), "l"(ahi), "l"(alo), "l"(bhi), "l"(blo), "r"(idesc)
            : "memory");
    }
}

// tcgen05.commit by one elected lane of a converged warp.
__device__ __forceinline__ void commit_elect(uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
        ::"r"(bar) : "memory");
}

struct Ctl {
    volatile int* abort;  // shared memory: the abort flag, then the wait bound (ns)
    int* err;
};

// The launch's bound on every wait, read only once a wait has spun a while.
__device__ __forceinline__ uint64_t wait_limit(const Ctl& c) {
    return *reinterpret_cast<const volatile uint64_t*>(c.abort + 1);
}

__device__ __forceinline__ bool timed_out(const Ctl& c, uint64_t t0) {
    if (ptx::globaltimer() - t0 > wait_limit(c)) {
        *c.abort = 1;
        atomicOr(c.err, ERRBIT_TIMEOUT);
        return true;
    }
    return false;
}

// Bounded wait for the phase of parity `parity` of barrier `bar`.  Returns
// false (and raises the abort flag) after the wait bound, or as soon as another role
// has aborted.
__device__ __forceinline__ bool wait_bar(const Ctl& c, uint32_t bar, uint32_t parity) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = ptx::globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*c.abort) return false;
            if (timed_out(c, t0)) return false;
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

// Tile `item` of problem P's launch: ty fastest, then tx within the launch's tile
// columns, then tb.
__device__ __forceinline__ void decode_item(const ProblemDev& P, int64_t item, int& tx, int& ty,
                                            int& tb) {
    const int ncx = P.ntxg > 0 ? P.ntxg : P.pl.ntx;
    ty = (int)(item % P.pl.nty);
    tx = P.tx0 + (int)((item / P.pl.nty) % ncx);
    tb = (int)(item / ((int64_t)P.pl.nty * ncx));
}

// Problem of batch tile g: the last problem whose first tile is <= g.
__device__ __forceinline__ int problem_of(const ProblemDev* __restrict__ table, int nprob, int64_t g) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (table[mid].item_base <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Problem p of the launch: the batch table's entry, or the single problem passed
// by value.
__device__ __forceinline__ ProblemDev fetch_problem(const ProblemDev& single,
                                                    const ProblemDev* __restrict__ table, int p) {
    return table ? table[p] : single;
}

template <int FORM, bool ADAPT>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tile_tc(ProblemDev single, const ProblemDev* __restrict__ table, int nprob,
          int* __restrict__ err, int* __restrict__ tile_ctr, const uint32_t* __restrict__ order,
          int64_t nitems, int flush_chunks, TcWait wc) {
    using C = Cfg<FORM>;
    constexpr int CHUNK = C::CHUNK;
    constexpr bool FP16 = C::FP16;
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t sb = ptx::smem_addr(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ctl c{reinterpret_cast<volatile int*>(smem + L::OFF_MISC + 4), err};
    auto bar = [sb](int i) -> uint32_t { return sb + L::OFF_BAR + 8u * (uint32_t)i; };
    int4* pmeta = reinterpret_cast<int4*>(smem + L::OFF_PMETA);   // [stream][page][3]
    int4* pkept = reinterpret_cast<int4*>(smem + L::OFF_KEPT);    // [stream][page]
    int2* ctab = reinterpret_cast<int2*>(smem + L::OFF_CTAB);     // [stream][page][chunk]
    uint16_t* pent = reinterpret_cast<uint16_t*>(smem + L::OFF_ENT);  // [stream][page][entry]

    if (threadIdx.x == 0) {
        for (int p = 0; p < NSTREAM; ++p) {
            for (int q = 0; q < NPAGES; ++q) {
                ptx::mbar_init(bar(L::pfull(p, q)), 1);
                ptx::mbar_init(bar(L::pempty(p, q)), NGEN);
                ptx::mbar_init(bar(L::pfilt(p, q)), 1);
            }
            for (int s = 0; s < NSTAGE; ++s) {
                ptx::mbar_init(bar(L::sfull(p, s)), 1);
                ptx::mbar_init(bar(L::sempty(p, s)), 1);
            }
            ptx::mbar_init(bar(L::afull(p)), 1);
            ptx::mbar_init(bar(L::aempty(p)), NEPI);
            ptx::mbar_init(bar(L::dfull(p)), 1);
            ptx::mbar_init(bar(L::drain(p)), 1);
        }
        *c.abort = 0;
        *reinterpret_cast<volatile uint64_t*>(smem + L::OFF_MISC + 8) = wc.wait_ns ? wc.wait_ns : WAIT_NS;
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(sb + L::OFF_MISC, NB * NSTREAM);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + L::OFF_MISC);
    const int gid = gen_id(warp);
    constexpr int PEV = ADAPT ? PAGE / 2 : PAGE;  // events per page

    if (load_stream(warp) >= 0) {
        // ------------------------------------------------------------ loader
        const int p = load_stream(warp);
        // test hook: block 0's first page of stream 0 never arrives
        const bool withhold = wc.withhold_page && blockIdx.x == 0 && p == 0;
        uint32_t pg = 0, fill = 0;
        bool open = false, ok = true;
        auto open_page = [&]() -> bool {
            if (!wait_warp(c, bar(L::pempty(p, pg % NPAGES)), ((pg / NPAGES) & 1u) ^ 1u)) return false;
            open = true;
            fill = 0;
            return true;
        };
        // Keeps the events of page fq (staged by this loader) whose cylinder
        // reaches their tile, compacted in place; records per chunk the covered
        // columns and the page's entry table; publishes the kept and entry counts.
        // The whole page is read into registers first (8 rounds of 32 events), so
        // the filter pays one shared-memory latency instead of one per round; the
        // chunks' column ranges are folded in with shared-memory min/max atomics.
        const uint32_t lt = (1u << lane) - 1u;
        auto filter_page = [&](uint32_t fq) {
            const uint32_t fp = p * NPAGES + fq % NPAGES;
            float4* fb = reinterpret_cast<float4*>(smem + L::OFF_PAGES + fp * PAGE_BYTES);
            float4* fbp = fb + PEV;  // per-event bandwidths (ADAPT)
            int2* ct = ctab + fp * MAXCH;
            uint16_t* ent = pent + fp * MAXENT;
            const int4 fm = pmeta[3 * fp], fmt4 = pmeta[3 * fp + 1];
            uint32_t kept = 0, nent = 0;
            if (!(fm.y & P_TERM)) {
                const Plan pl = fetch_problem(single, table, fmt4.w).pl;
                const TileGeom fg = tile_geom(pl, fmt4.x, fmt4.y, fmt4.z, NB);
                const int nev = fm.x, T0 = fg.T0, nbv = fg.T1 - fg.T0;
                constexpr int R = PEV / 32;
                float4 e[R], bw[R];
                uint32_t bal[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    e[r] = fb[r * 32 + lane];
                    if constexpr (ADAPT) bw[r] = fbp[r * 32 + lane];
                }
                if (lane < MAXCH) ct[lane] = make_int2(0x7fffffff, -1);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    bool in = r * 32 + lane < nev;
                    if constexpr (ADAPT) in = in && reaches_bw(fg, e[r], bw[r].x, bw[r].y);
                    else in = in && reaches(pl, fg, e[r]);
                    bal[r] = __ballot_sync(0xffffffffu, in);
                }
                __syncwarp();  // every read of the page before the first compacting write
                // columns covered by each chunk's windows, clipped into the block
                // (the filter's margin can keep an event whose window misses the
                // block; its K_t values are zero anyway)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if ((bal[r] >> lane) & 1u) {
                        const uint32_t at = kept + __popc(bal[r] & lt);
                        fb[at] = e[r];
                        if constexpr (ADAPT) fbp[at] = bw[r];
                        const float z = e[r].z;
                        const float htv = ADAPT ? bw[r].y : pl.htv;
                        const int lo = min(max((int)ceilf(z - 0.5f - htv) - T0, 0), nbv - 1);
                        const int hi = min(max((int)floorf(z - 0.5f + htv) - T0, lo), nbv - 1);
                        atomicMin(&ct[at / CHUNK].x, lo);
                        atomicMax(&ct[at / CHUNK].y, hi);
                    }
                    kept += __popc(bal[r]);
                }
                __syncwarp();
                const int nch = (int)(kept + CHUNK - 1) / CHUNK;
                // entries per chunk (column windows of up to NCAP) and their offsets
                uint32_t nw = 0;
                int2 t = make_int2(0, 0);
                if (lane < nch) {
                    const int2 mm = ct[lane];
                    t.x = (mm.x & ~15) | (((mm.y + 16) & ~15) << 16);
                    nw = (uint32_t)(((t.x >> 16) - (t.x & 0xffff) + NCAP - 1) / NCAP);
                }
                uint32_t incl = nw;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                // entry table: entry j of the page -> (chunk, window)
                if (lane < nch) {
                    t.y = (int)((incl - nw) | (nw << 16));
                    ct[lane] = t;
                    for (uint32_t w = 0; w < nw; ++w) ent[incl - nw + w] = (uint16_t)(lane | (w << 8));
                }
                nent = __shfl_sync(0xffffffffu, incl, 31);
                // a tile whose last page adds nothing still needs its end marker
                if (nent == 0 && (fm.y & P_ITEM_END)) {
                    nent = 1;
                    if (lane == 0) ent[0] = 0xffffu;
                }
            }
            // the compaction wrote the page: order it before the loader's next
            // bulk copy into the page
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                pkept[fp] = make_int4((int)kept, (int)nent, 0, 0);
                ptx::mbar_arrive(bar(L::pfilt(p, fq % NPAGES)));
            }
            __syncwarp();
        };
        // filters the page staged before the last one closed: its copies have had
        // the time of a page fill to land
        uint32_t nfilt = 0;  // pages filtered so far
        auto filter_upto = [&](uint32_t lim) -> bool {
            for (; nfilt < lim; ++nfilt) {
                if (!wait_warp(c, bar(L::pfull(p, nfilt % NPAGES)), (nfilt / NPAGES) & 1u)) return false;
                filter_page(nfilt);
            }
            return true;
        };
        // page meta: fill, flags, item, the item's tile coordinates and problem,
        // and the problem's reciprocal bandwidths and bandwidths
        auto close_page = [&](int flags, int64_t item, int tx, int ty, int tb, int pi, const Plan* ppl) {
            __syncwarp();
            if (lane == 0) {
                const uint32_t q = p * NPAGES + pg % NPAGES;
                pmeta[3 * q] = make_int4((int)fill, flags, (int)(item & 0xffffffff), (int)(item >> 32));
                pmeta[3 * q + 1] = make_int4(tx, ty, tb, pi);
                pmeta[3 * q + 2] = ppl ? make_int4(__float_as_int(ppl->inv_hs), __float_as_int(ppl->inv_ht),
                                                   __float_as_int(ppl->hsv), __float_as_int(ppl->htv))
                                       : make_int4(0, 0, 0, 0);
                if (!(withhold && pg == 0)) ptx::mbar_arrive(bar(L::pfull(p, pg % NPAGES)));
            }
            __syncwarp();
            ++pg;
            open = false;
            if (!(flags & P_TERM)) ok = ok && filter_upto(pg - 1);
        };
        while (ok) {
            // the next tile of the launch's global queue (heaviest first when ordered)
            int k = 0;
            if (lane == 0) {
                k = atomicAdd(tile_ctr, 1);
                if (order && k < nitems) k = (int)order[k];
            }
            const int64_t gk = (int64_t)__shfl_sync(0xffffffffu, k, 0);
            if (gk >= nitems) break;
            const int pi = table ? problem_of(table, nprob, gk) : 0;
            const ProblemDev P = fetch_problem(single, table, pi);
            const Plan& pl = P.pl;
            const float4* __restrict__ ev = P.ev;
            const float4* __restrict__ evp = P.evp;
            const uint32_t* __restrict__ start = P.start;
            const int64_t item = gk - P.item_base;  // tile of the problem
            int tx, ty, tb;
            decode_item(P, item, tx, ty, tb);
            // the bins of each bandwidth class around the tile, within the class's reach
            const int ncls = plan_classes(pl);
            for (int cls = 0; cls < ncls && ok; ++cls) {
            const TileGeom g = ncls == 1 ? tile_geom(pl, tx, ty, tb, NB)
                                         : tile_geom_r(pl, class_hsv(pl, cls), class_htv(pl, cls), tx, ty, tb, NB);
            const int ncx = g.cx_hi - g.cx_lo + 1;
            const int nr = (g.s_hi >= g.s_lo && ncx > 0) ? (g.s_hi - g.s_lo + 1) * ncx : 0;
            for (int r0 = 0; r0 < nr && ok; r0 += 32) {
                // 32 bin runs at a time: lane-parallel lengths, offsets by a warp scan
                uint32_t a = 0, len = 0;
                const int r = r0 + lane;
                if (r < nr) {
                    const int s = g.s_lo + r / ncx, cx = g.cx_lo + r % ncx;
                    const uint32_t kb = bin_row(pl, cls, s, cx);
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
                    const uint32_t q = p * NPAGES + pg % NPAGES;
                    const uint32_t take = min((uint32_t)PEV - fill, tot - done);
                    // this page takes pass positions [done, done + take); each lane copies
                    // the part of its own run that falls there
                    const uint32_t lo = max(off, done), hi = min(off + len, done + take);
                    if (hi > lo && !(withhold && pg == 0)) {
                        const uint32_t fb = bar(L::pfull(p, pg % NPAGES));
                        const uint32_t dst = sb + L::OFF_PAGES + q * PAGE_BYTES + (fill + (lo - done)) * 16u;
                        ptx::mbar_expect_tx(fb, (hi - lo) * (ADAPT ? 32u : 16u));
                        ptx::bulk_g2s(dst, ev + a + (lo - off), (hi - lo) * 16u, fb);
                        if constexpr (ADAPT)
                            ptx::bulk_g2s(dst + PEV * 16u, evp + a + (lo - off), (hi - lo) * 16u, fb);
                    }
                    fill += take;
                    done += take;
                    if (fill == (uint32_t)PEV) {
                        close_page(0, item, tx, ty, tb, pi, &pl);
                        if (!ok) break;  // a wait gave up: stage nothing more
                    }
                }
            }
            }
            if (!ok) break;
            if (!open && !(ok = open_page())) break;
            close_page(P_ITEM_END, item, tx, ty, tb, pi, &pl);  // the tile's last page, possibly empty
        }
        // termination page (every generator of the stream reads every page)
        if (ok) ok = filter_upto(pg);
        if (ok && (ok = open_page())) close_page(P_TERM, 0, 0, 0, 0, 0, nullptr);
        if (!ok) {
            if (open) close_page(P_TERM, 0, 0, 0, 0, 0, nullptr);
            for (uint32_t q = (pg > NPAGES ? pg - NPAGES : 0); q < pg; ++q)
                drain_bar(bar(L::pfull(p, q % NPAGES)), (q / NPAGES) & 1u);
        }
    } else if (gid >= 0) {
        // -------------------------------------------------------- generators
        const int p = gid / NGEN, gi = gid % NGEN;
        uint8_t* tab = smem + L::OFF_TAB + gid * TAB_BYTES;
        float* xa = reinterpret_cast<float*>(tab + TAB_XA);
        float* yb = reinterpret_cast<float*>(tab + TAB_YB);
        float* tkt = reinterpret_cast<float*>(tab + TAB_TK);
        float* tih = tkt + CHUNK;  // per-event 1/htv_i (ADAPT)
        const uint32_t fmt = C::ABFMT;
        bool ok = true;
        uint32_t ebase = 0;  // the stream's entries before the current page
        uint32_t emod = 0;   // ebase mod NGEN

        // waits until entry e's stage is free (its previous entry consumed)
        auto slot_wait = [&](uint32_t e) -> bool {
            const uint32_t use = e / NSTAGE;
            if (use == 0) return true;
            return wait_warp(c, bar(L::sempty(p, e % NSTAGE)), (use - 1u) & 1u);
        };
        // hands entry e to the stream's MMA warp, with what it needs precomputed:
        // the instruction descriptor, the 32-column blocks the MMAs touch and the
        // per-block chunk-count increments (bytes, four blocks per word)
        auto publish = [&](uint32_t e, int c0, int ncols, int flags, int64_t item, int pi) {
            const uint32_t s = e % NSTAGE;
            if (lane == 0) {
                uint32_t idesc = 0, mask = 0, inc_lo = 0, inc_hi = 0;
                if (flags & F_MMA) {
                    idesc = ptx::idesc_mma(128, (uint32_t)ncols, fmt);
                    const uint32_t b0 = (uint32_t)c0 >> 5, b1 = (uint32_t)(c0 + ncols - 1) >> 5;
                    mask = ((2u << b1) - 1u) & ~((1u << b0) - 1u);
                    inc_lo = ((mask & 15u) * 0x204081u) & 0x01010101u;
                    inc_hi = ((mask >> 4) * 0x204081u) & 0x01010101u;
                }
                int4* h = reinterpret_cast<int4*>(smem + L::OFF_HDR + (p * NSTAGE + s) * 32);
                h[0] = make_int4(c0, (int)idesc, flags, (int)mask);
                h[1] = make_int4((int)inc_lo, (int)inc_hi, (int)item, pi);
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(bar(L::sfull(p, s)));
        };
        for (uint32_t q = 0; ok; ++q) {
            const uint32_t pq = p * NPAGES + q % NPAGES;
            const uint32_t ph = (q / NPAGES) & 1u;
            const float4* page = reinterpret_cast<const float4*>(smem + L::OFF_PAGES + pq * PAGE_BYTES);
            if (!(ok = wait_warp(c, bar(L::pfull(p, q % NPAGES)), ph))) break;
            const int4 meta = pmeta[3 * pq], mt = pmeta[3 * pq + 1], mr = pmeta[3 * pq + 2];
            if (meta.y & P_TERM) {
                // the stream's sequence ends with entry ebase
                if (ebase % NGEN == (uint32_t)gi && (ok = slot_wait(ebase))) publish(ebase, 0, 0, F_TERM, 0, 0);
                break;
            }
            const int64_t item = (int64_t)(uint32_t)meta.z | ((int64_t)meta.w << 32);
            const int pi = mt.w;
            const float inv_hs = __int_as_float(mr.x), inv_ht = __int_as_float(mr.y);
            const float hs_max = __int_as_float(mr.z), ht_max = __int_as_float(mr.w);
            const int end = meta.y & P_ITEM_END;
            const int X0 = mt.x * TX, Y0 = mt.y * TY, T0 = mt.z * NB;
            if (!(ok = wait_warp(c, bar(L::pfilt(p, q % NPAGES)), ph))) break;
            const int4 ki = pkept[pq];
            const int kept = ki.x;
            const uint32_t nent = (uint32_t)ki.y;
            const int nch = (kept + CHUNK - 1) / CHUNK;
            const int2* ct = ctab + pq * MAXCH;
            const uint16_t* ent = pent + pq * MAXENT;
            // entry e is always built by generator e mod NGEN, so each generator's
            // entries are exactly NGEN apart and its stage waits are never more
            // than one barrier phase behind
            for (uint32_t j = ((uint32_t)gi + NGEN - emod) % NGEN; j < nent && ok; j += NGEN) {
                const uint32_t e = ebase + j;
                const uint32_t code = ent[j];
                if (code == 0xffffu) {
                    // end marker of a tile whose last page keeps nothing
                    if (!(ok = slot_wait(e))) break;
                    publish(e, 0, 0, F_ITEM_END, item, pi);
                    continue;
                }
                const int ch = (int)(code & 0xffu), w = (int)(code >> 8);
                const int2 cinfo = ct[ch];
                const int nw = cinfo.y >> 16;
                const int c0 = cinfo.x & 0xffff, cend = cinfo.x >> 16;
                const int count = min(CHUNK, kept - ch * CHUNK);

                // factor tables of K_s for the chunk's events (missing events get
                // u, v >= 2: negative factors, masked below); lane = (part, event)
                constexpr int NPART = 32 / CHUNK;
                const int k = lane % CHUNK, half = lane / CHUNK;
                const bool real = k < count;
                float4 ek = make_float4(0.f, 0.f, 0.f, 0.f);
                if (real) ek = page[ch * CHUNK + k];
                // the event's bandwidth reciprocals and weight (ADAPT), else the plan's
                float ihs = inv_hs, iht = inv_ht, wk = 1.0f;
                if constexpr (ADAPT) {
                    if (real) {
                        const float4 bk = page[PEV + ch * CHUNK + k];
                        ihs = bk.z;
                        iht = bk.w;
                        const float hr = hs_max * bk.z;
                        wk = hr * hr * (ht_max * bk.w);
                    }
                }
                const float cu = real ? ((float)X0 + 0.5f - ek.x) * ihs : 2.0f;
                const float cv = real ? ((float)Y0 + 0.5f - ek.y) * ihs : 2.0f;
#pragma unroll
                for (int i = 0; i < TX / NPART; ++i) {
                    const int x = half + NPART * i;
                    const float u = fmaf((float)x, ihs, cu);
                    if constexpr (ADAPT) xa[x * XA_STRIDE + k] = wk * fmaf(-u, u, 1.0f);
                    else xa[x * XA_STRIDE + k] = fmaf(-u, u, 1.0f);
                }
#pragma unroll
                for (int i = 0; i < TY / NPART; ++i) {
                    const int y = half + NPART * i;
                    const float v = fmaf((float)y, ihs, cv);
                    const float vv = v * v;
                    yb[y * YB_STRIDE + k] = 1.0f - vv;
                    if constexpr (ADAPT) yb[y * YB_STRIDE + 16 + k] = wk * vv;
                    else yb[y * YB_STRIDE + 16 + k] = vv;
                }
                const int cw = c0 + w * NCAP;
                const int ncols = min(NCAP, cend - cw);
                // event time relative to the window's first voxel centre
                if (lane < CHUNK) {
                    tkt[lane] = real ? ek.z - ((float)(T0 + cw) + 0.5f) : 1.0e9f;
                    if constexpr (ADAPT) tih[lane] = iht;
                }
                __syncwarp();
                if (!(ok = slot_wait(e))) break;
                uint8_t* st = smem + L::OFF_STAGE + (p * NSTAGE + e % NSTAGE) * STAGE_BYTES;

                // A = K_s without c_s: row r = voxel (x = r / 8, y = r % 8); lane
                // owns rows lane + 32 j, all with y = lane % 8.  The disk test
                // (u^2 + v^2 < 1, i.e. (1 - u^2) - v^2 > 0) masks both halves.
                // A row holds CHUNK events in 32 bytes: 16-bit parts packed in
                // pairs (kind::f16) or one 32-bit part per event (kind::tf32).
                {
                    constexpr int PP = CHUNK / 2;  // event pairs per row
                    const float* yrow = yb + (lane & 7) * YB_STRIDE;
                    float2 bq[PP], vq[PP];
#pragma unroll
                    for (int i = 0; i < PP / 2; ++i) {
                        const float4 tb4 = *reinterpret_cast<const float4*>(yrow + 4 * i);
                        const float4 tv4 = *reinterpret_cast<const float4*>(yrow + 16 + 4 * i);
                        bq[2 * i] = make_float2(tb4.x, tb4.y);
                        bq[2 * i + 1] = make_float2(tb4.z, tb4.w);
                        vq[2 * i] = make_float2(tv4.x, tv4.y);
                        vq[2 * i + 1] = make_float2(tv4.z, tv4.w);
                    }
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const float* xrow = xa + ((lane >> 3) + 4 * jj) * XA_STRIDE;
                        uint32_t ah[8], al[8];
#pragma unroll
                        for (int i = 0; i < PP / 2; ++i) {
                            const float4 t4 = *reinterpret_cast<const float4*>(xrow + 4 * i);
                            const float2 aq[2] = {make_float2(t4.x, t4.y), make_float2(t4.z, t4.w)};
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int pp = 2 * i + h;
                                const float2 pr = __fmul2_rn(aq[h], bq[pp]);
                                const float2 d = __fadd2_rn(aq[h], fneg2(vq[pp]));
                                if constexpr (C::TF32) {
                                    split_tf32(pr, d, ah[2 * pp], ah[2 * pp + 1], al[2 * pp], al[2 * pp + 1]);
                                } else {
                                    split_rn<FP16>(pr, ah[pp], al[pp]);
                                    const uint32_t m = sign_mask2(d.x, d.y);
                                    ah[pp] &= ~m;
                                    al[pp] &= ~m;
                                }
                            }
                        }
                        const int r = lane + 32 * jj;
                        const uint32_t off = (uint32_t)(r >> 3) * CORE_SBO + (uint32_t)(r & 7) * 16;
                        *reinterpret_cast<uint4*>(st + off) = make_uint4(ah[0], ah[1], ah[2], ah[3]);
                        *reinterpret_cast<uint4*>(st + off + CORE_LBO) = make_uint4(ah[4], ah[5], ah[6], ah[7]);
                        *reinterpret_cast<uint4*>(st + A_BYTES + off) = make_uint4(al[0], al[1], al[2], al[3]);
                        *reinterpret_cast<uint4*>(st + A_BYTES + off + CORE_LBO) =
                            make_uint4(al[4], al[5], al[6], al[7]);
                    }
                }
                // B = K_t without c_t: (1 - w^2)_+ for the window's columns
                {
                    constexpr int EH = CHUNK / 2;   // events of one core-matrix row (16 bytes)
                    // lanes 8h .. 8h + 7 of each 16 write events EH hh .. EH hh + EH - 1 of 8
                    // consecutive columns: 128 contiguous bytes per 8 lanes, no bank conflict
                    const int hh = (lane >> 3) & 1;
                    float2 tq[EH / 2], iq[EH / 2];
#pragma unroll
                    for (int i = 0; i < EH / 4; ++i) {
                        const float4 t4 = *reinterpret_cast<const float4*>(tkt + EH * hh + 4 * i);
                        tq[2 * i] = make_float2(-t4.x, -t4.y);
                        tq[2 * i + 1] = make_float2(-t4.z, -t4.w);
                        if constexpr (ADAPT) {
                            const float4 i4 = *reinterpret_cast<const float4*>(tih + EH * hh + 4 * i);
                            iq[2 * i] = make_float2(i4.x, i4.y);
                            iq[2 * i + 1] = make_float2(i4.z, i4.w);
                        }
                    }
                    const float2 ih2 = make_float2(inv_ht, inv_ht), one2 = make_float2(1.0f, 1.0f);
                    uint8_t* bh = st + 2 * A_BYTES;
                    uint8_t* bl = bh + B_BYTES;
                    // columns n0, n0 + 16, ... (ncols is a multiple of 16)
                    for (int n = ((lane >> 4) << 3) | (lane & 7); n < ncols; n += 16) {
                        const float2 n2 = make_float2((float)n, (float)n);
                        uint32_t h[4], l[4];
#pragma unroll
                        for (int i = 0; i < EH / 2; ++i) {
                            const float2 wv = __fmul2_rn(__fadd2_rn(n2, tq[i]), ADAPT ? iq[i] : ih2);
                            const float2 kt = __ffma2_rn(fneg2(wv), wv, one2);
                            const float2 kp = make_float2(fmaxf(kt.x, 0.0f), fmaxf(kt.y, 0.0f));
                            if constexpr (C::TF32) split_tf32(kp, kp, h[2 * i], h[2 * i + 1], l[2 * i], l[2 * i + 1]);
                            else split_rn<FP16>(kp, h[i], l[i]);
                        }
                        const uint32_t off = (uint32_t)(n >> 3) * CORE_SBO + (uint32_t)(n & 7) * 16 + hh * CORE_LBO;
                        *reinterpret_cast<uint4*>(bh + off) = make_uint4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<uint4*>(bl + off) = make_uint4(l[0], l[1], l[2], l[3]);
                    }
                }
                const int fl = F_MMA | ((end && ch == nch - 1 && w + 1 == nw) ? F_ITEM_END : 0);
                publish(e, cw, ncols, fl, item, pi);
            }
            if (!ok) break;
            // done with the page (only read here; the owner fenced its compaction)
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(bar(L::pempty(p, q % NPAGES)));
            ebase += nent;
            emod = (emod + nent) % NGEN;
        }
    } else if (mma_stream(warp) >= 0) {
        // --------------------------------------------------------------- MMA
        // The whole warp runs the loop (converged); one elected lane issues.
        const int p = mma_stream(warp);
        const uint32_t acc = tmem + (uint32_t)(p * NB);
        uint32_t nseg = 0;  // drains handed to the epilogue so far
        bool ok = true;
        // descriptors of the stream's stage 0; stage s adds s * STAGE_BYTES / 16
        const uint64_t d_ahi = ptx::smem_desc(sb + L::OFF_STAGE + p * NSTAGE * STAGE_BYTES, CORE_LBO, CORE_SBO);
        const uint64_t d_alo = d_ahi + (A_BYTES >> 4);
        const uint64_t d_bhi = d_ahi + ((2 * A_BYTES) >> 4);
        const uint64_t d_blo = d_ahi + ((2 * A_BYTES + B_BYTES) >> 4);
        // chunks per 32-column block at which the block is drained (a power of
        // two, at most 128), as a bit mask over the four byte counters of a word
        const uint32_t flush4 = (uint32_t)flush_chunks * 0x01010101u;
        const int4* hdr = reinterpret_cast<const int4*>(smem + L::OFF_HDR + p * NSTAGE * 32);
        int4* desc = reinterpret_cast<int4*>(smem + L::OFF_DESC + p * 16);
        uint32_t stored = 0;              // 32-column blocks of the tile already in global memory
        uint32_t touched = 0;             // 32-column blocks written since their last drain
        uint32_t cnt_lo = 0, cnt_hi = 0;  // chunks per 32-column block (bytes)
        // hands the blocks `drain` (all blocks with D_LAST) to the epilogue and
        // waits until they have been drained (this stream has one accumulator)
        auto close_segment = [&](int tile, int pi, int flags, uint32_t drain) -> bool {
            if (lane == 0) {
                *desc = make_int4(tile, pi, flags, (int)(touched | (drain << 8) | (stored << 16)));
                ptx::mbar_arrive(bar(L::dfull(p)));
            }
            __syncwarp();
            commit_elect(bar(L::afull(p)));
            ++nseg;
            if (flags & D_TERM) return true;
            if (!wait_warp(c, bar(L::aempty(p)), nseg & 1u)) return false;
            ptx::tc_fence_after();
            if (flags & D_LAST) {
                touched = 0;
                stored = 0;
                cnt_lo = 0;
                cnt_hi = 0;
            } else {
                stored |= drain;
                touched &= ~drain;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    if ((drain >> b) & 1u) cnt_lo &= ~(0xffu << (8 * b));
                    if ((drain >> (4 + b)) & 1u) cnt_hi &= ~(0xffu << (8 * b));
                }
            }
            return true;
        };
        ok = wait_warp(c, bar(L::aempty(p)), 0);
        ptx::tc_fence_after();
        for (uint32_t e = 0; ok; ++e) {
            const uint32_t s = e % NSTAGE;
            if (!(ok = wait_warp(c, bar(L::sfull(p, s)), (e / NSTAGE) & 1u))) break;
            ptx::tc_fence_after();
            const int4 h0 = hdr[2 * s], h1 = hdr[2 * s + 1];
            const int flags = h0.z;
            if (flags & F_TERM) {
                close_segment(0, 0, D_TERM, 0);
                break;
            }
            const int tile = h1.z, pi = h1.w;
            if (flags & F_MMA) {
                const int c0 = h0.x;
                const uint32_t idesc = (uint32_t)h0.y;
                const int ncols = (int)((idesc >> 17) & 0x3Fu) << 3;
                // never issue an MMA outside the accumulator
                const bool in_range = c0 >= 0 && c0 + ncols <= NB && ncols >= 16 && ncols <= NCAP &&
                                      ((c0 | ncols) & 15) == 0;
                if (!in_range) {
                    if (lane == 0) atomicOr(err, ERRBIT_BOUNDS);
                } else {
                    const uint32_t inc_lo = (uint32_t)h1.x, inc_hi = (uint32_t)h1.y;
                    // a byte (chunk count of one 32-column block) reaching the
                    // power-of-two flush count drains that block first
                    const uint32_t ov_lo = (cnt_lo + inc_lo) & flush4, ov_hi = (cnt_hi + inc_hi) & flush4;
                    if (ov_lo | ov_hi) {
                        // drain just the blocks that reached the flush count
                        uint32_t drain = 0;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            if ((ov_lo >> (8 * b)) & 0xffu) drain |= 1u << b;
                            if ((ov_hi >> (8 * b)) & 0xffu) drain |= 1u << (4 + b);
                        }
                        if (!(ok = close_segment(tile, pi, 0, drain))) break;
                    }
                    cnt_lo += inc_lo;
                    cnt_hi += inc_hi;
                    touched |= (uint32_t)h0.w;
                    const uint64_t so = (uint64_t)s * (STAGE_BYTES >> 4);
                    mma3_elect<FORM>(acc + (uint32_t)c0, d_ahi + so, d_alo + so, d_bhi + so, d_blo + so, idesc);
                }
            }
            if (flags & F_ITEM_END) {
                if (!(ok = close_segment(tile, pi, D_LAST, 0xffu))) break;
            }
            commit_elect(bar(L::sempty(p, s)));
        }
        // every MMA issued has completed before the accumulator is released
        commit_elect(bar(L::drain(p)));
        drain_bar(bar(L::drain(p)), 0);
        __syncwarp();
    } else if (warp >= WARP_EPI0) {
        // ---------------------------------------------------------- epilogue
        const int qtr = warp & 3;
        const uint32_t trow = tmem + ((uint32_t)(32 * qtr) << 16);
        for (int col = 0; col < NB * NSTREAM; col += 32) ptx::tmem_st32_zero(trow + (uint32_t)col);
        ptx::tmem_wait_st();
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0)
            for (int p = 0; p < NSTREAM; ++p) ptx::mbar_arrive(bar(L::aempty(p)));
        bool ok = true;
        uint32_t seg[NSTREAM] = {0, 0};
        bool done[NSTREAM] = {false, false};
        while (ok && !(done[0] && done[1])) {
            // the next segment of whichever stream has one ready (lane 0 picks)
            int p = -1;
            if (lane == 0) {
                const uint64_t t0 = ptx::globaltimer();
                for (uint32_t it = 0; p < 0; ++it) {
                    for (int s = 0; s < NSTREAM && p < 0; ++s)
                        if (!done[s] && ptx::mbar_try_wait_ns(bar(L::dfull(s)), seg[s] & 1u, 400)) p = s;
                    if (p < 0 && (it & 7) == 7 && (*c.abort || timed_out(c, t0))) break;
                }
            }
            p = __shfl_sync(0xffffffffu, p, 0);
            if (p < 0) break;
            if (!(ok = wait_warp(c, bar(L::dfull(p)), seg[p] & 1u))) break;
            if (!(ok = wait_warp(c, bar(L::afull(p)), seg[p] & 1u))) break;
            ptx::tc_fence_after();
            const int4 dsc = ptx::lds_i4(sb + L::OFF_DESC + p * 16);
            ++seg[p];
            if (dsc.z & D_TERM) {
                done[p] = true;
                continue;
            }
            const int64_t item = dsc.x;
            const ProblemDev P = fetch_problem(single, table, dsc.y);
            const Plan& pl = P.pl;
            float* __restrict__ out = P.out;
            // float4 loads and stores need every voxel column 16-byte aligned
            const bool vec = (pl.gt & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
            // A and B carry neither c_s nor c_t: both join the normalisation here
            const float scale = pl.norm * (pl.cs * pl.ct);
            const bool last = (dsc.z & D_LAST) != 0;
            const uint32_t touched = (uint32_t)dsc.w & 0xffu, drain = ((uint32_t)dsc.w >> 8) & 0xffu;
            const uint32_t stored = ((uint32_t)dsc.w >> 16) & 0xffu;
            int tx, ty, tb;
            decode_item(P, item, tx, ty, tb);
            const int m = 32 * qtr + lane;
            const int X = tx * TX + m / TY, Y = ty * TY + m % TY, T0 = tb * NB;
            const int nbv = min(NB, pl.gt - T0);
            const bool valid = X < pl.gx && Y < pl.gy;
            float* dst = out + ((int64_t)X * pl.gy + Y) * (int64_t)pl.gt + T0;
            for (int col = 0; col < nbv; col += 32) {
                const int bk = col >> 5;
                const bool hit = (touched >> bk) & 1u;
                const bool first = !((stored >> bk) & 1u);
                if (!(last || ((drain >> bk) & 1u))) continue;
                if (!first && !hit) continue;
                uint32_t r[32];
                const uint32_t ta = trow + (uint32_t)(p * NB + col);
                const int nv = min(32, nbv - col);
                float4* p4 = reinterpret_cast<float4*>(dst + col);
                float4 pv[8];
                // earlier drains of this block: their sums are read back while the
                // tensor-memory load is in flight
                if (valid && vec && nv == 32 && !first) {
#pragma unroll
                    for (int v4 = 0; v4 < 8; ++v4) pv[v4] = p4[v4];
                }
                ptx::tmem_ld32(ta, r);
                ptx::tmem_wait_ld();
                if (hit) ptx::tmem_st32_zero(ta);
                if (!valid) continue;
                if (vec && nv == 32) {
#pragma unroll
                    for (int v4 = 0; v4 < 8; ++v4) {
                        float4 o = make_float4(__uint_as_float(r[4 * v4]) * scale,
                                               __uint_as_float(r[4 * v4 + 1]) * scale,
                                               __uint_as_float(r[4 * v4 + 2]) * scale,
                                               __uint_as_float(r[4 * v4 + 3]) * scale);
                        if (!first) {
                            o.x += pv[v4].x; o.y += pv[v4].y; o.z += pv[v4].z; o.w += pv[v4].w;
                        }
                        if (last) __stcs(p4 + v4, o); else p4[v4] = o;
                    }
                } else {
#pragma unroll
                    for (int jx = 0; jx < 32; ++jx) {
                        if (jx < nv) {
                            float o = __uint_as_float(r[jx]) * scale;
                            if (!first) o += dst[col + jx];
                            dst[col + jx] = o;
                        }
                    }
                }
            }
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(bar(L::aempty(p)));
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, NB * NSTREAM);
    }
}

// Tile ordering, heaviest first (an LPT schedule for the tile queue: the
// clustered workloads' tiles differ in cost by orders of magnitude, and a heavy
// tile started last sets the kernel's tail).  Cost of a tile = events in its bin
// neighbourhood; tiles are bucketed by floor(log2(cost + 1)), buckets in
// descending order; the order inside a bucket does not matter (each tile is
// computed independently and deterministically).
constexpr int NBUCKET = 33;

__global__ void k_tile_cost(ProblemDev single, const ProblemDev* __restrict__ table, int nprob,
                            int nitems, uint32_t* __restrict__ cost, uint32_t* __restrict__ hist) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nitems) return;
    const ProblemDev P = fetch_problem(single, table, table ? problem_of(table, nprob, i) : 0);
    const Plan& pl = P.pl;
    const uint32_t* __restrict__ start = P.start;
    int tx, ty, tb;
    decode_item(P, i - P.item_base, tx, ty, tb);
    uint32_t sum = 0;
    const int ncls = plan_classes(pl);
    for (int cls = 0; cls < ncls; ++cls) {
        const TileGeom g = ncls == 1 ? tile_geom(pl, tx, ty, tb, NB)
                                     : tile_geom_r(pl, class_hsv(pl, cls), class_htv(pl, cls), tx, ty, tb, NB);
        for (int s = g.s_lo; s <= g.s_hi; ++s)
            for (int cx = g.cx_lo; cx <= g.cx_hi; ++cx) {
                const uint32_t kb = bin_row(pl, cls, s, cx);
                sum += start[kb + g.cy_hi + 1] - start[kb + g.cy_lo];
            }
    }
    cost[i] = sum;
    atomicAdd(&hist[32 - __clz(sum)], 1u);
}

__global__ void k_tile_order(int nitems, const uint32_t* __restrict__ cost,
                             const uint32_t* __restrict__ hist, uint32_t* __restrict__ cursor,
                             uint32_t* __restrict__ order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nitems) return;
    const int b = 32 - __clz(cost[i]);
    uint32_t base = 0;
    for (int h = NBUCKET - 1; h > b; --h) base += hist[h];
    order[base + atomicAdd(&cursor[b], 1u)] = (uint32_t)i;
}

template <int FORM, bool ADAPT>
bool launch_cfg(const ProblemDev& single, const ProblemDev* table, int nprob, int64_t items,
                int* err, int* tile_ctr, uint32_t* order_ws, cudaStream_t st, TcWait wc) {
    auto kern = k_tile_tc<FORM, ADAPT>;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    // the shared-memory limit is raised once per device this process uses
    // (a function attribute per device and form; setting it again is harmless,
    // so host threads that race here at worst set it twice)
    constexpr int MAXDEV = 64;
    static std::atomic<bool> attr[MAXDEV];
    if (dev < 0 || dev >= MAXDEV) return false;
    if (!attr[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::TOTAL) !=
            cudaSuccess)
            return false;
        attr[dev].store(true, std::memory_order_release);
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (items <= 0) return true;
    if (items >= (int64_t)1 << 31) return false;  // the tile queue counts in int
    const int grid = (int)(items < sms ? items : sms);
    if (cudaMemsetAsync(tile_ctr, 0, sizeof(int), st) != cudaSuccess) return false;
    const uint32_t* order = nullptr;
    if (order_ws) {
        uint32_t* hist = order_ws;
        uint32_t* cursor = order_ws + 64;
        uint32_t* cost = order_ws + 128;
        uint32_t* ord = cost + items;
        if (cudaMemsetAsync(order_ws, 0, 128 * sizeof(uint32_t), st) != cudaSuccess) return false;
        const int blocks = (int)((items + 255) / 256);
        k_tile_cost<<<blocks, 256, 0, st>>>(single, table, nprob, (int)items, cost, hist);
        k_tile_order<<<blocks, 256, 0, st>>>((int)items, cost, hist, cursor, ord);
        order = ord;
    }
    // chunks (K steps, three accumulation steps each) per 32-column block at
    // which the block is drained (a power of two: the MMA warp tests it as a bit
    // mask): bounds the round-toward-zero drift of the tensor-core accumulation
    // per drain.  kind::tf32 takes twice the K steps per event and drifts more
    // per step.
    const int flush_chunks = FORM == FORM_FP16X3 ? 64 : FORM == FORM_TF32X3 ? 32 : 128;
    kern<<<grid, NTHREADS, L::TOTAL, st>>>(single, table, nprob, err, tile_ctr, order, items,
                                           flush_chunks, wc);
    return true;
}

}  // namespace

int64_t tile_tc_items(const Plan& pl) {
    return (int64_t)pl.ntx * pl.nty * ((pl.gt + NB - 1) / NB);
}

size_t tile_order_bytes_items(int64_t items) {
    return sizeof(uint32_t) * (128 + 2 * (size_t)(items > 0 ? items : 0));
}

size_t tile_order_bytes(const Plan& pl) { return tile_order_bytes_items(tile_tc_items(pl)); }

// The kernel of form `form` (0 bf16x3, 1 fp16x3, 2 tf32x3, 3 tf32x1; per-event
// bandwidths with the 16-bit forms only).
template <bool ADAPT>
bool launch_form(int form, const ProblemDev& single, const ProblemDev* table, int nprob, int64_t items,
                 int* err, int* tile_ctr, uint32_t* order_ws, cudaStream_t st, TcWait wc) {
    switch (form) {
        case FORM_BF16X3:
            return launch_cfg<FORM_BF16X3, ADAPT>(single, table, nprob, items, err, tile_ctr, order_ws, st, wc);
        case FORM_FP16X3:
            return launch_cfg<FORM_FP16X3, ADAPT>(single, table, nprob, items, err, tile_ctr, order_ws, st, wc);
        default:
            break;
    }
    if constexpr (!ADAPT) {
        if (form == FORM_TF32X3)
            return launch_cfg<FORM_TF32X3, false>(single, table, nprob, items, err, tile_ctr, order_ws, st, wc);
        if (form == FORM_TF32X1)
            return launch_cfg<FORM_TF32X1, false>(single, table, nprob, items, err, tile_ctr, order_ws, st, wc);
    }
    return false;
}

bool launch_tile_tc(const Plan& pl, const Bins& b, float* out, int* err, int* tile_ctr,
                    uint32_t* order_ws, int form, cudaStream_t st, int tx0, int ntxg, TcWait wc) {
    ProblemDev single{};
    single.pl = pl;
    single.ev = b.ev;
    single.start = b.start;
    single.out = out;
    single.item_base = 0;
    single.evp = b.evp;
    single.tx0 = tx0;
    single.ntxg = ntxg;
    const int64_t items = ntxg > 0 ? tile_tc_items(pl) / pl.ntx * ntxg : tile_tc_items(pl);
    if (b.evp) return launch_form<true>(form, single, nullptr, 1, items, err, tile_ctr, order_ws, st, wc);
    return launch_form<false>(form, single, nullptr, 1, items, err, tile_ctr, order_ws, st, wc);
}

bool launch_tile_tc_batch(const ProblemDev* table, int nprob, int64_t total_items, int* err,
                          int* tile_ctr, uint32_t* order_ws, int form, cudaStream_t st, TcWait wc) {
    if (nprob <= 0) return true;
    const ProblemDev none{};
    return launch_form<false>(form, none, table, nprob, total_items, err, tile_ctr, order_ws, st, wc);
}

}  // namespace stkde
