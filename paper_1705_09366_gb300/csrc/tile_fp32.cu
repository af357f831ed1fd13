// K4: fp32 CUDA-core tile kernel.
//
// PB-SYM (Section 3.2, Algorithm 3) evaluated owner-computes: one CTA owns an
// output tile of 16 x 8 voxels in the plane by 64 voxels of T and is the only
// writer of those voxels, so no atomics are needed and every voxel sums its
// events in one fixed order (the bin order), which makes the result
// bit-reproducible.  The CTA walks the event bins around the tile (the
// subdomain assignment of Algorithm 5, done by reading neighbouring bins instead
// of replicating events) and keeps the events whose cylinder reaches the tile.
// For each batch of kept events it tabulates both invariants in shared memory:
// the spatial invariant K_s of every event at each of the tile's 128 voxels
// (the disk, zero outside it) and the temporal invariant K_t over the tile's 64
// voxels of T (the bar).  Then the outer product is accumulated register-blocked:
// warp w owns T voxels 8w .. 8w + 7 and lane l owns voxels 4l .. 4l + 3, so per
// event a lane loads 4 K_s values and 8 K_t values (a broadcast) and issues 32
// multiply-adds as 16 paired FMAs; a warp skips the events whose bar misses its
// 8 voxels of T.  Each voxel is written once, zeros included, so the grid needs
// no separate initialisation (the Theta(G) init of Algorithm 2 becomes part of
// the store stream).
//
// With per-event bandwidths (ADAPT) each kept event also carries (hsv_i, htv_i,
// 1/hsv_i, 1/htv_i): its reach test, T window and K_s, K_t use its own
// bandwidths, and its K_t row is weighted by (hs_max/hs_i)^2 (ht_max/ht_i), the
// plan holding the largest bandwidths and the matching normalisation.
#include "internal.cuh"
#include "tile_common.cuh"

#include <atomic>

namespace stkde {

namespace {

constexpr int F_THREADS = 256;   // 8 warps
constexpr int F_TB = 64;         // voxels of T per tile
constexpr int F_TW = 8;          // voxels of T per warp
constexpr int F_VL = 4;          // voxels of the plane per lane
constexpr int F_BATCH = 64;      // events per table batch
constexpr int F_BUF = F_BATCH + F_THREADS;

static_assert(F_TW * (F_THREADS / 32) == F_TB, "warps tile the T block");
static_assert(F_VL * 32 == TILE_XY, "lanes tile the plane");

// dynamic shared memory: candidate events (and their bandwidths), K_s table
// [batch][voxel], K_t table [batch][T], bar windows
template <bool ADAPT>
struct FL {
    static constexpr size_t BUF = 0;
    static constexpr size_t BUFP = BUF + 16 * F_BUF;
    static constexpr size_t KS = BUFP + (ADAPT ? 16 * F_BUF : 0);
    static constexpr size_t KT = KS + 4 * F_BATCH * TILE_XY;
    static constexpr size_t WIN = KT + 4 * F_BATCH * F_TB;
    static constexpr size_t TOTAL = WIN + 8 * F_BATCH;
};

// With BATCH, block b computes tile b of the batch's fp32 tile numbering: the
// problem is the last table entry whose fitem_base is <= b, and its plan, bins
// and output replace the arguments.
template <bool ADAPT, bool BATCH>
__global__ void __launch_bounds__(F_THREADS, 3)
k_tile_fp32(Plan pl, const float4* __restrict__ ev, const float4* __restrict__ evp,
            const uint32_t* __restrict__ start, float* __restrict__ out,
            const ProblemDev* __restrict__ table, int nprob) {
    using L = FL<ADAPT>;
    extern __shared__ __align__(16) uint8_t fsm[];
    float4* buf = reinterpret_cast<float4*>(fsm + L::BUF);
    float4* bufp = reinterpret_cast<float4*>(fsm + L::BUFP);
    float* kst = reinterpret_cast<float*>(fsm + L::KS);    // [F_BATCH][TILE_XY]
    float* ktt = reinterpret_cast<float*>(fsm + L::KT);    // [F_BATCH][F_TB]
    int2* win = reinterpret_cast<int2*>(fsm + L::WIN);
    __shared__ int wcount[F_THREADS / 32];
    __shared__ int s_count;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t item = blockIdx.x;
    if constexpr (BATCH) {
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (table[mid].fitem_base <= item) lo = mid; else hi = mid - 1;
        }
        const ProblemDev& P = table[lo];
        pl = P.pl;
        pl.tblock = F_TB;
        pl.ntb = (pl.gt + F_TB - 1) / F_TB;
        ev = P.ev;
        start = P.start;
        out = P.out;
        item -= P.fitem_base;
    }
    const int ty = (int)(item % pl.nty);
    const int tx = (int)((item / pl.nty) % pl.ntx);
    const int tb = (int)(item / ((int64_t)pl.nty * pl.ntx));
    const TileGeom g = tile_geom(pl, tx, ty, tb, F_TB);
    const int c0 = warp * F_TW;  // this warp's T voxels: T0 + c0 .. T0 + c0 + 7

    // acc[v][h] = (T c0 + 2h, c0 + 2h + 1) of voxel 4 lane + v
    float2 acc[F_VL][F_TW / 2];
#pragma unroll
    for (int v = 0; v < F_VL; ++v)
#pragma unroll
        for (int h = 0; h < F_TW / 2; ++h) acc[v][h] = make_float2(0.0f, 0.0f);

    if (tid == 0) s_count = 0;
    __syncthreads();

    // Adds the events buf[off, off+cnt) into the accumulators.
    auto process = [&](int off, int cnt) {
        // K_s[j][m] for voxel m = x * TY + y of the tile (c_s and, with ADAPT, nothing else)
        for (int q = tid; q < cnt * TILE_XY; q += F_THREADS) {
            const int j = q / TILE_XY, m = q % TILE_XY;
            const float4 e = buf[off + j];
            const float ihs = ADAPT ? bufp[off + j].z : pl.inv_hs;
            const float u = ((float)(g.X0 + m / TY) + 0.5f - e.x) * ihs;
            const float v = ((float)(g.Y0 + m % TY) + 0.5f - e.y) * ihs;
            const float s = fmaf(u, u, v * v);
            kst[j * TILE_XY + m] = s < 1.0f ? pl.cs * fmaf(-u, u, 1.0f) * fmaf(-v, v, 1.0f) : 0.0f;
        }
        // K_t[j][c] over the tile's T block (with ADAPT weighted by (hs_max/hs_i)^2 (ht_max/ht_i))
        for (int q = tid; q < cnt * F_TB; q += F_THREADS) {
            const int j = q / F_TB, c = q % F_TB;
            if constexpr (ADAPT) {
                const float4 b = bufp[off + j];
                const float hr = pl.hsv * b.z;
                const float w = ((float)(g.T0 + c) + 0.5f - buf[off + j].z) * b.w;
                ktt[j * F_TB + c] = (pl.ct * (hr * hr * (pl.htv * b.w))) * fmaxf(fmaf(-w, w, 1.0f), 0.0f);
            } else {
                const float w = ((float)(g.T0 + c) + 0.5f - buf[off + j].z) * pl.inv_ht;
                ktt[j * F_TB + c] = pl.ct * fmaxf(fmaf(-w, w, 1.0f), 0.0f);
            }
        }
        // the bar's columns relative to T0, widened by one (a superset)
        for (int j = tid; j < cnt; j += F_THREADS) {
            const float pt = buf[off + j].z;
            const float htv = ADAPT ? bufp[off + j].y : pl.htv;
            win[j] = make_int2((int)floorf(pt - 0.5f - htv) - g.T0 - 1,
                               (int)ceilf(pt - 0.5f + htv) - g.T0 + 1);
        }
        __syncthreads();
        const float4* ks4 = reinterpret_cast<const float4*>(kst) + lane;
        const float4* kt4 = reinterpret_cast<const float4*>(ktt) + c0 / 4;
        for (int j = 0; j < cnt; ++j) {
            const int2 wj = win[j];
            if (wj.x > c0 + F_TW - 1 || wj.y < c0) continue;  // the bar misses this warp's T
            const float4 ks = ks4[j * (TILE_XY / 4)];
            const float4 ka = kt4[j * (F_TB / 4)], kb = kt4[j * (F_TB / 4) + 1];
            const float2 kt[F_TW / 2] = {make_float2(ka.x, ka.y), make_float2(ka.z, ka.w),
                                         make_float2(kb.x, kb.y), make_float2(kb.z, kb.w)};
            const float kv[F_VL] = {ks.x, ks.y, ks.z, ks.w};
#pragma unroll
            for (int v = 0; v < F_VL; ++v) {
                const float2 a2 = make_float2(kv[v], kv[v]);
#pragma unroll
                for (int h = 0; h < F_TW / 2; ++h) acc[v][h] = __ffma2_rn(a2, kt[h], acc[v][h]);
            }
        }
        __syncthreads();
    };

    const uint32_t lt = (1u << lane) - 1u;
    const int ncls = plan_classes(pl);
    for (int cls = 0; cls < ncls; ++cls) {
    // the bins of bandwidth class cls around the tile, within the class's reach
    const TileGeom gc = ncls == 1 ? g : tile_geom_r(pl, class_hsv(pl, cls), class_htv(pl, cls), tx, ty, tb, F_TB);
    for (int s = gc.s_lo; s <= gc.s_hi; ++s) {
        for (int cx = gc.cx_lo; cx <= gc.cx_hi; ++cx) {
            const uint32_t kb = bin_row(pl, cls, s, cx);
            const int a = (int)start[kb + gc.cy_lo];
            const int b = (int)start[kb + gc.cy_hi + 1];
            for (int base = a; base < b; base += F_THREADS) {
                const int p = base + tid;
                float4 e = make_float4(0.f, 0.f, 0.f, 0.f), bw = e;
                bool keep = false;
                if (p < b) {
                    e = ev[p];
                    if constexpr (ADAPT) {
                        bw = evp[p];
                        keep = reaches_bw(g, e, bw.x, bw.y);
                    } else {
                        keep = reaches(pl, g, e);
                    }
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) wcount[warp] = __popc(bal);
                __syncthreads();
                int pre = s_count, tot = 0;
#pragma unroll
                for (int w = 0; w < F_THREADS / 32; ++w) {
                    const int c = wcount[w];
                    pre += w < warp ? c : 0;
                    tot += c;
                }
                if (keep) {
                    buf[pre + __popc(bal & lt)] = e;
                    if constexpr (ADAPT) bufp[pre + __popc(bal & lt)] = bw;
                }
                const int cnt = s_count + tot;
                __syncthreads();
                if (tid == 0) s_count = cnt;
                if (cnt >= F_BATCH) {
                    const int full = (cnt / F_BATCH) * F_BATCH;
                    for (int off = 0; off < full; off += F_BATCH) process(off, F_BATCH);
                    const int rem = cnt - full;  // < F_BATCH <= full: no overlap
                    for (int q = tid; q < rem; q += F_THREADS) {
                        buf[q] = buf[full + q];
                        if constexpr (ADAPT) bufp[q] = bufp[full + q];
                    }
                    if (tid == 0) s_count = rem;
                }
                __syncthreads();
            }
        }
    }
    }
    const int rem = s_count;
    if (rem > 0) process(0, rem);

    // each lane writes its 4 voxels x 8 voxels of T, scaled by 1/(n hs^2 ht)
    const int Tb = g.T0 + c0;
    const int nvalid = min(F_TW, pl.gt - Tb);
    if (nvalid <= 0) return;
#pragma unroll
    for (int v = 0; v < F_VL; ++v) {
        const int m = F_VL * lane + v;
        const int X = g.X0 + m / TY, Y = g.Y0 + m % TY;
        if (X >= pl.gx || Y >= pl.gy) continue;
        float* dst = out + ((int64_t)X * pl.gy + Y) * (int64_t)pl.gt + Tb;
        float o[F_TW];
#pragma unroll
        for (int h = 0; h < F_TW / 2; ++h) {
            o[2 * h] = acc[v][h].x * pl.norm;
            o[2 * h + 1] = acc[v][h].y * pl.norm;
        }
        if (nvalid == F_TW && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
            __stcs(reinterpret_cast<float4*>(dst), make_float4(o[0], o[1], o[2], o[3]));
            __stcs(reinterpret_cast<float4*>(dst) + 1, make_float4(o[4], o[5], o[6], o[7]));
        } else {
#pragma unroll
            for (int c = 0; c < F_TW; ++c)
                if (c < nvalid) dst[c] = o[c];
        }
    }
}

// The dynamic shared-memory limit of each instantiation is raised once per
// device (setting it again is harmless).
template <bool ADAPT, bool BATCH>
bool prepare() {
    constexpr int MAXDEV = 64;
    static std::atomic<bool> done[MAXDEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return false;
    if (!done[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(k_tile_fp32<ADAPT, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FL<ADAPT>::TOTAL) != cudaSuccess)
            return false;
        done[dev].store(true, std::memory_order_release);
    }
    return true;
}

}  // namespace

bool launch_tile_fp32(const Plan& pl, const Bins& b, float* out, int* err, cudaStream_t st) {
    (void)err;
    Plan p = pl;
    p.tblock = F_TB;
    p.ntb = (pl.gt + F_TB - 1) / F_TB;
    const int64_t items = (int64_t)p.ntx * p.nty * p.ntb;
    if (items <= 0) return true;
    if (items >= ((int64_t)1 << 31)) return false;
    if (b.evp) {
        if (!prepare<true, false>()) return false;
        k_tile_fp32<true, false><<<(unsigned)items, F_THREADS, FL<true>::TOTAL, st>>>(
            p, b.ev, b.evp, b.start, out, nullptr, 0);
    } else {
        if (!prepare<false, false>()) return false;
        k_tile_fp32<false, false><<<(unsigned)items, F_THREADS, FL<false>::TOTAL, st>>>(
            p, b.ev, nullptr, b.start, out, nullptr, 0);
    }
    return true;
}

int64_t tile_fp32_items(const Plan& pl) {
    return (int64_t)pl.ntx * pl.nty * ((pl.gt + F_TB - 1) / F_TB);
}

bool launch_tile_fp32_batch(const ProblemDev* table, int nprob, int64_t total_items, cudaStream_t st) {
    if (nprob <= 0 || total_items <= 0) return true;
    if (total_items >= ((int64_t)1 << 31)) return false;
    if (!prepare<false, true>()) return false;
    k_tile_fp32<false, true><<<(unsigned)total_items, F_THREADS, FL<false>::TOTAL, st>>>(
        Plan{}, nullptr, nullptr, nullptr, nullptr, table, nprob);
    return true;
}

}  // namespace stkde
