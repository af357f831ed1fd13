// K4: fp32 CUDA-core tile kernel.
//
// PB-SYM (Section 3.2, Algorithm 3) evaluated owner-computes: one CTA owns an
// output tile of 16 x 8 voxels in the plane by 64 voxels of T and is the only
// writer of those voxels, so no atomics are needed and every voxel sums its
// events in one fixed order (the bin order), which makes the result
// bit-reproducible.  The CTA walks the event bins around the tile (the
// subdomain assignment of Algorithm 5, done by reading neighbouring bins instead
// of replicating events), keeps the events whose cylinder reaches the tile,
// builds each kept event's temporal invariant K_t over the tile's T range in
// shared memory, and every thread adds K_s(voxel) * K_t[T] into the 32
// accumulators it holds in registers.  Each voxel is written once, zeros
// included, so the grid needs no separate initialisation (the Theta(G) init of
// Algorithm 2 becomes part of the store stream).
//
// With per-event bandwidths (ADAPT) each kept event also carries (hsv_i, htv_i,
// 1/hsv_i, 1/htv_i): its reach test, T window and K_s, K_t use its own
// bandwidths, and its K_t row is weighted by (hs_max/hs_i)^2 (ht_max/ht_i), the
// plan holding the largest bandwidths and the matching normalisation.
#include "internal.cuh"
#include "tile_common.cuh"

namespace stkde {

namespace {

constexpr int F_THREADS = 256;   // 128 voxels x 2 halves of the T block
constexpr int F_TB = 64;         // voxels of T per tile
constexpr int F_HALF = 32;       // T accumulators per thread
constexpr int F_BATCH = 128;     // events per K_t table
constexpr int F_BUF = F_BATCH + F_THREADS;

// With BATCH, block b computes tile b of the batch's fp32 tile numbering: the
// problem is the last table entry whose fitem_base is <= b, and its plan, bins
// and output replace the arguments.
template <bool ADAPT, bool BATCH>
__global__ void __launch_bounds__(F_THREADS, 2)
k_tile_fp32(Plan pl, const float4* __restrict__ ev, const float4* __restrict__ evp,
            const uint32_t* __restrict__ start, float* __restrict__ out,
            const ProblemDev* __restrict__ table, int nprob) {
    __shared__ float4 buf[F_BUF];
    __shared__ float4 bufp[ADAPT ? F_BUF : 1];  // per-event bandwidths of buf
    __shared__ __align__(16) float ktab[F_BATCH][F_TB];
    __shared__ int2 win[F_BATCH];
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

    const int m = tid & (TILE_XY - 1), h = tid >> 7;
    const int X = g.X0 + m / TY, Y = g.Y0 + m % TY;
    const float xc = (float)X + 0.5f, yc = (float)Y + 0.5f;

    float acc[F_HALF];
#pragma unroll
    for (int c = 0; c < F_HALF; ++c) acc[c] = 0.0f;

    if (tid == 0) s_count = 0;
    __syncthreads();

    // Adds the events buf[off, off+cnt) into the accumulators.
    auto process = [&](int off, int cnt) {
        // temporal invariants K_t[T] over the tile's T block (Algorithm 3's bar)
        for (int q = tid; q < cnt * F_TB; q += F_THREADS) {
            const int j = q / F_TB, c = q % F_TB;
            if constexpr (ADAPT) {
                const float4 b = bufp[off + j];
                const float hr = pl.hsv * b.z;
                const float w = ((float)(g.T0 + c) + 0.5f - buf[off + j].z) * b.w;
                ktab[j][c] = (pl.ct * (hr * hr * (pl.htv * b.w))) * fmaxf(fmaf(-w, w, 1.0f), 0.0f);
            } else {
                const float w = ((float)(g.T0 + c) + 0.5f - buf[off + j].z) * pl.inv_ht;
                ktab[j][c] = pl.ct * fmaxf(fmaf(-w, w, 1.0f), 0.0f);
            }
        }
        for (int j = tid; j < cnt; j += F_THREADS) {
            const float pt = buf[off + j].z;
            const float htv = ADAPT ? bufp[off + j].y : pl.htv;
            win[j] = make_int2((int)floorf(pt - 0.5f - htv) - g.T0 - 1,
                               (int)ceilf(pt - 0.5f + htv) - g.T0 + 1);
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const float4 e = buf[off + j];
            const float ihs = ADAPT ? bufp[off + j].z : pl.inv_hs;
            const float u = (xc - e.x) * ihs;
            const float v = (yc - e.y) * ihs;
            const float s = fmaf(u, u, v * v);
            const float a = s < 1.0f ? pl.cs * fmaf(-u, u, 1.0f) * fmaf(-v, v, 1.0f) : 0.0f;
            if (!__any_sync(0xffffffffu, a != 0.0f)) continue;
            const int2 wj = win[j];
#pragma unroll
            for (int gq = 0; gq < F_HALF / 16; ++gq) {
                const int c0 = h * F_HALF + gq * 16;
                if (wj.x <= c0 + 15 && wj.y >= c0) {
                    const float4* kr = reinterpret_cast<const float4*>(&ktab[j][c0]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 k4 = kr[q];
                        acc[gq * 16 + 4 * q + 0] = fmaf(a, k4.x, acc[gq * 16 + 4 * q + 0]);
                        acc[gq * 16 + 4 * q + 1] = fmaf(a, k4.y, acc[gq * 16 + 4 * q + 1]);
                        acc[gq * 16 + 4 * q + 2] = fmaf(a, k4.z, acc[gq * 16 + 4 * q + 2]);
                        acc[gq * 16 + 4 * q + 3] = fmaf(a, k4.w, acc[gq * 16 + 4 * q + 3]);
                    }
                }
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

    if (X < pl.gx && Y < pl.gy) {
        const int Tb = g.T0 + h * F_HALF;
        float* dst = out + ((int64_t)X * pl.gy + Y) * (int64_t)pl.gt + Tb;
        const int nvalid = min(F_HALF, pl.gt - Tb);
        if (nvalid == F_HALF && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
            for (int q = 0; q < F_HALF / 4; ++q)
                reinterpret_cast<float4*>(dst)[q] =
                    make_float4(acc[4 * q] * pl.norm, acc[4 * q + 1] * pl.norm,
                                acc[4 * q + 2] * pl.norm, acc[4 * q + 3] * pl.norm);
        } else {
#pragma unroll
            for (int c = 0; c < F_HALF; ++c)
                if (c < nvalid) dst[c] = acc[c] * pl.norm;
        }
    }
}

}  // namespace

void launch_tile_fp32(const Plan& pl, const Bins& b, float* out, int* err, cudaStream_t st) {
    (void)err;
    Plan p = pl;
    p.tblock = F_TB;
    p.ntb = (pl.gt + F_TB - 1) / F_TB;
    const int64_t items = (int64_t)p.ntx * p.nty * p.ntb;
    if (items <= 0) return;
    if (b.evp)
        k_tile_fp32<true, false><<<(unsigned)items, F_THREADS, 0, st>>>(p, b.ev, b.evp, b.start, out,
                                                                        nullptr, 0);
    else
        k_tile_fp32<false, false><<<(unsigned)items, F_THREADS, 0, st>>>(p, b.ev, nullptr, b.start, out,
                                                                         nullptr, 0);
}

int64_t tile_fp32_items(const Plan& pl) {
    return (int64_t)pl.ntx * pl.nty * ((pl.gt + F_TB - 1) / F_TB);
}

bool launch_tile_fp32_batch(const ProblemDev* table, int nprob, int64_t total_items, cudaStream_t st) {
    if (nprob <= 0 || total_items <= 0) return true;
    if (total_items >= ((int64_t)1 << 31)) return false;
    k_tile_fp32<false, true><<<(unsigned)total_items, F_THREADS, 0, st>>>(Plan{}, nullptr, nullptr, nullptr,
                                                                          nullptr, table, nprob);
    return true;
}

}  // namespace stkde
