// K6: plain GPU scatter, a direct port of PB-SYM (Section 3.2, Algorithm 3).
//
// One CTA per event builds the event's temporal invariant K_t[T] (the bar) in
// shared memory; its warps then walk the (X, Y) columns of the event's box,
// evaluate the spatial invariant K_s[X][Y] (the disk) and add K_s * K_t[T] along
// T with atomic adds into a grid zeroed beforehand.  The lanes of a warp run
// along T of one column (or of a few columns when the bar is short), so each
// atomic instruction covers contiguous addresses; when G_t is a multiple of 4
// and the grid 16-byte aligned, every lane adds four consecutive voxels with
// one vector reduction (float4 atomicAdd).  It is the baseline the tile kernels are
// measured against: correct to rounding, but the order in which events reach a
// voxel, and so the last bits, change from run to run.
#include "internal.cuh"

namespace stkde {

namespace {

constexpr int S_THREADS = 128;

// VEC: 4 voxels of T per lane (G_t % 4 == 0), else 1.
template <int VEC>
__global__ void __launch_bounds__(S_THREADS)
k_scatter(Plan pl, const float4* __restrict__ ev, float* __restrict__ out) {
    extern __shared__ float kt[];  // K_t over [T0, T0 + VEC * nq), zero outside the bar and grid
    const float4 e = ev[blockIdx.x];
    if (!(fabsf(e.x) < 1e9f && fabsf(e.y) < 1e9f && fabsf(e.z) < 1e9f)) return;
    const int Hs = (int)ceilf(pl.hsv), Ht = (int)ceilf(pl.htv);
    const int Xi = (int)floorf(e.x), Yi = (int)floorf(e.y), Ti = (int)floorf(e.z);
    const int Xlo = max(0, Xi - Hs), Xhi = min(pl.gx - 1, Xi + Hs);
    const int Ylo = max(0, Yi - Hs), Yhi = min(pl.gy - 1, Yi + Hs);
    const int Tlo = max(0, Ti - Ht), Thi = min(pl.gt - 1, Ti + Ht);
    if (Xlo > Xhi || Ylo > Yhi || Tlo > Thi) return;
    const int T0 = VEC == 4 ? (Tlo & ~3) : Tlo;
    const int nq = (Thi - T0) / VEC + 1;  // lanes' work items along T
    for (int q = threadIdx.x; q < nq * VEC; q += S_THREADS) {
        const int T = T0 + q;
        const float w = ((float)T + 0.5f - e.z) * pl.inv_ht;
        kt[q] = (T >= Tlo && T <= Thi) ? pl.ct * fmaxf(fmaf(-w, w, 1.0f), 0.0f) : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // columns handled by one warp pass: lanes split into groups of nq (>= 1 column)
    const int cpw = nq < 32 ? 32 / nq : 1;
    const int c_in = nq < 32 ? lane / nq : 0;
    const int q0 = nq < 32 ? lane % nq : lane;
    const bool active = c_in < cpw;
    const int ny = Yhi - Ylo + 1;
    const int ncol = (Xhi - Xlo + 1) * ny;
    const float norm_cs = pl.norm * pl.cs;
    for (int base = warp * cpw; base < ncol; base += (S_THREADS / 32) * cpw) {
        const int col = base + c_in;
        if (!active || col >= ncol) continue;
        const int X = Xlo + col / ny, Y = Ylo + col % ny;
        const float u = ((float)X + 0.5f - e.x) * pl.inv_hs;
        const float v = ((float)Y + 0.5f - e.y) * pl.inv_hs;
        if (!(fmaf(u, u, v * v) < 1.0f)) continue;
        const float a = norm_cs * fmaf(-u, u, 1.0f) * fmaf(-v, v, 1.0f);
        float* dst = out + ((int64_t)X * pl.gy + Y) * (int64_t)pl.gt + T0;
        for (int q = q0; q < nq; q += (nq < 32 ? nq : 32)) {
            if constexpr (VEC == 4) {
                const float4 k = reinterpret_cast<const float4*>(kt)[q];
                if (k.x != 0.0f || k.y != 0.0f || k.z != 0.0f || k.w != 0.0f)
                    atomicAdd(reinterpret_cast<float4*>(dst) + q,
                              make_float4(a * k.x, a * k.y, a * k.z, a * k.w));
            } else {
                const float k = kt[q];
                if (k != 0.0f) atomicAdd(dst + q, a * k);
            }
        }
    }
}

}  // namespace

void launch_scatter(const Plan& pl, const float4* ev, float* out, cudaStream_t st) {
    if (pl.n <= 0) return;
    const int Ht = (int)ceilf(pl.htv);
    const size_t sm = sizeof(float) * (size_t)(2 * Ht + 1 + 8);
    // the vector form needs every column start 16-byte aligned
    if ((pl.gt & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0)
        k_scatter<4><<<pl.n, S_THREADS, sm, st>>>(pl, ev, out);
    else
        k_scatter<1><<<pl.n, S_THREADS, sm, st>>>(pl, ev, out);
}

}  // namespace stkde
