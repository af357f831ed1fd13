// K6: plain GPU scatter, a direct port of PB-SYM (Section 3.2, Algorithm 3).
//
// One CTA per event builds the event's temporal invariant K_t[T] (the bar) in
// shared memory, each thread takes (X, Y) columns of the event's box, evaluates
// the spatial invariant K_s[X][Y] (the disk), and adds K_s * K_t[T] along T with
// atomic adds into a grid zeroed beforehand.  It is the baseline the tile
// kernels are measured against: correct to rounding, but the order in which
// events reach a voxel, and so the last bits, change from run to run.
#include "internal.cuh"

namespace stkde {

namespace {

__global__ void __launch_bounds__(128)
k_scatter(Plan pl, const float4* __restrict__ ev, float* __restrict__ out) {
    extern __shared__ float kt[];
    const float4 e = ev[blockIdx.x];
    if (!(fabsf(e.x) < 1e9f && fabsf(e.y) < 1e9f && fabsf(e.z) < 1e9f)) return;
    const int Hs = (int)ceilf(pl.hsv), Ht = (int)ceilf(pl.htv);
    const int Xi = (int)floorf(e.x), Yi = (int)floorf(e.y), Ti = (int)floorf(e.z);
    const int Xlo = max(0, Xi - Hs), Xhi = min(pl.gx - 1, Xi + Hs);
    const int Ylo = max(0, Yi - Hs), Yhi = min(pl.gy - 1, Yi + Hs);
    const int Tlo = max(0, Ti - Ht), Thi = min(pl.gt - 1, Ti + Ht);
    if (Xlo > Xhi || Ylo > Yhi || Tlo > Thi) return;
    const int nt = Thi - Tlo + 1;
    for (int q = threadIdx.x; q < nt; q += blockDim.x) {
        const float w = ((float)(Tlo + q) + 0.5f - e.z) * pl.inv_ht;
        kt[q] = pl.ct * fmaxf(fmaf(-w, w, 1.0f), 0.0f);
    }
    __syncthreads();
    const int ny = Yhi - Ylo + 1;
    const int ncol = (Xhi - Xlo + 1) * ny;
    for (int col = threadIdx.x; col < ncol; col += blockDim.x) {
        const int X = Xlo + col / ny, Y = Ylo + col % ny;
        const float u = ((float)X + 0.5f - e.x) * pl.inv_hs;
        const float v = ((float)Y + 0.5f - e.y) * pl.inv_hs;
        if (!(fmaf(u, u, v * v) < 1.0f)) continue;
        const float a = pl.norm * pl.cs * fmaf(-u, u, 1.0f) * fmaf(-v, v, 1.0f);
        float* dst = out + ((int64_t)X * pl.gy + Y) * (int64_t)pl.gt + Tlo;
        for (int q = 0; q < nt; ++q) {
            const float k = kt[q];
            if (k != 0.0f) atomicAdd(dst + q, a * k);
        }
    }
}

}  // namespace

void launch_scatter(const Plan& pl, const float4* ev, float* out, cudaStream_t st) {
    if (pl.n <= 0) return;
    const int Ht = (int)ceilf(pl.htv);
    const size_t sm = sizeof(float) * (size_t)(2 * Ht + 1);
    k_scatter<<<pl.n, 128, sm, st>>>(pl, ev, out);
}

}  // namespace stkde
