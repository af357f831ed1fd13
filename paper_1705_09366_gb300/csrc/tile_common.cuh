// Tile geometry shared by the tile kernels: which bins to read for a tile and
// which events reach it.
#pragma once

#include "internal.cuh"

namespace stkde {

// One output tile: X in [X0, X1), Y in [Y0, Y1), T in [T0, T1), plus the range
// of event bins (slabs s_lo..s_hi, cell rows cx_lo..cx_hi, cells cy_lo..cy_hi
// within a row) that can hold events whose cylinder reaches it.
struct TileGeom {
    int X0, X1, Y0, Y1, T0, T1;
    float rx0, rx1, ry0, ry1;  // in-grid voxel-centre rectangle of the tile
    int cx_lo, cx_hi, cy_lo, cy_hi, s_lo, s_hi;
};

// Bandwidth class `cls` of the plan (a = cls / ncls_t, b = cls % ncls_t) and its
// reach in voxels: the class's largest possible bandwidths.
__device__ __forceinline__ int plan_classes(const Plan& pl) { return pl.ncls_s * pl.ncls_t; }
__device__ __forceinline__ float class_hsv(const Plan& pl, int cls) {
    return ldexpf(pl.hsv, -(cls / pl.ncls_t));
}
__device__ __forceinline__ float class_htv(const Plan& pl, int cls) {
    return ldexpf(pl.htv, -(cls % pl.ncls_t));
}
// First key of bin (class cls, slab s, cell x cx); cells y follow.
__device__ __forceinline__ uint32_t bin_row(const Plan& pl, int cls, int s, int cx) {
    return (((uint32_t)cls * (uint32_t)pl.nslab + (uint32_t)s) * (uint32_t)pl.ntx + (uint32_t)cx) *
           (uint32_t)pl.nty;
}

// The tile with the reach (hsv, htv) of one bandwidth class.
__device__ __forceinline__ TileGeom tile_geom_r(const Plan& pl, float hsv, float htv, int tx, int ty,
                                                int tb, int tblock) {
    TileGeom g;
    g.X0 = tx * TX; g.X1 = min(g.X0 + TX, pl.gx);
    g.Y0 = ty * TY; g.Y1 = min(g.Y0 + TY, pl.gy);
    g.T0 = tb * tblock; g.T1 = min(g.T0 + tblock, pl.gt);
    g.rx0 = (float)g.X0 + 0.5f; g.rx1 = (float)g.X1 - 0.5f;
    g.ry0 = (float)g.Y0 + 0.5f; g.ry1 = (float)g.Y1 - 0.5f;
    const float m = 0.01f;  // widen: binning only needs a superset
    g.cx_lo = max(0, (int)floorf((g.rx0 - hsv - m) * (1.0f / TX)));
    g.cx_hi = min(pl.ntx - 1, (int)floorf((g.rx1 + hsv + m) * (1.0f / TX)));
    g.cy_lo = max(0, (int)floorf((g.ry0 - hsv - m) * (1.0f / TY)));
    g.cy_hi = min(pl.nty - 1, (int)floorf((g.ry1 + hsv + m) * (1.0f / TY)));
    const float t0 = (float)g.T0 + 0.5f - htv - m, t1 = (float)g.T1 - 0.5f + htv + m;
    g.s_lo = max(0, (int)floorf(t0 / (float)pl.slab));
    g.s_hi = min(pl.nslab - 1, (int)floorf(t1 / (float)pl.slab));
    return g;
}

__device__ __forceinline__ TileGeom tile_geom(const Plan& pl, int tx, int ty, int tb, int tblock) {
    return tile_geom_r(pl, pl.hsv, pl.htv, tx, ty, tb, tblock);
}

// Does the cylinder of radius hsv and half-height htv (voxels) around the event
// reach a voxel centre of the tile?  A superset test (bandwidths widened by 0.01
// voxel): events that pass but reach nothing add zeros.
__device__ __forceinline__ bool reaches_bw(const TileGeom& g, float4 e, float hsv, float htv) {
    const float dx = fmaxf(fmaxf(g.rx0 - e.x, e.x - g.rx1), 0.0f);
    const float dy = fmaxf(fmaxf(g.ry0 - e.y, e.y - g.ry1), 0.0f);
    const float r = hsv + 0.01f;
    const bool xy = dx * dx + dy * dy < r * r;
    const bool t = (e.z + htv + 0.01f > (float)g.T0 + 0.5f) &&
                   (e.z - htv - 0.01f < (float)g.T1 - 0.5f);
    return xy && t;
}

// The same with the problem's bandwidths.
__device__ __forceinline__ bool reaches(const Plan& pl, const TileGeom& g, float4 e) {
    return reaches_bw(g, e, pl.hsv, pl.htv);
}

}  // namespace stkde
