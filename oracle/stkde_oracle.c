/*
 * FP64 CPU oracle for space-time kernel density estimation (STKDE).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * GPU library is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never does, and
 * the two share no code.
 *
 * What is computed (Section 2.1, the density equation and kernels k_s, k_t):
 *
 *   f(x,y,t) = 1/(n hs^2 ht) * sum_{i : d_i < hs, |t - t_i| <= ht}
 *                 k_s((x - x_i)/hs, (y - y_i)/hs) * k_t((t - t_i)/ht)
 *
 * with d_i the planar distance of event i to the sampling point (x, y).
 * Readings taken where the printed text is garbled or silent:
 *   - kernels: k_s(u,v) = c_s (1-u^2)(1-v^2), k_t(w) = c_t (1-w^2); the printed
 *     (1-u)^2 forms are not even in u, which the "distance decay" description
 *     rules out.  c_s and c_t are parameters (printed values pi/2 and 3/4).
 *   - sampling point of voxel (X,Y,T) is its centre: x = x0 + (X + 1/2) sres
 *     (Table 1 calls s = (x,y,t) the voxel's sampling coordinate); the offset
 *     is a parameter so tests can also use the corner.
 *   - space is compared strictly (d < hs), time inclusively (|dt| <= ht), as
 *     in Algorithms 1-3.
 *   - every event counts in n, including events outside the grid; voxels of a
 *     cylinder that fall outside the grid are dropped (Algorithm 1 scans all
 *     events for each in-grid voxel).
 *   - n = 0 gives an all-zero grid.
 *
 * Two independent evaluations are provided:
 *   - oracle_vb*: Algorithm 1 (VB), voxel loop outside, every event inside,
 *     distances in domain units exactly as the pseudo-code writes them;
 *   - oracle_pb*: Algorithm 2 (PB), event loop outside, then the voxel box
 *     around the event's voxel, in voxel units after re-centring the event on
 *     the grid origin (Section 2.1 discretisation, Table 1).
 *
 * Grid layout: out[(X*gy + Y)*gt + T], T fastest (the stkde[X][Y][T] array of
 * Algorithms 1-3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double x0, y0, t0;    /* domain origin = corner of voxel (0,0,0) */
    double sres, tres;    /* voxel size: space (x and y), time */
    int64_t gx, gy, gt;   /* grid size in voxels */
    double hs, ht;        /* bandwidths, domain units */
    double cs, ct;        /* kernel constants c_s, c_t */
    double sample_off;    /* 0.5 = voxel centre (default reading), 0 = corner */
    int32_t round_fp32;   /* 1: re-centred voxel-unit event coordinates rounded to binary32 */
    int32_t nthreads;     /* OpenMP threads for the full-grid PB (<= 0: all) */
} oracle_params;

/* Half-width of the band |u^2+v^2 - 1| <= TIE_BAND inside which a binary32
 * evaluation of the spatial membership test may disagree with FP64. */
#define TIE_BAND (1.0 / 1048576.0)

static void set_threads(const oracle_params* p) {
#ifdef _OPENMP
    if (p->nthreads > 0) omp_set_num_threads(p->nthreads);
#else
    (void)p;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Event i in voxel units, re-centred on the grid origin (Section 2.1: the domain
 * is discretised with resolutions sres, tres).  Optionally rounded to binary32,
 * the precision in which the GPU path evaluates the kernels. */
static void recentre(const oracle_params* p, const double* pts, int64_t i,
                     double* px, double* py, double* pt) {
    double x = (pts[3 * i + 0] - p->x0) / p->sres;
    double y = (pts[3 * i + 1] - p->y0) / p->sres;
    double t = (pts[3 * i + 2] - p->t0) / p->tres;
    if (p->round_fp32) {
        x = (double)(float)x;
        y = (double)(float)y;
        t = (double)(float)t;
    }
    *px = x; *py = y; *pt = t;
}

/* Event i in domain units, as Algorithm 1 reads it.  With round_fp32 the event is
 * moved to the binary32-rounded voxel position so that VB and PB describe the
 * same event set. */
static void event_domain(const oracle_params* p, const double* pts, int64_t i,
                         double* xi, double* yi, double* ti) {
    if (p->round_fp32) {
        double px, py, pt;
        recentre(p, pts, i, &px, &py, &pt);
        *xi = p->x0 + px * p->sres;
        *yi = p->y0 + py * p->sres;
        *ti = p->t0 + pt * p->tres;
    } else {
        *xi = pts[3 * i + 0];
        *yi = pts[3 * i + 1];
        *ti = pts[3 * i + 2];
    }
}

static double k_s(const oracle_params* p, double u, double v) {
    return p->cs * (1.0 - u * u) * (1.0 - v * v);
}

static double k_t(const oracle_params* p, double w) {
    return p->ct * (1.0 - w * w);
}

static double norm_factor(const oracle_params* p, int64_t n) {
    return 1.0 / ((double)n * p->hs * p->hs * p->ht);
}

/* ---------------------------------------------------------------- VB --- */

/* Algorithm 1 (VB) for one voxel: scan every event, test the cylinder in
 * domain units, sum k_s * k_t, divide by n hs^2 ht. */
static double vb_voxel(const oracle_params* p, const double* pts, int64_t n,
                       int64_t X, int64_t Y, int64_t T) {
    const double x = p->x0 + ((double)X + p->sample_off) * p->sres;
    const double y = p->y0 + ((double)Y + p->sample_off) * p->sres;
    const double t = p->t0 + ((double)T + p->sample_off) * p->tres;
    double sum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double xi, yi, ti;
        event_domain(p, pts, i, &xi, &yi, &ti);
        const double d = sqrt((xi - x) * (xi - x) + (yi - y) * (yi - y));
        if (d < p->hs && fabs(ti - t) <= p->ht)
            sum += k_s(p, (x - xi) / p->hs, (y - yi) / p->hs) * k_t(p, (t - ti) / p->ht);
    }
    return sum * norm_factor(p, n);
}

/* Full grid by VB.  Cost Theta(gx gy gt n): tiny inputs only. */
int oracle_vb(const oracle_params* p, const double* pts, int64_t n, double* out) {
    const int64_t G = p->gx * p->gy * p->gt;
    if (n == 0) { memset(out, 0, sizeof(double) * (size_t)G); return 0; }
    set_threads(p);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t X = 0; X < p->gx; ++X)
        for (int64_t Y = 0; Y < p->gy; ++Y)
            for (int64_t T = 0; T < p->gt; ++T)
                out[(X * p->gy + Y) * p->gt + T] = vb_voxel(p, pts, n, X, Y, T);
    return 0;
}

/* VB on a list of voxels vox[3*j + {0,1,2}] = (X, Y, T). */
int oracle_vb_voxels(const oracle_params* p, const double* pts, int64_t n,
                     const int64_t* vox, int64_t m, double* vals) {
    set_threads(p);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < m; ++j)
        vals[j] = n == 0 ? 0.0 : vb_voxel(p, pts, n, vox[3 * j], vox[3 * j + 1], vox[3 * j + 2]);
    return 0;
}

/* ---------------------------------------------------------------- PB --- */

/* Voxel box of an event: [Xi - H, Xi + H] with Xi = floor(px) and
 * H = ceil(h / res), the bandwidth in voxels of Section 2.1.  The box covers the
 * cylinder for any sampling offset off in [0, 1): voxel X is reached only if
 * |X + off - px| <= h/res, and px - Xi lies in [0, 1), so
 * Xi - h/res - 1 < X < Xi + h/res + 1. */
static int event_box(double pc, double hhat, int64_t lo_clip, int64_t hi_clip,
                     int64_t* lo, int64_t* hi) {
    if (!(pc > -4.0e15 && pc < 4.0e15)) return 0;   /* non-finite or far away */
    const int64_t c = (int64_t)floor(pc);
    const int64_t H = (int64_t)ceil(hhat);
    int64_t a = c - H, b = c + H;
    if (a < lo_clip) a = lo_clip;
    if (b > hi_clip) b = hi_clip;
    *lo = a; *hi = b;
    return a <= b;
}

/* Algorithm 2 (PB) restricted to the voxel box [bx0,bx1) x [by0,by1) x [bt0,bt1),
 * written into box[((X-bx0)*(by1-by0) + (Y-by0))*(bt1-bt0) + (T-bt0)].
 * If slack != NULL it receives, per voxel, the sum of |term| over the event-voxel
 * pairs whose spatial test sits within TIE_BAND of the cylinder wall: pairs for
 * which a binary32 evaluation may legitimately decide the other way. */
static void pb_box(const oracle_params* p, const double* pts, int64_t n,
                   int64_t bx0, int64_t bx1, int64_t by0, int64_t by1,
                   int64_t bt0, int64_t bt1, double* box, double* slack, uint64_t* npairs) {
    const int64_t ny = by1 - by0, nt = bt1 - bt0;
    const size_t cells = (size_t)(bx1 - bx0) * (size_t)ny * (size_t)nt;
    memset(box, 0, sizeof(double) * cells);
    if (slack) memset(slack, 0, sizeof(double) * cells);
    if (npairs) *npairs = 0;
    if (n == 0) return;
    uint64_t pairs = 0;
    const double hsv = p->hs / p->sres, htv = p->ht / p->tres;   /* bandwidths in voxels */
    const double nrm = norm_factor(p, n);
    for (int64_t i = 0; i < n; ++i) {
        double px, py, pt;
        recentre(p, pts, i, &px, &py, &pt);
        int64_t xa, xb, ya, yb, ta, tb;
        if (!event_box(px, hsv, bx0, bx1 - 1, &xa, &xb)) continue;
        if (!event_box(py, hsv, by0, by1 - 1, &ya, &yb)) continue;
        if (!event_box(pt, htv, bt0, bt1 - 1, &ta, &tb)) continue;
        for (int64_t X = xa; X <= xb; ++X) {
            const double u = ((double)X + p->sample_off - px) / hsv;
            for (int64_t Y = ya; Y <= yb; ++Y) {
                const double v = ((double)Y + p->sample_off - py) / hsv;
                const double s = u * u + v * v;
                const int inside = s < 1.0;
                const int tie = fabs(s - 1.0) <= TIE_BAND;
                if (!inside && !tie) continue;
                const double ks = k_s(p, u, v);
                const size_t base = (size_t)(((X - bx0) * ny + (Y - by0)) * nt);
                for (int64_t T = ta; T <= tb; ++T) {
                    const double w = ((double)T + p->sample_off - pt) / htv;
                    if (!(fabs(w) <= 1.0)) continue;
                    const double term = ks * k_t(p, w) * nrm;
                    pairs += (uint64_t)inside;
                    if (inside) box[base + (size_t)(T - bt0)] += term;
                    if (tie && slack) slack[base + (size_t)(T - bt0)] += fabs(term);
                }
            }
        }
    }
    if (npairs) *npairs = pairs;
}

/* Full grid by PB.  OpenMP over X-slabs: each thread owns whole X planes and
 * scans all events, so every voxel sums its events in index order and the
 * result does not depend on the thread count. */
int oracle_pb(const oracle_params* p, const double* pts, int64_t n, double* out, double* slack) {
    set_threads(p);
    const int64_t gx = p->gx;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t X = 0; X < gx; ++X) {
        const size_t off = (size_t)X * (size_t)p->gy * (size_t)p->gt;
        pb_box(p, pts, n, X, X + 1, 0, p->gy, 0, p->gt, out + off, slack ? slack + off : NULL, NULL);
    }
    return 0;
}

/* PB on one box of the grid (sampled-tile parity on large grids). */
int oracle_pb_box(const oracle_params* p, const double* pts, int64_t n,
                  int64_t bx0, int64_t bx1, int64_t by0, int64_t by1,
                  int64_t bt0, int64_t bt1, double* box, double* slack) {
    if (bx0 < 0 || by0 < 0 || bt0 < 0 || bx1 > p->gx || by1 > p->gy || bt1 > p->gt ||
        bx0 >= bx1 || by0 >= by1 || bt0 >= bt1)
        return 1;
    pb_box(p, pts, n, bx0, bx1, by0, by1, bt0, bt1, box, slack, NULL);
    return 0;
}

/* Many boxes at once, one OpenMP task per box (boxes[6*j..6*j+5] =
 * bx0,bx1,by0,by1,bt0,bt1; outputs packed one after another).  npairs[j], if
 * given, receives the number of in-cylinder (event, voxel) pairs of box j. */
int oracle_pb_boxes(const oracle_params* p, const double* pts, int64_t n,
                    const int64_t* boxes, int64_t nbox, double* out, double* slack,
                    uint64_t* npairs) {
    set_threads(p);
    int64_t* offs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nbox + 1));
    if (!offs) return 2;
    offs[0] = 0;
    for (int64_t j = 0; j < nbox; ++j) {
        const int64_t* b = boxes + 6 * j;
        if (b[0] < 0 || b[2] < 0 || b[4] < 0 || b[1] > p->gx || b[3] > p->gy || b[5] > p->gt ||
            b[0] >= b[1] || b[2] >= b[3] || b[4] >= b[5]) { free(offs); return 1; }
        offs[j + 1] = offs[j] + (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4]);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < nbox; ++j) {
        const int64_t* b = boxes + 6 * j;
        pb_box(p, pts, n, b[0], b[1], b[2], b[3], b[4], b[5], out + offs[j],
               slack ? slack + offs[j] : NULL, npairs ? npairs + j : NULL);
    }
    free(offs);
    return 0;
}

/* Work count: the number of (event, in-grid voxel) pairs inside the cylinder
 * (spatial test strict, temporal inclusive), i.e. the voxel-point updates that
 * Algorithm 2 performs with a non-rejected test.  Exact integer, summed in a
 * fixed order per event. */
int oracle_count_updates(const oracle_params* p, const double* pts, int64_t n, uint64_t* count) {
    set_threads(p);
    const double hsv = p->hs / p->sres, htv = p->ht / p->tres;
    uint64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : total)
    for (int64_t i = 0; i < n; ++i) {
        double px, py, pt;
        recentre(p, pts, i, &px, &py, &pt);
        int64_t xa, xb, ya, yb, ta, tb;
        if (!event_box(px, hsv, 0, p->gx - 1, &xa, &xb)) continue;
        if (!event_box(py, hsv, 0, p->gy - 1, &ya, &yb)) continue;
        if (!event_box(pt, htv, 0, p->gt - 1, &ta, &tb)) continue;
        uint64_t nt = 0;
        for (int64_t T = ta; T <= tb; ++T) {
            const double w = ((double)T + p->sample_off - pt) / htv;
            nt += fabs(w) <= 1.0;
        }
        uint64_t nxy = 0;
        for (int64_t X = xa; X <= xb; ++X) {
            const double u = ((double)X + p->sample_off - px) / hsv;
            for (int64_t Y = ya; Y <= yb; ++Y) {
                const double v = ((double)Y + p->sample_off - py) / hsv;
                nxy += (u * u + v * v) < 1.0;
            }
        }
        total += nxy * nt;
    }
    *count = total;
    return 0;
}

/* ---------------------------------------------------- adaptive bandwidth --- */

/* Per-event bandwidths, the generalisation the conclusion names as future work
 * (a bandwidth that adapts to the local density of the population): event i
 * carries its own hs_i, ht_i (domain units) and its own normalisation,
 *
 *   f(x,y,t) = 1/n * sum_{i : d_i < hs_i, |t - t_i| <= ht_i}
 *                 k_s((x - x_i)/hs_i, (y - y_i)/hs_i) * k_t((t - t_i)/ht_i) / (hs_i^2 ht_i),
 *
 * so each event still contributes a separable cylinder of unit-scaled mass and
 * every hs_i = hs, ht_i = ht gives the density above.  p->hs and p->ht are not
 * used.  VB (Algorithm 1 with the per-event test) and PB (Algorithm 2 with a
 * per-event box) are again written independently. */

int oracle_vb_adaptive(const oracle_params* p, const double* pts, const double* hs,
                       const double* ht, int64_t n, double* out) {
    const int64_t G = p->gx * p->gy * p->gt;
    if (n == 0) { memset(out, 0, sizeof(double) * (size_t)G); return 0; }
    set_threads(p);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t X = 0; X < p->gx; ++X)
        for (int64_t Y = 0; Y < p->gy; ++Y)
            for (int64_t T = 0; T < p->gt; ++T) {
                const double x = p->x0 + ((double)X + p->sample_off) * p->sres;
                const double y = p->y0 + ((double)Y + p->sample_off) * p->sres;
                const double t = p->t0 + ((double)T + p->sample_off) * p->tres;
                double sum = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    double xi, yi, ti;
                    event_domain(p, pts, i, &xi, &yi, &ti);
                    const double d = sqrt((xi - x) * (xi - x) + (yi - y) * (yi - y));
                    if (d < hs[i] && fabs(ti - t) <= ht[i])
                        sum += k_s(p, (x - xi) / hs[i], (y - yi) / hs[i]) * k_t(p, (t - ti) / ht[i]) /
                               (hs[i] * hs[i] * ht[i]);
                }
                out[(X * p->gy + Y) * p->gt + T] = sum / (double)n;
            }
    return 0;
}

/* PB with per-event bandwidths over the voxel box [bx0,bx1) x [by0,by1) x
 * [bt0,bt1); slack as in pb_box, with the tie band on each event's own disk. */
static void pb_box_adaptive(const oracle_params* p, const double* pts, const double* hs,
                            const double* ht, int64_t n, int64_t bx0, int64_t bx1, int64_t by0,
                            int64_t by1, int64_t bt0, int64_t bt1, double* box, double* slack,
                            uint64_t* npairs) {
    const int64_t ny = by1 - by0, nt = bt1 - bt0;
    const size_t cells = (size_t)(bx1 - bx0) * (size_t)ny * (size_t)nt;
    memset(box, 0, sizeof(double) * cells);
    if (slack) memset(slack, 0, sizeof(double) * cells);
    if (npairs) *npairs = 0;
    if (n == 0) return;
    uint64_t pairs = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double hsv = hs[i] / p->sres, htv = ht[i] / p->tres;   /* bandwidths in voxels */
        const double nrm = 1.0 / ((double)n * hs[i] * hs[i] * ht[i]);
        double px, py, pt;
        recentre(p, pts, i, &px, &py, &pt);
        int64_t xa, xb, ya, yb, ta, tb;
        if (!event_box(px, hsv, bx0, bx1 - 1, &xa, &xb)) continue;
        if (!event_box(py, hsv, by0, by1 - 1, &ya, &yb)) continue;
        if (!event_box(pt, htv, bt0, bt1 - 1, &ta, &tb)) continue;
        for (int64_t X = xa; X <= xb; ++X) {
            const double u = ((double)X + p->sample_off - px) / hsv;
            for (int64_t Y = ya; Y <= yb; ++Y) {
                const double v = ((double)Y + p->sample_off - py) / hsv;
                const double s = u * u + v * v;
                const int inside = s < 1.0;
                const int tie = fabs(s - 1.0) <= TIE_BAND;
                if (!inside && !tie) continue;
                const double ks = k_s(p, u, v);
                const size_t base = (size_t)(((X - bx0) * ny + (Y - by0)) * nt);
                for (int64_t T = ta; T <= tb; ++T) {
                    const double w = ((double)T + p->sample_off - pt) / htv;
                    if (!(fabs(w) <= 1.0)) continue;
                    const double term = ks * k_t(p, w) * nrm;
                    if (inside) box[base + (size_t)(T - bt0)] += term;
                    if (tie && slack) slack[base + (size_t)(T - bt0)] += fabs(term);
                    pairs += (uint64_t)inside;
                }
            }
        }
    }
    if (npairs) *npairs = pairs;
}

/* Full grid by adaptive PB; OpenMP over X planes as oracle_pb. */
int oracle_pb_adaptive(const oracle_params* p, const double* pts, const double* hs,
                       const double* ht, int64_t n, double* out, double* slack) {
    set_threads(p);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t X = 0; X < p->gx; ++X) {
        const size_t off = (size_t)X * (size_t)p->gy * (size_t)p->gt;
        pb_box_adaptive(p, pts, hs, ht, n, X, X + 1, 0, p->gy, 0, p->gt, out + off,
                        slack ? slack + off : NULL, NULL);
    }
    return 0;
}

/* Adaptive PB on a list of boxes (bx0, bx1, by0, by1, bt0, bt1); npairs[j], if
 * given, receives the in-cylinder (event, voxel) pairs of box j. */
int oracle_pb_adaptive_boxes(const oracle_params* p, const double* pts, const double* hs,
                             const double* ht, int64_t n, const int64_t* boxes, int64_t nbox,
                             double* out, double* slack, uint64_t* npairs) {
    set_threads(p);
    int64_t* offs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nbox + 1));
    if (!offs) return 1;
    offs[0] = 0;
    for (int64_t j = 0; j < nbox; ++j) {
        const int64_t* b = boxes + 6 * j;
        offs[j + 1] = offs[j] + (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4]);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < nbox; ++j) {
        const int64_t* b = boxes + 6 * j;
        pb_box_adaptive(p, pts, hs, ht, n, b[0], b[1], b[2], b[3], b[4], b[5], out + offs[j],
                        slack ? slack + offs[j] : NULL, npairs ? npairs + j : NULL);
    }
    free(offs);
    return 0;
}

/* ------------------------------------------- bandwidths from a pilot grid --- */

/* Per-event bandwidths that follow the population density (the adaptive
 * bandwidth of the conclusion), by Abramson's square-root law: a pilot density
 * f~ computed with the fixed pair (hs, ht) (p->hs, p->ht) is read at each
 * event's voxel, X_i = floor((x_i - x0)/sres) clamped into the grid (likewise Y,
 * T), floored at 1e-6 of the largest such value, and
 *
 *   lambda_i = clamp((f~_i / g)^(-alpha), lam_min, lam_max),
 *   g = exp(mean_i log f~_i),   hs_i = hs lambda_i,   ht_i = ht lambda_i,
 *
 * so dense areas get narrower kernels; alpha = 1/2 is Abramson's choice.  pilot
 * is the gx*gy*gt grid in the layout of oracle_pb; lam_out may be NULL. */
int oracle_abramson(const oracle_params* p, const double* pts, int64_t n, const double* pilot,
                    double alpha, double lam_min, double lam_max, double* hs_out, double* ht_out,
                    double* lam_out) {
    if (n <= 0) return 0;
    double* f = (double*)malloc(sizeof(double) * (size_t)n);
    if (!f) return 1;
    double fmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t X = (int64_t)floor((pts[3 * i + 0] - p->x0) / p->sres);
        int64_t Y = (int64_t)floor((pts[3 * i + 1] - p->y0) / p->sres);
        int64_t T = (int64_t)floor((pts[3 * i + 2] - p->t0) / p->tres);
        X = X < 0 ? 0 : X >= p->gx ? p->gx - 1 : X;
        Y = Y < 0 ? 0 : Y >= p->gy ? p->gy - 1 : Y;
        T = T < 0 ? 0 : T >= p->gt ? p->gt - 1 : T;
        f[i] = pilot[(X * p->gy + Y) * p->gt + T];
        if (f[i] > fmax) fmax = f[i];
    }
    const double floor_f = 1e-6 * fmax;
    double slog = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (f[i] < floor_f) f[i] = floor_f;
        slog += log(f[i]);
    }
    const double g = exp(slog / (double)n);
    for (int64_t i = 0; i < n; ++i) {
        double lam = fmax > 0.0 ? pow(f[i] / g, -alpha) : 1.0;
        lam = lam < lam_min ? lam_min : lam > lam_max ? lam_max : lam;
        hs_out[i] = p->hs * lam;
        ht_out[i] = p->ht * lam;
        if (lam_out) lam_out[i] = lam;
    }
    free(f);
    return 0;
}
