// Uniform bucketing grid over the first min(d,3) coordinates, used by the
// ordering and the pattern search.  A point p lies in cell
// floor((x_p,t - lo_t) / c) (clamped); any point within distance R of p lies
// in the cells within span = floor(R/c) + 1 of p's cell along each gridded
// axis, because a coordinate difference never exceeds the distance.
#pragma once
#include "common.cuh"

namespace kc {

struct Grid {
    int dg = 1;           // gridded axes
    double lo[3] = {0, 0, 0};
    double c = 1.0;       // cell size
    double inv_c = 1.0;   // 1 / c (multiplications only on the device)
    int n[3] = {1, 1, 1}; // cells per axis
    int64_t ncells = 1;
};

__device__ __forceinline__ int cell_coord(const Grid& g, double v, int t) {
    double f = (v - g.lo[t]) * g.inv_c;
    int q = (f <= 0.0) ? 0 : (f >= (double)(g.n[t] - 1) ? g.n[t] - 1 : (int)f);
    return q;
}
__device__ __forceinline__ int64_t cell_of(const Grid& g, const double* x) {
    int64_t key = 0;
    for (int t = g.dg - 1; t >= 0; --t) key = key * g.n[t] + cell_coord(g, x[t], t);
    return key;
}
// number of cells to either side covering radius R (R may be +inf)
__device__ __forceinline__ int span_for(const Grid& g, double R, int t) {
    if (!(R < 1e300)) return g.n[t];
    // a hair of slack so that rounding in R*inv_c or in the cell coordinates
    // can never drop a cell layer
    double f = R * g.inv_c * (1.0 + 1e-12) + 1e-9;
    if (f > 4.0e9) return g.n[t];
    int s = (int)f + 1;
    return s > g.n[t] ? g.n[t] : s;
}

// Search box of a query point x with radius R, packed as (cell x, cell y,
// cell z, span); computed once per query and expanded by box_range.
__device__ __forceinline__ int4 query_box(const Grid& g, const double* x, double R) {
    int c[3] = {0, 0, 0};
    int sp = 0;
    for (int t = 0; t < g.dg; ++t) {
        c[t] = cell_coord(g, x[t], t);
        sp = max(sp, span_for(g, R, t));
    }
    return make_int4(c[0], c[1], c[2], sp);
}
__device__ __forceinline__ void box_range(const Grid& g, int4 b, int* lo, int* hi) {
    const int c[3] = {b.x, b.y, b.z};
    for (int t = 0; t < 3; ++t) {
        lo[t] = t < g.dg ? max(0, c[t] - b.w) : 0;
        hi[t] = t < g.dg ? min(g.n[t] - 1, c[t] + b.w) : 0;
    }
}

// FP32 screen of a distance test.  a, b: coordinates minus a common origin,
// rounded to float from double; delta bounds the error of one coordinate
// difference (2^-23 times the largest |x - origin|).  Returns 1 when dist <= R
// surely holds, 0 when dist > R surely holds, -1 when only the exact FP64 test
// can tell.  The margin covers the float rounding of the inputs, of the sum of
// squares and of sqrtf (first order, with a factor of two to spare).
// Rf may carry up to two float roundings of the exact threshold.
__device__ __forceinline__ int screen_f32(const float* a, const float* b, int d, float Rf, float delta) {
    float s = 0.f;
    for (int t = 0; t < d; ++t) {
        const float w = a[t] - b[t];
        s = fmaf(w, w, s);
    }
    const float dist = sqrtf(s);
    const float M = sqrtf((float)d) * delta + (float)(d + 6) * 1.1920929e-7f * fmaxf(dist, Rf);
    if (dist - M > Rf) return 0;
    if (dist + M < Rf) return 1;
    return -1;
}

// Morton code of the first min(d,3) coordinates, quantised in the box
// [lo, lo + 1/inv] (16 bits per axis in 2-D, 10 in 3-D): points close in
// space get close codes.
struct Box3 {
    double lo[3], inv[3];
};
__device__ __forceinline__ uint32_t morton_of(const double* x, int d, const Box3& box) {
    const int dg = d < 3 ? d : 3;
    const int bits = dg <= 2 ? 16 : 10;
    uint32_t q[3] = {0, 0, 0};
    for (int t = 0; t < dg; ++t) {
        double f = (x[t] - box.lo[t]) * box.inv[t];
        f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
        q[t] = (uint32_t)(f * (double)((1u << bits) - 1));
    }
    uint32_t m = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int t = 0; t < dg; ++t) m = (m << 1) | ((q[t] >> b) & 1u);
    return m;
}

// Host: choose a grid for `npts` points in the box [lo, hi] with target cell
// size `want` (0 = automatic), at most `max_cells` cells.
Grid make_grid(int d, const double* lo, const double* hi, int64_t npts, double want, int64_t max_cells);

// Build the cell-sorted arrangement of the points `ids` (or 0..n-1 when ids is
// NULL) with coordinates x (row-major, stride d): outputs
//   sorted[q]      = the id at sorted position q
//   cell_start[c]  = first sorted position of cell c, cell_start[ncells] = n
kc_status grid_build(const Grid& g, const double* x, int d, const int32_t* ids, int64_t n, int32_t* sorted,
                     int64_t* cell_start, Arena& A, cudaStream_t s);

// Bounding box of x (row-major N x d) over the first min(d,3) axes; host out.
kc_status bbox(const double* x, int64_t N, int d, double* lo, double* hi, Arena& A, cudaStream_t s);

// Grid coordinates of the points x (row-major N x d): for d <= 3 the points
// themselves (*gx = x, *gs = d); for d > 3 their projections on the three
// principal axes of the point cloud (*gx: device N x 3 from the arena, *gs =
// 3).  The axes are orthonormal, so a grid coordinate of two points differs
// by no more than their distance and every search box stays exact; for data
// near a low-dimensional subspace they keep the boxes as tight as the data
// (the first three raw coordinates are an arbitrary projection of it).
kc_status grid_coords(const double* x, int64_t N, int d, Arena& A, cudaStream_t s, const double** gx, int* gs);

// Bounding box over all d <= 32 axes (host out), for the float copies used by
// the FP32 distance screens; E = the largest extent.
constexpr int MAXD = 32;
struct Origin {
    double lo[MAXD];
};
kc_status bbox_all(const double* x, int64_t N, int d, Origin* lo, double* E, Arena& A, cudaStream_t s);

}  // namespace kc
