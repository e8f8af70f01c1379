// a2: the maximin ordering (Section 2.3), exact, on the device.
//
// Definition (greedy): the first point is original index 0; each next point
// is the unselected point with the largest squared distance v(p) to the
// selected set, ties to the smaller original index; l = sqrt(v at selection).
// Write key(p) = (v(p), -index).  The l values are non-increasing, so the
// order is the sort of the points by final key, and each point's final v is
// what must be found.
//
// Parallel rounds.  Keep for every undecided point its v over the points
// selected so far.  An undecided point q is *dominant* when no undecided
// point of larger key lies at squared distance < v(q).  Then v(q) is final:
// no point that ends up before q can come closer than v(q) -- the first such
// point would have to be selected while q, of larger key, is still
// available.  All dominant points of a round are selected together.  A
// selected p then lowers v(q) := min(v(q), d2(p,q)) for undecided q of
// smaller key; undecided q of larger key are left alone, which is exact: q
// was within reach of p only if d2(p,q) >= v(p), and if q later falls below
// p its value is already below d2(p,q).
//
// Rounds run in bands of keys: with vmax the largest undecided v, the band
// holds the undecided points with v >= vmax/4 (KC_ORDER_BAND); only band points can dominate
// band points, so the dominance search uses a grid of band points with cell
// size sqrt(vmax).  The updates scan a fixed fine grid of all points.
// Finally the points are sorted by (v descending, index ascending).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "grid.cuh"

namespace kc {

__global__ void finite_check_k(const double* __restrict__ x, int64_t n, int* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) atomicExch(bad, 1);
}

kc_status check_finite(const double* x, int64_t n, Arena& A, cudaStream_t s) {
    int* bad;
    KC_TRY(A.get(&bad, 1));
    KC_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    ::kc::note_launch(), finite_check_k<<<blocks_for(n, 256), 256, 0, s>>>(x, n, bad);
    KC_CUDA(cudaGetLastError());
    int h = 0;
    KC_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (h) return fail(KC_EINVAL, "points must be finite");
    return KC_OK;
}

// out[q] = rows ids[q] of the n x w array a
__global__ void gather_rows_k(const double* __restrict__ a, int w, const int32_t* __restrict__ ids, int64_t n,
                              double* __restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n)
        for (int t = 0; t < w; ++t) out[q * w + t] = a[(int64_t)ids[q] * w + t];
}

// state in grid order (gpos): coordinates xg, original index idg, v2, stat
__global__ void ord_init_k(const double* __restrict__ x, int d, const int32_t* __restrict__ gsorted, int64_t N,
                           double* __restrict__ xg, int32_t* __restrict__ idg, double* __restrict__ v2,
                           int* __restrict__ stat, Origin org, float* __restrict__ xgf) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N) return;
    int64_t id = gsorted[q];
    for (int t = 0; t < d; ++t) {
        xg[q * d + t] = x[id * d + t];
        if (xgf) xgf[q * d + t] = (float)(x[id * d + t] - org.lo[t]);
    }
    idg[q] = (int32_t)id;
    if (id == 0) {
        v2[q] = INFINITY;
        stat[q] = 1;
    } else {
        v2[q] = dist2_exact(x + id * d, x, d);
        stat[q] = 0;
    }
}

// max of v2 over undecided points and their count
__global__ void ord_vmax_k(const double* __restrict__ v2, const int* __restrict__ stat, int64_t N,
                           unsigned long long* __restrict__ vmax_bits, unsigned long long* __restrict__ count) {
    unsigned long long m = 0, c = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
        if (stat[q] == 0) {
            m = max(m, (unsigned long long)__double_as_longlong(v2[q]));
            c++;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane_id() == 0) {
        atomicMax(vmax_bits, m);
        atomicAdd(count, c);
    }
}

__global__ void ord_band_k(const double* __restrict__ v2, const int* __restrict__ stat, int64_t N, double T,
                           int32_t* __restrict__ blist, unsigned long long* __restrict__ nb) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < N && stat[q] == 0 && v2[q] >= T) blist[atomicAdd(nb, 1ULL)] = (int32_t)q;
}

// per band cell: the largest squared distance (as bits) of its undecided band
// points, -1 if none; a dominance scan skips the cells whose largest value is
// below its own (no point of larger key there)
__global__ void ord_cellmax_k(const int32_t* __restrict__ bsorted, const int64_t* __restrict__ bstart,
                              int64_t ncells, const double* __restrict__ v2, const int* __restrict__ stat,
                              long long* __restrict__ cmax) {
    const int64_t cidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cidx >= ncells) return;
    long long m = -1;
    const long long* __restrict__ v2b = (const long long*)v2;
    for (int64_t f = bstart[cidx]; f < bstart[cidx + 1]; ++f) {
        const int p = bsorted[f];
        if (stat[p] == 0) m = max(m, v2b[p]);
    }
    cmax[cidx] = m;
}

#ifndef KC_DOM_BUDGET
#define KC_DOM_BUDGET 256
#endif
constexpr int DOM_THREAD_BUDGET = KC_DOM_BUDGET;

// One thread per band point: is it dominant?  Most band points meet a
// dominator among their first candidates; a point whose scan would go past
// DOM_THREAD_BUDGET candidates (an undominated point has to look at every
// band point within sqrt(v)) is handed, undecided, to ord_dominance_warp_k.
__global__ void ord_dominance_k(Grid gb, const int32_t* __restrict__ bsorted, const int64_t* __restrict__ bstart,
                                int64_t nb, const double* __restrict__ xg, int d, const int32_t* __restrict__ idg,
                                const double* __restrict__ v2, const int* __restrict__ stat, double T,
                                int32_t* __restrict__ sel, unsigned long long* __restrict__ nsel,
                                unsigned long long* __restrict__ nactive, const float* __restrict__ xgf,
                                float delta, const long long* __restrict__ cmax, const double* __restrict__ gxg,
                                int gs, int32_t* __restrict__ hard, unsigned long long* __restrict__ nhard) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    const int q = bsorted[e];
    if (stat[q] != 0) return;
    const double vq = v2[q];
    if (!(vq >= T)) return;
    const long long bq = __double_as_longlong(vq);
    const long long* __restrict__ v2b = (const long long*)v2;
    atomicAdd(nactive, 1ULL);
    const double* xq = xg + (int64_t)q * d;
    const float rq = sqrtf((float)vq);
    const int idq = idg[q];
    const double R = sqrt(vq);
    // Scan the band grid ring by ring outward from q's cell, so a dominated
    // point usually meets a dominator within the first rings; ring r holds no
    // point closer than (r-1) cells.
    const int dg = gb.dg;
    int c[3] = {0, 0, 0};
    int maxr = 0;
    for (int t = 0; t < dg; ++t) {
        c[t] = cell_coord(gb, gxg[(int64_t)q * gs + t], t);
        maxr = max(maxr, span_for(gb, R, t));
    }
    bool dom = true;
    int budget = DOM_THREAD_BUDGET;  // candidates this thread examines before handing q to a warp
    for (int r = 0; r <= maxr && dom; ++r) {
        if (r >= 2 && (double)(r - 1) * gb.c > R) break;
        const int z0 = dg > 2 ? max(0, c[2] - r) : 0, z1 = dg > 2 ? min(gb.n[2] - 1, c[2] + r) : 0;
        const int y0 = dg > 1 ? max(0, c[1] - r) : 0, y1 = dg > 1 ? min(gb.n[1] - 1, c[1] + r) : 0;
        for (int cz = z0; cz <= z1 && dom; ++cz)
            for (int cy = y0; cy <= y1 && dom; ++cy) {
                const bool edge = r == 0 || (dg > 2 && abs(cz - c[2]) == r) || (dg > 1 && abs(cy - c[1]) == r);
                const int64_t base = ((int64_t)cz * gb.n[1] + cy) * gb.n[0];
                // the cells of this ring in the row: all of [c-r, c+r] on an edge row, else the two ends
                int seg[2][2];
                int nseg = 0;
                if (edge) {
                    seg[0][0] = max(0, c[0] - r);
                    seg[0][1] = min(gb.n[0] - 1, c[0] + r);
                    nseg = 1;
                } else {
                    if (c[0] - r >= 0) {
                        seg[nseg][0] = seg[nseg][1] = c[0] - r;
                        ++nseg;
                    }
                    if (c[0] + r <= gb.n[0] - 1) {
                        seg[nseg][0] = seg[nseg][1] = c[0] + r;
                        ++nseg;
                    }
                }
                for (int sg = 0; sg < nseg && dom; ++sg)
                    for (int cx = seg[sg][0]; cx <= seg[sg][1] && dom; ++cx) {
                        if (cmax[base + cx] < bq) continue;  // no larger key in this cell
                        const int64_t f0 = bstart[base + cx], f1 = bstart[base + cx + 1];
                        if (f1 - f0 > budget) {  // too many candidates left for one thread
                            hard[atomicAdd(nhard, 1ULL)] = q;
                            return;
                        }
                        budget -= (int)(f1 - f0);
                        for (int64_t f = f0; f < f1; ++f) {
                            const int p = bsorted[f];
                            if (p == q || stat[p] != 0) continue;
                            const long long bp = v2b[p];
                            if (bp > bq || (bp == bq && idg[p] < idq)) {
                                if (xgf && screen_f32(xgf + (int64_t)p * d, xgf + (int64_t)q * d, d, rq, delta) == 0)
                                    continue;  // surely farther than sqrt(vq)
                                if (dist2_exact(xg + (int64_t)p * d, xq, d) < vq) {
                                    dom = false;
                                    break;
                                }
                            }
                        }
                    }
            }
    }
    if (dom) sel[atomicAdd(nsel, 1ULL)] = q;
}

// The points the threads handed over, one warp each (grid-stride over the
// list): the same scan in the same ring and cell order, a cell's points 32 at
// a time, so a long scan costs a 32nd of a serial one (with a thread per
// point those few scans were the whole duration of a round).
__global__ void ord_dominance_warp_k(Grid gb, const int32_t* __restrict__ hard,
                                     const unsigned long long* __restrict__ nhard, const int64_t* __restrict__ bstart,
                                     const int32_t* __restrict__ bsorted, const double* __restrict__ xg, int d,
                                     const int32_t* __restrict__ idg, const double* __restrict__ v2,
                                     const int* __restrict__ stat, int32_t* __restrict__ sel,
                                     unsigned long long* __restrict__ nsel, const float* __restrict__ xgf, float delta,
                                     const long long* __restrict__ cmax, const double* __restrict__ gxg, int gs) {
    const int lane = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nh = (int64_t)*nhard;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nh; e += nw) {
        const int q = hard[e];
        const double vq = v2[q];
        const long long bq = __double_as_longlong(vq);
        const long long* __restrict__ v2b = (const long long*)v2;
        const double* xq = xg + (int64_t)q * d;
        const float rq = sqrtf((float)vq);
        const int idq = idg[q];
        const double R = sqrt(vq);
        const int dg = gb.dg;
        int c[3] = {0, 0, 0};
        int maxr = 0;
        for (int t = 0; t < dg; ++t) {
            c[t] = cell_coord(gb, gxg[(int64_t)q * gs + t], t);
            maxr = max(maxr, span_for(gb, R, t));
        }
        bool dom = true;  // uniform across the warp
        for (int r = 0; r <= maxr && dom; ++r) {
            if (r >= 2 && (double)(r - 1) * gb.c > R) break;
            const int z0 = dg > 2 ? max(0, c[2] - r) : 0, z1 = dg > 2 ? min(gb.n[2] - 1, c[2] + r) : 0;
            const int y0 = dg > 1 ? max(0, c[1] - r) : 0, y1 = dg > 1 ? min(gb.n[1] - 1, c[1] + r) : 0;
            for (int cz = z0; cz <= z1 && dom; ++cz)
                for (int cy = y0; cy <= y1 && dom; ++cy) {
                    const bool edge = r == 0 || (dg > 2 && abs(cz - c[2]) == r) || (dg > 1 && abs(cy - c[1]) == r);
                    const int64_t base = ((int64_t)cz * gb.n[1] + cy) * gb.n[0];
                    int seg[2][2];
                    int nseg = 0;
                    if (edge) {
                        seg[0][0] = max(0, c[0] - r);
                        seg[0][1] = min(gb.n[0] - 1, c[0] + r);
                        nseg = 1;
                    } else {
                        if (c[0] - r >= 0) {
                            seg[nseg][0] = seg[nseg][1] = c[0] - r;
                            ++nseg;
                        }
                        if (c[0] + r <= gb.n[0] - 1) {
                            seg[nseg][0] = seg[nseg][1] = c[0] + r;
                            ++nseg;
                        }
                    }
                    for (int sg = 0; sg < nseg && dom; ++sg)
                        for (int cx = seg[sg][0]; cx <= seg[sg][1] && dom; ++cx) {
                            if (cmax[base + cx] < bq) continue;  // no larger key in this cell
                            const int64_t f0 = bstart[base + cx], f1 = bstart[base + cx + 1];
                            for (int64_t fb = f0; fb < f1 && dom; fb += 32) {
                                bool hit = false;
                                const int64_t f = fb + lane;
                                if (f < f1) {
                                    const int p = bsorted[f];
                                    if (p != q && stat[p] == 0) {
                                        const long long bp = v2b[p];
                                        if (bp > bq || (bp == bq && idg[p] < idq)) {
                                            const bool far = xgf && screen_f32(xgf + (int64_t)p * d, xgf + (int64_t)q * d,
                                                                               d, rq, delta) == 0;
                                            hit = !far && dist2_exact(xg + (int64_t)p * d, xq, d) < vq;
                                        }
                                    }
                                }
                                if (__any_sync(0xffffffffu, hit)) dom = false;
                            }
                        }
                }
        }
        if (dom && lane == 0) sel[atomicAdd(nsel, 1ULL)] = q;
    }
}

// ---- greedy steps for the coarsest points: each step selects the argmax of
// the previous step's per-block candidates and pushes it to every point.
constexpr int GREEDY_BLOCKS_PER_SM = 4;
#ifndef KC_GREEDY_STEPS
#define KC_GREEDY_STEPS 256
#endif
constexpr int64_t GREEDY_STEPS = KC_GREEDY_STEPS;  // coarsest points selected one at a time
// A band holds the undecided points with v >= KC_ORDER_BAND * (largest v).
#ifndef KC_ORDER_BAND
#define KC_ORDER_BAND 0.25
#endif

// Keys compare on the bit patterns of the squared distances: for v >= 0
// (and +inf) IEEE doubles order like their bits as integers, and integer
// compares stay off the GB300's small FP64 pipe.
__device__ __forceinline__ long long vbits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ bool key_above(double va, int ia, double vb, int ib) {
    const long long a = vbits(va), b = vbits(vb);
    return a > b || (a == b && ia < ib);
}

// per-block best (v2 desc, original index asc) over undecided points; cand_g = -1 if none
__device__ void block_best(double v, int id, int g, double* sv, int* si, int* sg, double* out_v, int* out_i,
                           int* out_g) {
    for (int o = 16; o > 0; o >>= 1) {
        double v2o = __shfl_xor_sync(0xffffffffu, v, o);
        int i2 = __shfl_xor_sync(0xffffffffu, id, o);
        int g2 = __shfl_xor_sync(0xffffffffu, g, o);
        if (g2 >= 0 && (g < 0 || key_above(v2o, i2, v, id))) {
            v = v2o;
            id = i2;
            g = g2;
        }
    }
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) {
        sv[w] = v;
        si[w] = id;
        sg[w] = g;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
            if (sg[q] >= 0 && (g < 0 || key_above(sv[q], si[q], v, id))) {
                v = sv[q];
                id = si[q];
                g = sg[q];
            }
        *out_v = v;
        *out_i = id;
        *out_g = g;
    }
}

// A grid-wide barrier for a cooperative launch (every block resident): the
// last block to arrive resets the count and advances the generation; the
// others poll the generation with backoff, at most `limit` cycles, after
// which (or when another block has failed) the status word is set and false
// returned.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, int* status, long long limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = ld_acquire_u32(gen);
        fence_acq_rel_gpu();  // this block's writes before its arrival
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            *count = 0u;
            fence_acq_rel_gpu();
            red_release_add_u32(gen, 1u);
        } else {
            const long long t0 = clock64();
            unsigned ns = 32;
            while (ld_acquire_u32(gen) == g) {
                if (clock64() - t0 > limit || ld_volatile_s32(status) != 0) {
                    atomicCAS(status, 0, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
            }
        }
        fence_acq_rel_gpu();  // acquire: the other blocks' writes
    }
    __syncthreads();
    return ok != 0;
}

// All greedy steps in one cooperative launch: phase 0 leaves every block's
// candidate (no winner yet); phase k >= 1 takes the winner of phase k-1's
// candidates (every block computes the same), marks it, pushes it to the
// block's points and leaves the block's new candidate.  The candidates
// alternate between two buffers; a grid barrier separates the phases.
__global__ void ord_greedy_loop_k(const double* __restrict__ xg, int d, const int32_t* __restrict__ idg,
                                  double* __restrict__ v2, int* __restrict__ stat, int64_t N, int64_t steps,
                                  double* pv0, int* pi0, int* pg0, double* pv1, int* pi1, int* pg1,
                                  const float* __restrict__ xgf, float delta, unsigned* bar, int* status,
                                  long long limit) {
    __shared__ double sv[32];
    __shared__ int si[32], sg[32];
    __shared__ double s_wv;
    __shared__ int s_wi, s_wg;
    const int nin = gridDim.x;
    for (int64_t k = 0; k <= steps; ++k) {
        const double* pv_in = (k & 1) ? pv0 : pv1;
        const int* pi_in = (k & 1) ? pi0 : pi1;
        const int* pg_in = (k & 1) ? pg0 : pg1;
        double* pv_out = (k & 1) ? pv1 : pv0;
        int* pi_out = (k & 1) ? pi1 : pi0;
        int* pg_out = (k & 1) ? pg1 : pg0;
        {
            double v = 0;
            int i = 0, g = -1;
            if (k > 0)
                for (int b = threadIdx.x; b < nin; b += blockDim.x) {
                    const int gb = __ldcg(&pg_in[b]);
                    const double vb = __ldcg(&pv_in[b]);
                    const int ib = __ldcg(&pi_in[b]);
                    if (gb >= 0 && (g < 0 || key_above(vb, ib, v, i))) {
                        v = vb;
                        i = ib;
                        g = gb;
                    }
                }
            block_best(v, i, g, sv, si, sg, &s_wv, &s_wi, &s_wg);
        }
        __syncthreads();
        const int w = s_wg;
        if (w >= 0 && blockIdx.x == 0 && threadIdx.x == 0) stat[w] = 1;  // v2[w] keeps its final value l^2
        double bv = 0;
        int bi = 0, bg = -1;
        const double* xw = w >= 0 ? xg + (int64_t)w * d : nullptr;
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
            if (q == w || __ldcg(&stat[q]) != 0) continue;
            double vq = v2[q];
            if (w >= 0 &&
                !(xgf && screen_f32(xgf + q * d, xgf + (int64_t)w * d, d, sqrtf((float)vq), delta) == 0)) {
                const double dd = dist2_exact(xg + q * d, xw, d);
                if (dd < vq) {
                    vq = dd;
                    v2[q] = dd;
                }
            }
            const int iq = idg[q];
            if (bg < 0 || key_above(vq, iq, bv, bi)) {
                bv = vq;
                bi = iq;
                bg = (int)q;
            }
        }
        __syncthreads();  // sv/si/sg are reused
        block_best(bv, bi, bg, sv, si, sg, &pv_out[blockIdx.x], &pi_out[blockIdx.x], &pg_out[blockIdx.x]);
        if (k < steps && !grid_barrier(bar, bar + 1, status, limit)) return;
    }
}

__global__ void ord_mark_k(const int32_t* __restrict__ sel, int64_t ns, int* __restrict__ stat) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ns) stat[sel[k]] = 1;
}

// cell-rows of the fine grid covered by the update ball of each selected
// point: the box is computed once per point (query_box) and kept in sbox
__global__ void ord_items_k(Grid g, const int32_t* __restrict__ sel, int64_t ns, const double* __restrict__ gxg,
                            int gs, const double* __restrict__ v2, int64_t* __restrict__ cnt, int4* __restrict__ sbox) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const int p = sel[k];
    const int4 b = query_box(g, gxg + (int64_t)p * gs, sqrt(v2[p]));
    sbox[k] = b;
    int lo[3], hi[3];
    box_range(g, b, lo, hi);
    cnt[k] = (int64_t)(hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
}
__global__ void ord_item_fill_k(const int64_t* __restrict__ off, int64_t ns, int32_t* __restrict__ item_sel) {
    int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= ns) return;
    for (int64_t t = off[k] + lane_id(); t < off[k + 1]; t += 32) item_sel[t] = (int32_t)k;
}

// one warp per (selected point, cell-row): lower v2 of undecided points of smaller key
__global__ void ord_update_k(Grid g, const int32_t* __restrict__ sel, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ item_sel, int64_t nitems, const int64_t* __restrict__ cstart,
                             const double* __restrict__ xg, int d, const int32_t* __restrict__ idg,
                             double* __restrict__ v2, const int* __restrict__ stat, const float* __restrict__ xgf,
                             float delta, const int4* __restrict__ sbox) {
    int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (it >= nitems) return;
    const int lane = lane_id();
    const int k = item_sel[it];
    const int p = sel[k];
    const double* xp = xg + (int64_t)p * d;
    const double vp = v2[p];  // final value of the selected point
    const int idp = idg[p];
    int lo[3], hi[3];
    box_range(g, sbox[k], lo, hi);
    int64_t r = it - off[k];
    const int ny = hi[1] - lo[1] + 1;
    const int cy = lo[1] + (int)(r % ny);
    const int cz = lo[2] + (int)(r / ny);
    const int64_t base = ((int64_t)cz * g.n[1] + cy) * g.n[0];
    const int64_t a = cstart[base + lo[0]], b = cstart[base + hi[0] + 1];
    unsigned long long* vb = (unsigned long long*)v2;
    for (int64_t q = a + lane; q < b; q += 32) {
        if (stat[q] != 0) continue;
        const double vq = v2[q];
        if (!(vq < vp || (vq == vp && idg[q] > idp))) continue;
        if (xgf && screen_f32(xgf + q * d, xgf + (int64_t)p * d, d, sqrtf((float)vq), delta) == 0) continue;
        const double dd = dist2_exact(xg + q * d, xp, d);
        if (dd < vq) atomicMin(vb + q, (unsigned long long)__double_as_longlong(dd));
    }
}

__global__ void ord_keys_k(const double* __restrict__ v2, const int32_t* __restrict__ idg, int64_t N,
                           uint64_t* __restrict__ key, int64_t* __restrict__ val) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N) return;
    int64_t id = idg[q];
    key[id] = ~(uint64_t)__double_as_longlong(v2[q]);
    val[id] = id;
}

__global__ void ord_out_k(const uint64_t* __restrict__ skey, const int64_t* __restrict__ sval, const double* __restrict__ x,
                          int64_t N, int d, int32_t* __restrict__ perm, double* __restrict__ l,
                          double* __restrict__ x_ord) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    int64_t id = sval[k];
    perm[k] = (int32_t)id;
    double v = __longlong_as_double((long long)~skey[k]);
    l[k] = __dsqrt_rn(v);
    for (int t = 0; t < d; ++t) x_ord[k * d + t] = x[id * d + t];
}

kc_status order_impl(const double* x, int64_t N, int d, int32_t* perm, double* l, double* x_ord, cudaStream_t s) {
    Arena A(s);
    KC_TRY(check_finite(x, N * d, A, s));
    // grid coordinates: the points (d <= 3) or their principal-axes projections
    const double* gx;
    int gs;
    KC_TRY(grid_coords(x, N, d, A, s, &gx, &gs));
    double lo[3], hi[3];
    KC_TRY(bbox(gx, N, gs, lo, hi, A, s));
    // fine grid of all points, about two points per cell
    Grid g0 = make_grid(gs, lo, hi, N, 0.0, N / 2 > 1 ? N / 2 : 1);
    int32_t* gsorted;
    int64_t* cstart;
    KC_TRY(A.get(&gsorted, N));
    KC_TRY(A.get(&cstart, g0.ncells + 1));
    KC_TRY(grid_build(g0, gx, gs, nullptr, N, gsorted, cstart, A, s));

    double *xg, *v2;
    int32_t *idg, *blist, *bsorted, *sel, *item_sel;
    int* stat;
    int64_t *bstart, *icnt, *ioff;
    unsigned long long* ctr;  // [0] vmax bits [1] undecided [2] nb [3] nsel [4] nactive [5] handed to warps
    KC_TRY(A.get(&xg, N * d));
    KC_TRY(A.get(&v2, N));
    KC_TRY(A.get(&idg, N));
    KC_TRY(A.get(&stat, N));
    KC_TRY(A.get(&blist, N));
    KC_TRY(A.get(&bsorted, N));
    KC_TRY(A.get(&sel, N));
    int32_t* hard;  // band points handed from the thread scan to the warp scan
    KC_TRY(A.get(&hard, N));
    KC_TRY(A.get(&icnt, N));
    int4* sbox;
    KC_TRY(A.get(&sbox, N));
    KC_TRY(A.get(&ioff, N + 1));
    KC_TRY(A.get(&bstart, 2 * N + 2));
    long long* cmax;  // per band cell (at most 2 N + 1 cells)
    KC_TRY(A.get(&cmax, 2 * N + 2));
    KC_TRY(A.get(&ctr, 8));
    // float copy of the coordinates (minus the box corner) for FP32 screens of
    // the distance tests; exact FP64 tests decide every close call
    float* xgf = nullptr;
    Origin org;
    double E = 0.0;
    KC_TRY(bbox_all(x, N, d, &org, &E, A, s));
    const float delta = (float)(E * 1.1920928955078125e-07);  // 2^-23 E
    KC_TRY(A.get(&xgf, N * d));
    ::kc::note_launch(), ord_init_k<<<blocks_for(N, 256), 256, 0, s>>>(x, d, gsorted, N, xg, idg, v2, stat, org, xgf);
    // grid coordinates in grid order
    const double* gxg = xg;
    if (gx != x) {
        double* p;
        KC_TRY(A.get(&p, (size_t)N * gs));
        ::kc::note_launch(), gather_rows_k<<<blocks_for(N, 256), 256, 0, s>>>(gx, gs, gsorted, N, p);
        gxg = p;
    }
    KC_CUDA(cudaGetLastError());
    int64_t item_cap = 0;
    item_sel = nullptr;
    const int sms = sm_count();

    // Greedy phase: the coarsest points are selected one at a time (every
    // step updates every point), because while few points are selected the
    // update balls cover the whole cloud and the band rounds would be
    // quadratic.  All steps run in one cooperative launch with a grid barrier
    // between them.
    {
        int per_sm = 0;
        KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ord_greedy_loop_k, 256, 0));
        const int nblk = sms * std::max(1, std::min(per_sm, GREEDY_BLOCKS_PER_SM));
        double* pv[2];
        int *pi[2], *pg[2];
        for (int k = 0; k < 2; ++k) {
            KC_TRY(A.get(&pv[k], nblk));
            KC_TRY(A.get(&pi[k], nblk));
            KC_TRY(A.get(&pg[k], nblk));
        }
        unsigned* bar;
        int* gst;
        KC_TRY(A.get(&bar, 2));
        KC_TRY(A.get(&gst, 1));
        KC_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
        KC_CUDA(cudaMemsetAsync(gst, 0, sizeof(int), s));
        int64_t steps = N - 1 < GREEDY_STEPS ? N - 1 : GREEDY_STEPS;
        const double* a_xg = xg;
        const int32_t* a_idg = idg;
        const float* a_xgf = xgf;
        long long limit = 4000000000LL;
        void* args[] = {(void*)&a_xg, (void*)&d, (void*)&a_idg, (void*)&v2, (void*)&stat, (void*)&N, (void*)&steps,
                        (void*)&pv[0], (void*)&pi[0], (void*)&pg[0], (void*)&pv[1], (void*)&pi[1], (void*)&pg[1],
                        (void*)&a_xgf, (void*)&delta, (void*)&bar, (void*)&gst, (void*)&limit};
        ::kc::note_launch();
        KC_CUDA(cudaLaunchCooperativeKernel((const void*)ord_greedy_loop_k, dim3(nblk), dim3(256), args, 0, s));
        int hst = 0;
        KC_CUDA(cudaMemcpyAsync(&hst, gst, sizeof(int), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        if (hst != 0) return fail(KC_ETIMEOUT, "ordering: a grid barrier of the greedy phase ran out");
    }
    int rounds = 0;
    const bool stats = getenv("KC_ORDER_STATS") != nullptr;
    for (;;) {
        KC_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), s));
        ::kc::note_launch(), ord_vmax_k<<<sms * 4, 256, 0, s>>>(v2, stat, N, ctr, ctr + 1);
        unsigned long long h[2];
        KC_CUDA(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        if (h[1] == 0) break;
        double vmax;
        memcpy(&vmax, &h[0], sizeof(double));
        const double T = vmax * KC_ORDER_BAND;
        KC_CUDA(cudaMemsetAsync(ctr + 2, 0, sizeof(unsigned long long), s));
        ::kc::note_launch(), ord_band_k<<<blocks_for(N, 256), 256, 0, s>>>(v2, stat, N, T, blist, ctr + 2);
        unsigned long long hnb = 0;
        KC_CUDA(cudaMemcpyAsync(&hnb, ctr + 2, sizeof(hnb), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        const int64_t nb = (int64_t)hnb;
        // band cells a quarter of the largest search radius (bounded by the
        // cell budget), scanned nearest ring first
        Grid gb = make_grid(gs, lo, hi, nb, vmax > 0 ? 0.25 * sqrt(vmax) : 0.0, 2 * nb + 1);
        {
            Arena B(s);
            int64_t* bst;
            KC_TRY(B.get(&bst, gb.ncells + 1));
            KC_TRY(grid_build(gb, gxg, gs, blist, nb, bsorted, bst, B, s));
            KC_CUDA(cudaMemcpyAsync(bstart, bst, sizeof(int64_t) * (gb.ncells + 1), cudaMemcpyDeviceToDevice, s));
        }
        const int band_r0 = rounds;
        const auto band_t0 = std::chrono::steady_clock::now();
        int64_t band_sel = 0, band_items = 0;
        for (;;) {
            if (++rounds > 1000000) return fail(KC_ECUDA, "ordering: too many rounds");
            KC_CUDA(cudaMemsetAsync(ctr + 3, 0, 3 * sizeof(unsigned long long), s));
            ::kc::note_launch(), ord_cellmax_k<<<blocks_for(gb.ncells, 256), 256, 0, s>>>(bsorted, bstart, gb.ncells, v2,
                                                                                         stat, cmax);
            ::kc::note_launch(), ord_dominance_k<<<blocks_for(nb, 128), 128, 0, s>>>(
                gb, bsorted, bstart, nb, xg, d, idg, v2, stat, T, sel, ctr + 3, ctr + 4, xgf, delta, cmax, gxg, gs, hard,
                ctr + 5);
            ::kc::note_launch(), ord_dominance_warp_k<<<sms * 8, 256, 0, s>>>(
                gb, hard, ctr + 5, bstart, bsorted, xg, d, idg, v2, stat, sel, ctr + 3, xgf, delta, cmax, gxg, gs);
            unsigned long long hs[2];
            KC_CUDA(cudaMemcpyAsync(hs, ctr + 3, sizeof(hs), cudaMemcpyDeviceToHost, s));
            KC_CUDA(cudaStreamSynchronize(s));
            const int64_t ns = (int64_t)hs[0];
            if (hs[1] == 0) {  // band exhausted
                if (stats) {
                    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - band_t0)
                                    .count();
                    fprintf(stderr, "[kc order] vmax=%.3e band=%lld rounds=%d selected=%lld items=%lld ms=%.2f\n", vmax,
                            (long long)nb, rounds - band_r0 - 1, (long long)band_sel, (long long)band_items, ms);
                }
                break;
            }
            band_sel += (int64_t)hs[0];
            if (ns == 0) return fail(KC_ECUDA, "ordering: no dominant point in a nonempty band");
            ::kc::note_launch(), ord_mark_k<<<blocks_for(ns, 256), 256, 0, s>>>(sel, ns, stat);
            ::kc::note_launch(), ord_items_k<<<blocks_for(ns, 256), 256, 0, s>>>(g0, sel, ns, gxg, gs, v2, icnt, sbox);
            Arena R(s);  // per-round scratch of the scan
            KC_TRY(exclusive_scan_i64(icnt, ioff, ns, R, s));
            int64_t nitems = 0;
            KC_CUDA(cudaMemcpyAsync(&nitems, ioff + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            KC_CUDA(cudaStreamSynchronize(s));
            band_items += nitems;
            if (nitems > item_cap) {
                item_cap = nitems * 2;
                if (item_sel) cudaFreeAsync(item_sel, s);
                item_sel = nullptr;
                KC_TRY(scratch_alloc((void**)&item_sel, sizeof(int32_t) * item_cap, s));
            }
            ::kc::note_launch(), ord_item_fill_k<<<blocks_for(ns * 32, 256), 256, 0, s>>>(ioff, ns, item_sel);
            ::kc::note_launch(), ord_update_k<<<blocks_for(nitems * 32, 256), 256, 0, s>>>(g0, sel, ioff, item_sel, nitems, cstart, xg, d,
                                                                     idg, v2, stat, xgf, delta, sbox);
            KC_CUDA(cudaGetLastError());
        }
    }
    if (item_sel) cudaFreeAsync(item_sel, s);
    uint64_t *k0, *k1;
    int64_t *w0, *w1;
    KC_TRY(A.get(&k0, N));
    KC_TRY(A.get(&k1, N));
    KC_TRY(A.get(&w0, N));
    KC_TRY(A.get(&w1, N));
    ::kc::note_launch(), ord_keys_k<<<blocks_for(N, 256), 256, 0, s>>>(v2, idg, N, k0, w0);
    KC_TRY(radix_sort_u64_i64(k0, w0, k1, w1, N, 64, A, s));
    ::kc::note_launch(), ord_out_k<<<blocks_for(N, 256), 256, 0, s>>>(k1, w1, x, N, d, perm, l, x_ord);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaStreamSynchronize(s));
    return KC_OK;
}

}  // namespace kc
