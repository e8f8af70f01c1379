// a3: the sparsity pattern S_rho (Section 2.3) on the device.
//
// For positions i < j of the maximin order, (j,i) is in S iff
//   dist(x_i, x_j) <= rho * l[i]   (max rule: l is non-increasing), or
//   dist(x_i, x_j) <= rho * l[j]   (min rule),
// with dist = sqrt(d2) correctly rounded and the product correctly rounded,
// so membership is bit-identical to a CPU evaluation of the definition.
// The diagonal is always in S.
//
// Column-centric search: column i looks at the points within rho*l[i] of
// x_i (a superset for the min rule) through a fine grid of all points, one
// warp per (column, row of grid cells); the points of consecutive cells are
// contiguous in the cell-sorted order.  A count pass gives the row lengths,
// a fill pass scatters the column indices with atomics, and a sort of each
// row (bitonic, in shared memory) restores ascending order.
#include <cmath>

#include "grid.cuh"

namespace kc {

kc_status check_finite(const double* x, int64_t n, Arena& A, cudaStream_t s);

struct PatArgs {
    Grid g;
    const double* xs;      // coordinates in cell-sorted order
    const int32_t* ps;     // position of each sorted point
    const int64_t* cstart;
    const double* xo;      // coordinates by position
    const double* l;
    int d;
    double rho;
    int rule;
    const int64_t* off;    // item offsets per column
    const int32_t* item_col;
    int64_t nitems;
    const float* xsf;      // float copy of xs minus the box corner
    const float* xof;      // the same by position
    float delta;           // error bound of one float coordinate difference
    const int4* colbox;    // search box of every column (query_box)
};

__device__ __forceinline__ double col_radius(double rho, double li) {
    return isinf(li) ? INFINITY : __dmul_rn(rho, li);
}

// exact membership of (j,i), i < j, given the squared distance
__device__ __forceinline__ bool in_s(double d2, double R) {
    if (isinf(R)) return true;
    const double Rs = R * R;
    if (d2 > Rs * (1.0 + 1e-12)) return false;
    if (d2 < Rs * (1.0 - 1e-12)) return true;
    return __dsqrt_rn(d2) <= R;
}

__global__ void pat_items_k(Grid g, const double* __restrict__ gxo, int gst, const double* __restrict__ l, int64_t N,
                            double rho, int64_t* __restrict__ cnt, int4* __restrict__ colbox) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int4 b = query_box(g, gxo + i * gst, col_radius(rho, l[i]));
    colbox[i] = b;
    int lo[3], hi[3];
    box_range(g, b, lo, hi);
    cnt[i] = (int64_t)(hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
}
// item counts in the cell order of the grid (gs[q]: the column at cell rank q)
__global__ void pat_cell_counts_k(const int32_t* __restrict__ gs, const int64_t* __restrict__ cnt, int64_t N,
                                  int64_t* __restrict__ cq) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < N) cq[q] = cnt[gs[q]];
}
// the first item of every column, indexed by column
__global__ void pat_cell_offsets_k(const int32_t* __restrict__ gs, const int64_t* __restrict__ oq, int64_t N,
                                   int64_t* __restrict__ off) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < N) off[gs[q]] = oq[q];
    if (q == 0) off[N] = oq[N];
}
// the column of every item, columns in cell order
__global__ void pat_item_fill_cell_k(const int32_t* __restrict__ gs, const int64_t* __restrict__ oq, int64_t N,
                                     int32_t* __restrict__ item_col) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= N) return;
    const int32_t i = gs[q];
    for (int64_t t = oq[q] + lane_id(); t < oq[q + 1]; t += 32) item_col[t] = i;
}

template <bool FILL>
__global__ void pat_scan_k(PatArgs P, int* __restrict__ cnt, const int64_t* __restrict__ rowptr,
                           int32_t* __restrict__ col) {
    int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (it >= P.nitems) return;
    const int lane = lane_id();
    const int i = P.item_col[it];
    const double* xi = P.xo + (int64_t)i * P.d;
    const double li = P.l[i];
    const double R = col_radius(P.rho, li);
    int lo[3], hi[3];
    box_range(P.g, P.colbox[i], lo, hi);
    const int64_t r = it - P.off[i];
    const int ny = hi[1] - lo[1] + 1;
    const int cy = lo[1] + (int)(r % ny);
    const int cz = lo[2] + (int)(r / ny);
    const int64_t base = ((int64_t)cz * P.g.n[1] + cy) * P.g.n[0];
    const int64_t a = P.cstart[base + lo[0]], b = P.cstart[base + hi[0] + 1];
    const float* xif = P.xof + (int64_t)i * P.d;
    for (int64_t q = a + lane; q < b; q += 32) {
        const int j = P.ps[q];
        if (j <= i) continue;
        const double Rj = P.rule == KC_RULE_MIN ? col_radius(P.rho, P.l[j]) : R;
        if (!isinf(Rj)) {
            // FP32 screen first; the exact FP64 test only near the boundary
            const int sc = screen_f32(P.xsf + q * P.d, xif, P.d, (float)Rj, P.delta);
            if (sc == 0) continue;
            if (sc < 0 && !in_s(dist2_exact(P.xs + q * P.d, xi, P.d), Rj)) continue;
        }
        if (!FILL) {
            atomicAdd(&cnt[j], 1);
        } else {
            const int slot = atomicAdd(&cnt[j], 1);
            col[rowptr[j] + slot] = i;
        }
    }
}

// Candidate range [a, b) (cell-sorted positions) of work item it, and its column.
__device__ __forceinline__ int item_range(const PatArgs& P, int64_t it, int64_t& a, int64_t& b) {
    const int i = P.item_col[it];
    int lo[3], hi[3];
    box_range(P.g, P.colbox[i], lo, hi);
    const int64_t r = it - P.off[i];
    const int ny = hi[1] - lo[1] + 1;
    const int cy = lo[1] + (int)(r % ny);
    const int cz = lo[2] + (int)(r / ny);
    const int64_t base = ((int64_t)cz * P.g.n[1] + cy) * P.g.n[0];
    a = P.cstart[base + lo[0]];
    b = P.cstart[base + hi[0] + 1];
    return i;
}

// Membership of candidate q (cell-sorted position) in column i: the same
// tests as pat_scan_k.
__device__ __forceinline__ bool pat_member(const PatArgs& P, int i, const double* xi, const float* xif, double R,
                                           int64_t q, int& j) {
    j = P.ps[q];
    if (j <= i) return false;
    const double Rj = P.rule == KC_RULE_MIN ? col_radius(P.rho, P.l[j]) : R;
    if (isinf(Rj)) return true;
    const int sc = screen_f32(P.xsf + q * P.d, xif, P.d, (float)Rj, P.delta);
    if (sc == 0) return false;
    return sc > 0 || in_s(dist2_exact(P.xs + q * P.d, xi, P.d), Rj);
}

// chunks of 32 candidates of every item (the hit masks' layout)
__global__ void pat_chunks_k(PatArgs P, int64_t* __restrict__ nch) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= P.nitems) return;
    int64_t a, b;
    item_range(P, it, a, b);
    nch[it] = (b - a + 31) / 32;
}

// Search pass of the builder: one warp per item; the row counts as in the
// count pass, and every 32 candidates' memberships as one mask word.
__global__ void pat_mask_k(PatArgs P, const int64_t* __restrict__ moff, int* __restrict__ cnt,
                           uint32_t* __restrict__ masks) {
    const int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (it >= P.nitems) return;
    const int lane = lane_id();
    int64_t a, b;
    const int i = item_range(P, it, a, b);
    const double* xi = P.xo + (int64_t)i * P.d;
    const float* xif = P.xof + (int64_t)i * P.d;
    const double R = col_radius(P.rho, P.l[i]);
    uint32_t* m = masks + moff[it];
    for (int64_t q0 = a; q0 < b; q0 += 32) {
        const int64_t q = q0 + lane;
        int j = 0;
        const bool hit = q < b && pat_member(P, i, xi, xif, R, q, j);
        const unsigned w = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) m[(q0 - a) >> 5] = w;
        if (hit) atomicAdd(&cnt[j], 1);
    }
}

// Fill pass of the builder: the members from the masks, no distance tests.
__global__ void pat_mask_fill_k(PatArgs P, const int64_t* __restrict__ moff, const uint32_t* __restrict__ masks,
                                int* __restrict__ cnt, const int64_t* __restrict__ rowptr, int32_t* __restrict__ col) {
    const int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (it >= P.nitems) return;
    const int lane = lane_id();
    const int i = P.item_col[it];
    const int64_t c0 = moff[it], c1 = moff[it + 1];
    int64_t a, b;
    item_range(P, it, a, b);
    for (int64_t c = c0; c < c1; ++c) {
        const uint32_t w = masks[c];
        if ((w >> lane) & 1u) {
            const int j = P.ps[a + ((c - c0) << 5) + lane];
            const int slot = atomicAdd(&cnt[j], 1);
            col[rowptr[j] + slot] = i;
        }
    }
}

__global__ void pat_gather_k(const double* __restrict__ xo, const int32_t* __restrict__ gs, int64_t N, int d,
                             Origin org, double* __restrict__ xs, float* __restrict__ xsf, float* __restrict__ xof) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < N)
        for (int t = 0; t < d; ++t) {
            const double v = xo[(int64_t)gs[q] * d + t];
            xs[q * d + t] = v;
            xsf[q * d + t] = (float)(v - org.lo[t]);
            xof[q * d + t] = (float)(xo[q * d + t] - org.lo[t]);
        }
}
__global__ void plus_one_k(const int* __restrict__ c, int64_t N, int32_t* __restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) out[j] = c[j] + 1;
}

// Shared setup of both passes: grid, cell-sorted coordinates, work items.
struct PatSetup {
    Grid g;
    int32_t* gs;
    int64_t* cstart;
    double* xs;
    int64_t* off;
    int32_t* item_col;
    int64_t nitems;
    int4* colbox = nullptr;
    float* xsf = nullptr;
    float* xof = nullptr;
    float delta = 0.f;
};

static kc_status pat_setup(const double* xo, const double* l, int64_t N, int d, double rho, PatSetup& S, Arena& A,
                           cudaStream_t s) {
    KC_TRY(check_finite(xo, N * d, A, s));
    // grid coordinates: the points (d <= 3) or their principal-axes projections
    const double* gxo;
    int gst;
    KC_TRY(grid_coords(xo, N, d, A, s, &gxo, &gst));
    double lo[3], hi[3];
    KC_TRY(bbox(gxo, N, gst, lo, hi, A, s));
    S.g = make_grid(gst, lo, hi, N, 0.0, N / 2 > 1 ? N / 2 : 1);
    Origin org;
    double E = 0.0;
    KC_TRY(bbox_all(xo, N, d, &org, &E, A, s));
    S.delta = (float)(E * 1.1920928955078125e-07);  // 2^-23 E
    KC_TRY(A.get(&S.xsf, N * d));
    KC_TRY(A.get(&S.xof, N * d));
    KC_TRY(A.get(&S.gs, N));
    KC_TRY(A.get(&S.cstart, S.g.ncells + 1));
    KC_TRY(grid_build(S.g, gxo, gst, nullptr, N, S.gs, S.cstart, A, s));
    KC_TRY(A.get(&S.xs, N * d));
    ::kc::note_launch(), pat_gather_k<<<blocks_for(N, 256), 256, 0, s>>>(xo, S.gs, N, d, org, S.xs, S.xsf, S.xof);
    int64_t* cnt;
    KC_TRY(A.get(&cnt, N));
    KC_TRY(A.get(&S.off, N + 1));
    KC_TRY(A.get(&S.colbox, N));
    ::kc::note_launch(), pat_items_k<<<blocks_for(N, 256), 256, 0, s>>>(S.g, gxo, gst, l, N, rho, cnt, S.colbox);
    KC_CUDA(cudaGetLastError());
    // The work items go column by column in the grid's cell order (neighbouring columns next to each
    // other), so that the rows a stretch of items writes into are few and stay in L2 meanwhile; off[i]
    // stays indexed by column.
    int64_t *cq, *oq;
    KC_TRY(A.get(&cq, N));
    KC_TRY(A.get(&oq, N + 1));
    ::kc::note_launch(), pat_cell_counts_k<<<blocks_for(N, 256), 256, 0, s>>>(S.gs, cnt, N, cq);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i64(cq, oq, N, A, s));
    ::kc::note_launch(), pat_cell_offsets_k<<<blocks_for(N, 256), 256, 0, s>>>(S.gs, oq, N, S.off);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaMemcpyAsync(&S.nitems, oq + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    KC_TRY(A.get(&S.item_col, S.nitems));
    ::kc::note_launch(), pat_item_fill_cell_k<<<blocks_for(N * 32, 256), 256, 0, s>>>(S.gs, oq, N, S.item_col);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

static PatArgs pat_args(const PatSetup& S, const double* xo, const double* l, int d, double rho, int rule) {
    PatArgs P;
    P.g = S.g;
    P.xs = S.xs;
    P.ps = S.gs;
    P.cstart = S.cstart;
    P.xo = xo;
    P.l = l;
    P.d = d;
    P.rho = rho;
    P.rule = rule;
    P.off = S.off;
    P.item_col = S.item_col;
    P.nitems = S.nitems;
    P.xsf = S.xsf;
    P.xof = S.xof;
    P.delta = S.delta;
    P.colbox = S.colbox;
    return P;
}

kc_status pattern_count_impl(const double* xo, const double* l, int64_t N, int d, double rho, int rule,
                             int64_t* rowptr, int64_t* nnz_out, cudaStream_t s) {
    Arena A(s);
    PatSetup S;
    KC_TRY(pat_setup(xo, l, N, d, rho, S, A, s));
    int* cnt;
    int32_t* len;
    KC_TRY(A.get(&cnt, N));
    KC_TRY(A.get(&len, N));
    KC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * N, s));
    PatArgs P = pat_args(S, xo, l, d, rho, rule);
    if (S.nitems > 0) ::kc::note_launch(), pat_scan_k<false><<<blocks_for(S.nitems * 32, 256), 256, 0, s>>>(P, cnt, nullptr, nullptr);
    ::kc::note_launch(), plus_one_k<<<blocks_for(N, 256), 256, 0, s>>>(cnt, N, len);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i32_to_i64(len, rowptr, N, A, s));
    int64_t nnz = 0;
    KC_CUDA(cudaMemcpyAsync(&nnz, rowptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (nnz_out) *nnz_out = nnz;
    return KC_OK;
}

// ---- per-row sort (ascending), the diagonal appended last
constexpr int SORT_WARP_CAP = 1024;
constexpr int SORT_BLOCK_CAP = 16384;

// Bitonic sort of 32*E keys held E per lane (element t = lane*E + r):
// compare-exchanges at distance >= E go through shfl_xor, shorter ones
// between a lane's own registers.  The keys of a row are distinct.
template <int E>
__device__ __forceinline__ void warp_bitonic(int (&v)[E], int lane) {
    for (int k = 2; k <= 32 * E; k <<= 1) {
        for (int jj = k >> 1; jj >= E; jj >>= 1) {  // partners in other lanes
            const int lm = jj / E;
            const bool lower = (lane & lm) == 0;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int pv = __shfl_xor_sync(0xffffffffu, v[r], lm);
                const bool up = ((lane * E + r) & k) == 0;
                v[r] = (lower == up) ? min(v[r], pv) : max(v[r], pv);
            }
        }
#pragma unroll
        for (int jb = E / 2; jb >= 1; jb >>= 1) {  // partners in this lane (compile-time distances)
            if (jb < k)
#pragma unroll
                for (int r = 0; r < E; ++r)
                    if ((r & jb) == 0) {
                        const bool up = ((lane * E + r) & k) == 0;
                        const int x0 = v[r], x1 = v[r | jb];
                        if ((x0 > x1) == up) {
                            v[r] = x1;
                            v[r | jb] = x0;
                        }
                    }
        }
    }
}
template <int E>
__device__ __forceinline__ void sort_row_regs(int32_t* __restrict__ c, int L, int lane) {
    int v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int t = lane * E + r;
        v[r] = t < L ? c[t] : INT_MAX;
    }
    warp_bitonic<E>(v, lane);
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int t = lane * E + r;
        if (t < L) c[t] = v[r];
    }
}

// One warp per row: put the diagonal last and sort the off-diagonal entries
// (written in arbitrary order by the fill's atomics) in registers; rows longer
// than SORT_WARP_CAP go to the block sort.
__global__ void row_sort_warp_k(const int64_t* __restrict__ rowptr, int64_t N, int32_t* __restrict__ col,
                                int32_t* __restrict__ long_rows, unsigned long long* __restrict__ nlong) {
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int64_t j = (int64_t)blockIdx.x * 8 + w;
    if (j >= N) return;
    const int64_t a = rowptr[j], b = rowptr[j + 1] - 1;  // off-diagonal part [a, b)
    col[b] = (int32_t)j;
    const int L = (int)(b - a);
    if (L <= 1) return;
    if (L > SORT_WARP_CAP) {
        if (lane == 0) long_rows[atomicAdd(nlong, 1ULL)] = (int32_t)j;
        return;
    }
    int32_t* c = col + a;
    if (L <= 32) sort_row_regs<1>(c, L, lane);
    else if (L <= 64) sort_row_regs<2>(c, L, lane);
    else if (L <= 128) sort_row_regs<4>(c, L, lane);
    else if (L <= 256) sort_row_regs<8>(c, L, lane);
    else if (L <= 512) sort_row_regs<16>(c, L, lane);
    else sort_row_regs<32>(c, L, lane);
}

__global__ void row_sort_block_k(const int64_t* __restrict__ rowptr, int32_t* __restrict__ col,
                                 const int32_t* __restrict__ long_rows) {
    extern __shared__ int sb[];
    const int64_t j = long_rows[blockIdx.x];
    const int64_t a = rowptr[j], b = rowptr[j + 1] - 1;
    const int L = (int)(b - a);
    int P = 1;
    while (P < L) P <<= 1;
    for (int t = threadIdx.x; t < P; t += blockDim.x) sb[t] = t < L ? col[a + t] : INT_MAX;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                int u = t ^ jj;
                if (u > t) {
                    int x0 = sb[t], x1 = sb[u];
                    bool up = (t & k) == 0;
                    if ((x0 > x1) == up) {
                        sb[t] = x1;
                        sb[u] = x0;
                    }
                }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < L; t += blockDim.x) col[a + t] = sb[t];
}

__global__ void max_len_k(const int64_t* __restrict__ rowptr, int64_t N, int* __restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int m = 0;
    if (j < N) m = (int)(rowptr[j + 1] - rowptr[j] - 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane_id() == 0) atomicMax(out, m);
}

kc_status pattern_fill_impl(const double* xo, const double* l, int64_t N, int d, double rho, int rule,
                            const int64_t* rowptr, int32_t* col, cudaStream_t s) {
    Arena A(s);
    int* mx;
    KC_TRY(A.get(&mx, 1));
    KC_CUDA(cudaMemsetAsync(mx, 0, sizeof(int), s));
    ::kc::note_launch(), max_len_k<<<blocks_for(N, 256), 256, 0, s>>>(rowptr, N, mx);
    int hmx = 0;
    KC_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (hmx > SORT_BLOCK_CAP) return fail(KC_EINVAL, "pattern row longer than 16384 entries");
    PatSetup S;
    KC_TRY(pat_setup(xo, l, N, d, rho, S, A, s));
    int* cnt;
    KC_TRY(A.get(&cnt, N));
    KC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * N, s));
    PatArgs P = pat_args(S, xo, l, d, rho, rule);
    if (S.nitems > 0) ::kc::note_launch(), pat_scan_k<true><<<blocks_for(S.nitems * 32, 256), 256, 0, s>>>(P, cnt, rowptr, col);
    KC_CUDA(cudaGetLastError());
    int32_t* long_rows;
    unsigned long long* nlong;
    KC_TRY(A.get(&long_rows, N));
    KC_TRY(A.get(&nlong, 1));
    KC_CUDA(cudaMemsetAsync(nlong, 0, sizeof(unsigned long long), s));
    ::kc::note_launch(), row_sort_warp_k<<<blocks_for(N, 8), 256, 0, s>>>(rowptr, N, col, long_rows, nlong);
    KC_CUDA(cudaGetLastError());
    unsigned long long hl = 0;
    KC_CUDA(cudaMemcpyAsync(&hl, nlong, sizeof(hl), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (hl > 0) {
        size_t sm = sizeof(int) * SORT_BLOCK_CAP;
        KC_TRY(allow_dynamic_smem(row_sort_block_k));
        ::kc::note_launch(), row_sort_block_k<<<(unsigned)hl, 1024, sm, s>>>(rowptr, col, long_rows);
        KC_CUDA(cudaGetLastError());
    }
    KC_CUDA(cudaStreamSynchronize(s));
    return KC_OK;
}


// ---- one search for both phases: the builder keeps the grid and the hit
// masks of the count pass for the fill (scratch held until end/abort)
struct PatternBuilder {
    cudaStream_t s;
    Arena* A = nullptr;
    PatSetup S;
    PatArgs P;
    int64_t N = 0;
    int64_t* moff = nullptr;
    uint32_t* masks = nullptr;
    int* cnt = nullptr;
    int64_t* rowptr = nullptr;
    int64_t nnz = 0;
};

kc_status pattern_begin_impl(const double* xo, const double* l, int64_t N, int d, double rho, int rule,
                             int64_t* rowptr, int64_t* nnz_out, void** out, cudaStream_t s) {
    PatternBuilder* B = new PatternBuilder();
    B->s = s;
    B->A = new Arena(s);
    B->N = N;
    B->rowptr = rowptr;
    auto fail_out = [&](kc_status st) {
        delete B->A;
        delete B;
        return st;
    };
    kc_status st = pat_setup(xo, l, N, d, rho, B->S, *B->A, s);
    if (st != KC_OK) return fail_out(st);
    B->P = pat_args(B->S, xo, l, d, rho, rule);
    const int64_t ni = B->S.nitems;
    int64_t* nch;
    if ((st = B->A->get(&nch, ni + 1)) != KC_OK) return fail_out(st);
    if ((st = B->A->get(&B->moff, ni + 1)) != KC_OK) return fail_out(st);
    if ((st = B->A->get(&B->cnt, N)) != KC_OK) return fail_out(st);
    int32_t* len;
    if ((st = B->A->get(&len, N)) != KC_OK) return fail_out(st);
    if (ni > 0) ::kc::note_launch(), pat_chunks_k<<<blocks_for(ni, 256), 256, 0, s>>>(B->P, nch);
    if ((st = exclusive_scan_i64(nch, B->moff, ni, *B->A, s)) != KC_OK) return fail_out(st);
    int64_t nchunks = 0;
    if (cudaMemcpyAsync(&nchunks, B->moff + ni, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail_out(fail(KC_ECUDA, "pattern: chunk count"));
    if ((st = B->A->get(&B->masks, nchunks)) != KC_OK) return fail_out(st);
    if (cudaMemsetAsync(B->cnt, 0, sizeof(int) * N, s) != cudaSuccess) return fail_out(fail(KC_ECUDA, "memset"));
    if (ni > 0) ::kc::note_launch(), pat_mask_k<<<blocks_for(ni * 32, 256), 256, 0, s>>>(B->P, B->moff, B->cnt, B->masks);
    ::kc::note_launch(), plus_one_k<<<blocks_for(N, 256), 256, 0, s>>>(B->cnt, N, len);
    if (cudaGetLastError() != cudaSuccess) return fail_out(fail(KC_ECUDA, "pattern: search launch"));
    if ((st = exclusive_scan_i32_to_i64(len, rowptr, N, *B->A, s)) != KC_OK) return fail_out(st);
    if (cudaMemcpyAsync(&B->nnz, rowptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail_out(fail(KC_ECUDA, "pattern: nnz"));
    if (nnz_out) *nnz_out = B->nnz;
    *out = B;
    return KC_OK;
}

void pattern_abort_impl(void* h) {
    PatternBuilder* B = (PatternBuilder*)h;
    if (!B) return;
    delete B->A;  // frees the scratch on the builder's stream
    delete B;
}

static kc_status pattern_fill_from(PatternBuilder* B, int32_t* col) {
    const cudaStream_t s = B->s;
    const int64_t N = B->N;
    Arena& A = *B->A;
    int* mx;
    KC_TRY(A.get(&mx, 1));
    KC_CUDA(cudaMemsetAsync(mx, 0, sizeof(int), s));
    ::kc::note_launch(), max_len_k<<<blocks_for(N, 256), 256, 0, s>>>(B->rowptr, N, mx);
    int hmx = 0;
    KC_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (hmx > SORT_BLOCK_CAP) return fail(KC_EINVAL, "pattern row longer than 16384 entries");
    KC_CUDA(cudaMemsetAsync(B->cnt, 0, sizeof(int) * N, s));
    if (B->S.nitems > 0)
        ::kc::note_launch(), pat_mask_fill_k<<<blocks_for(B->S.nitems * 32, 256), 256, 0, s>>>(B->P, B->moff, B->masks,
                                                                                            B->cnt, B->rowptr, col);
    KC_CUDA(cudaGetLastError());
    int32_t* long_rows;
    unsigned long long* nlong;
    KC_TRY(A.get(&long_rows, N));
    KC_TRY(A.get(&nlong, 1));
    KC_CUDA(cudaMemsetAsync(nlong, 0, sizeof(unsigned long long), s));
    ::kc::note_launch(), row_sort_warp_k<<<blocks_for(N, 8), 256, 0, s>>>(B->rowptr, N, col, long_rows, nlong);
    KC_CUDA(cudaGetLastError());
    unsigned long long hl = 0;
    KC_CUDA(cudaMemcpyAsync(&hl, nlong, sizeof(hl), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (hl > 0) {
        size_t sm = sizeof(int) * SORT_BLOCK_CAP;
        KC_TRY(allow_dynamic_smem(row_sort_block_k));
        ::kc::note_launch(), row_sort_block_k<<<(unsigned)hl, 1024, sm, s>>>(B->rowptr, col, long_rows);
        KC_CUDA(cudaGetLastError());
    }
    KC_CUDA(cudaStreamSynchronize(s));
    return KC_OK;
}

kc_status pattern_end_impl(void* h, int32_t* col) {
    PatternBuilder* B = (PatternBuilder*)h;
    const kc_status st = pattern_fill_from(B, col);
    pattern_abort_impl(B);
    return st;
}

}  // namespace kc
