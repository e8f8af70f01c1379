// Section 6: factors of a given sparse matrix (the precision matrix A, or
// sigma^2 A + I for a nugget) in the reverse maximin elimination order.
//
// The reversed order puts position N-1-a of the maximin order at position a.
// A symmetric pattern's lower triangle in reversed positions is its upper
// triangle in maximin positions, i.e. the CSC of the maximin-order lower
// triangle read backwards: reversed row q lists N-1-b for the rows b of
// maximin column N-1-q, in descending b, so columns ascend and the diagonal
// comes last (the layout every other kernel takes).
#include <algorithm>

#include "common.cuh"

namespace kc {

__global__ void rev_len_k(const int64_t* __restrict__ colptr, int64_t N, int64_t* __restrict__ len) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N) return;
    const int64_t a = N - 1 - q;
    len[q] = colptr[a + 1] - colptr[a];
}

// one warp per reversed row
__global__ void rev_fill_k(const int64_t* __restrict__ colptr, const int32_t* __restrict__ rowidx, int64_t N,
                           const int64_t* __restrict__ rowptr, int32_t* __restrict__ col) {
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= N) return;
    const int64_t a = N - 1 - q;
    const int64_t c0 = colptr[a], len = colptr[a + 1] - c0, w = rowptr[q];
    for (int64_t t = lane_id(); t < len; t += 32) col[w + t] = (int32_t)(N - 1 - rowidx[c0 + len - 1 - t]);
}

kc_status pattern_reverse_impl(int64_t N, const int64_t* colptr, const int32_t* rowidx, int64_t* rowptr, int32_t* col,
                               cudaStream_t s) {
    Arena A(s);
    int64_t* len;
    KC_TRY(A.get(&len, N));
    note_launch(), rev_len_k<<<blocks_for(N, 256), 256, 0, s>>>(colptr, N, len);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i64(len, rowptr, N, A, s));
    note_launch(), rev_fill_k<<<blocks_for(N, 8), 256, 0, s>>>(colptr, rowidx, N, rowptr, col);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// aval[e] = A(orig[j], orig[col[e]]) for the entries e of pattern row j (one
// warp per row); 0 where A has no entry
__global__ void gather_k(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t N,
                         const int32_t* __restrict__ orig, const int64_t* __restrict__ arp,
                         const int32_t* __restrict__ acol, const double* __restrict__ aval_in,
                         double* __restrict__ aval) {
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= N) return;
    const int32_t u = orig[j];
    const int64_t f0 = arp[u], f1 = arp[u + 1];
    for (int64_t e = rowptr[j] + lane_id(); e < rowptr[j + 1]; e += 32) {
        const int32_t v = orig[col[e]];
        int64_t lo = f0, hi = f1;
        while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (__ldg(&acol[m]) < v) lo = m + 1;
            else hi = m;
        }
        aval[e] = (lo < f1 && __ldg(&acol[lo]) == v) ? __ldg(&aval_in[lo]) : 0.0;
    }
}

__global__ void inverse_perm_k(const int32_t* __restrict__ orig, int64_t N, int32_t* __restrict__ pos) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < N) pos[orig[q]] = (int32_t)q;
}

// A's off-diagonal entries (u, v) whose positions are not a pattern pair (one
// warp per row u of A)
__global__ void outside_k(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t N,
                          const int32_t* __restrict__ pos, const int64_t* __restrict__ arp,
                          const int32_t* __restrict__ acol, unsigned long long* __restrict__ count) {
    const int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u >= N) return;
    unsigned long long n = 0;
    for (int64_t f = arp[u] + lane_id(); f < arp[u + 1]; f += 32) {
        const int32_t v = acol[f];
        if (v == u) continue;
        const int32_t pu = pos[u], pv = pos[v];
        const int32_t j = max(pu, pv), i = min(pu, pv);
        int64_t lo = rowptr[j], hi = rowptr[j + 1];
        while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (__ldg(&col[m]) < i) lo = m + 1;
            else hi = m;
        }
        if (!(lo < rowptr[j + 1] && __ldg(&col[lo]) == i)) ++n;
    }
    n = warp_sum(n);
    if (lane_id() == 0 && n) atomicAdd(count, n);
}

kc_status gather_impl(int64_t N, const int64_t* rowptr, const int32_t* col, const int32_t* orig, const int64_t* arp,
                      const int32_t* acol, const double* aval_in, double* aval, int64_t* outside_out,
                      cudaStream_t s) {
    note_launch(), gather_k<<<blocks_for(N, 8), 256, 0, s>>>(rowptr, col, N, orig, arp, acol, aval_in, aval);
    KC_CUDA(cudaGetLastError());
    if (!outside_out) return KC_OK;
    Arena A(s);
    int32_t* pos;
    unsigned long long* cnt;
    KC_TRY(A.get(&pos, N));
    KC_TRY(A.get(&cnt, 1));
    KC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    note_launch(), inverse_perm_k<<<blocks_for(N, 256), 256, 0, s>>>(orig, N, pos);
    KC_CUDA(cudaGetLastError());
    note_launch(), outside_k<<<blocks_for(N, 8), 256, 0, s>>>(rowptr, col, N, pos, arp, acol, cnt);
    KC_CUDA(cudaGetLastError());
    unsigned long long h = 0;
    KC_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    *outside_out = (int64_t)h;
    return KC_OK;
}

}  // namespace kc
