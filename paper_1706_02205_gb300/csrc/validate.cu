// Structural check of a pattern and its schedule (kc_pattern_validate): the
// invariants every other kernel assumes, tested with every index checked
// against its range before it is used, so a corrupt pattern cannot take the
// check itself out of bounds.
#include "common.cuh"

namespace kc {

enum : int {
    PV_ROWPTR = 1,   // rowptr not 0 .. nnz, nondecreasing, or a row without its diagonal
    PV_COL = 2,      // a column index out of range, not ascending, or the diagonal not last
    PV_COLPTR = 3,   // colptr not consistent
    PV_ROWIDX = 4,   // a row index out of range, not ascending, or the diagonal not first
    PV_SLOT = 5,     // slot does not point at the same entry in the rows
    PV_ORDER = 6,    // order is not a permutation
};

__device__ __forceinline__ void pv_report(int* err, long long* where, int code, long long at) {
    if (atomicCAS(err, 0, code) == 0) *where = at;
}

// one warp per row j
__global__ void pv_rows_k(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t N, int64_t nnz,
                          int* err, long long* where) {
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= N) return;
    const int lane = lane_id();
    const int64_t a = rowptr[j], b = rowptr[j + 1];
    if (a < 0 || b > nnz || b <= a || (j == 0 && a != 0) || (j == N - 1 && b != nnz)) {
        if (lane == 0) pv_report(err, where, PV_ROWPTR, j);
        return;
    }
    for (int64_t e = a + lane; e < b; e += 32) {
        const int32_t c = col[e];
        const bool bad = c < 0 || c > j || (e + 1 < b && !(c < col[e + 1])) || (e + 1 == b && c != j);
        if (bad) pv_report(err, where, PV_COL, j);
    }
}

// one warp per column i
__global__ void pv_cols_k(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const int64_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                          const int64_t* __restrict__ slot, int64_t N, int64_t nnz, int* err, long long* where) {
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= N) return;
    const int lane = lane_id();
    const int64_t a = colptr[i], b = colptr[i + 1];
    if (a < 0 || b > nnz || b <= a || (i == 0 && a != 0) || (i == N - 1 && b != nnz)) {
        if (lane == 0) pv_report(err, where, PV_COLPTR, i);
        return;
    }
    for (int64_t q = a + lane; q < b; q += 32) {
        const int32_t r = rowidx[q];
        if (r < i || r >= N || (q == a && r != i) || (q + 1 < b && !(r < rowidx[q + 1]))) {
            pv_report(err, where, PV_ROWIDX, i);
            continue;
        }
        const int64_t sl = slot[q];
        if (sl < rowptr[r] || sl >= rowptr[r + 1] || col[sl] != i) pv_report(err, where, PV_SLOT, i);
    }
}

__global__ void pv_order_k(const int32_t* __restrict__ order, int64_t N, unsigned* __restrict__ seen, int* err,
                           long long* where) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int32_t c = order[t];
    if (c < 0 || c >= N || atomicAdd(&seen[c], 1u) != 0) pv_report(err, where, PV_ORDER, t);
}

kc_status pattern_validate_impl(const kc_pattern* P, cudaStream_t s) {
    const int64_t N = P->N, nnz = P->nnz;
    Arena A(s);
    int* err;
    long long* where;
    unsigned* seen;
    KC_TRY(A.get(&err, 1));
    KC_TRY(A.get(&where, 1));
    KC_TRY(A.get(&seen, N));
    KC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    KC_CUDA(cudaMemsetAsync(where, 0, sizeof(long long), s));
    KC_CUDA(cudaMemsetAsync(seen, 0, sizeof(unsigned) * N, s));
    note_launch(), pv_rows_k<<<blocks_for(N, 8), 256, 0, s>>>(P->rowptr, P->col, N, nnz, err, where);
    KC_CUDA(cudaGetLastError());
    int h = 0;
    long long at = 0;
    KC_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (h == 0) {  // the columns index into the rows: only once the rows are sound
        note_launch(), pv_cols_k<<<blocks_for(N, 8), 256, 0, s>>>(P->rowptr, P->col, P->colptr, P->rowidx, P->slot, N,
                                                                   nnz, err, where);
        KC_CUDA(cudaGetLastError());
        note_launch(), pv_order_k<<<blocks_for(N, 256), 256, 0, s>>>(P->order, N, seen, err, where);
        KC_CUDA(cudaGetLastError());
        KC_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    KC_CUDA(cudaMemcpyAsync(&at, where, sizeof(long long), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (h == 0) return KC_OK;
    static const char* what[] = {"", "rowptr", "col", "colptr", "rowidx", "slot", "order"};
    return fail(KC_EINVAL, std::string("pattern check: bad ") + what[h] + " at index " + std::to_string(at));
}

}  // namespace kc
