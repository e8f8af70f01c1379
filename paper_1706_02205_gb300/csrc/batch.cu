// Batching of independent point sets: block-diagonal concatenation of their
// patterns and coordinates, so that one persistent factor launch (and one
// solve) handles every set.  The factorisation of a block-diagonal pattern is
// the set of the blocks' factorisations, entry for entry.
#include <vector>

#include "common.cuh"

namespace kc {

__global__ void shift_rowptr_k(const int64_t* __restrict__ src, int64_t n, int64_t val_off, int64_t* __restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + val_off;
}
__global__ void shift_col_k(const int32_t* __restrict__ src, int64_t n, int32_t off, int32_t* __restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + off;
}
__global__ void fill_i32_k(int32_t* __restrict__ dst, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = v;
}
__global__ void pad_points_k(const double* __restrict__ src, int64_t n, int ds, int dout, double* __restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        for (int t = 0; t < dout; ++t) dst[i * dout + t] = t < ds ? src[i * ds + t] : 0.0;
}

kc_status pattern_concat_impl(int nsets, const int64_t* const* rowptrs, const int32_t* const* cols, const int64_t* Ns,
                              int64_t* rowptr_out, int32_t* col_out, int32_t* set_out, cudaStream_t s) {
    int64_t pos = 0, nz = 0;
    for (int k = 0; k < nsets; ++k) {
        const int64_t N = Ns[k];
        if (N < 1) return fail(KC_EINVAL, "every set needs N >= 1");
        int64_t nnz = 0;
        KC_CUDA(cudaMemcpyAsync(&nnz, rowptrs[k] + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        if (pos + N > INT32_MAX) return fail(KC_EINVAL, "total N must fit in int32");
        ::kc::note_launch(), shift_rowptr_k<<<blocks_for(N, 256), 256, 0, s>>>(rowptrs[k], N, nz, rowptr_out + pos);
        ::kc::note_launch(), shift_col_k<<<blocks_for(nnz, 256), 256, 0, s>>>(cols[k], nnz, (int32_t)pos, col_out + nz);
        if (set_out) ::kc::note_launch(), fill_i32_k<<<blocks_for(N, 256), 256, 0, s>>>(set_out + pos, N, k);
        KC_CUDA(cudaGetLastError());
        pos += N;
        nz += nnz;
    }
    KC_CUDA(cudaMemcpyAsync(rowptr_out + pos, &nz, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    KC_CUDA(cudaStreamSynchronize(s));
    return KC_OK;
}

kc_status index_concat_impl(int nsets, const int32_t* const* idx, const int64_t* Ns, int32_t* out, cudaStream_t s) {
    int64_t pos = 0;
    for (int k = 0; k < nsets; ++k) {
        if (pos + Ns[k] > INT32_MAX) return fail(KC_EINVAL, "total N must fit in int32");
        ::kc::note_launch(), shift_col_k<<<blocks_for(Ns[k], 256), 256, 0, s>>>(idx[k], Ns[k], (int32_t)pos, out + pos);
        KC_CUDA(cudaGetLastError());
        pos += Ns[k];
    }
    return KC_OK;
}

kc_status points_concat_impl(int nsets, const double* const* xs, const int64_t* Ns, const int32_t* ds, int dout,
                             double* out, cudaStream_t s) {
    int64_t pos = 0;
    for (int k = 0; k < nsets; ++k) {
        if (ds[k] < 1 || ds[k] > dout) return fail(KC_EINVAL, "every set needs 1 <= d <= dout");
        ::kc::note_launch(), pad_points_k<<<blocks_for(Ns[k], 256), 256, 0, s>>>(xs[k], Ns[k], ds[k], dout,
                                                                                  out + pos * dout);
        KC_CUDA(cudaGetLastError());
        pos += Ns[k];
    }
    return KC_OK;
}

}  // namespace kc
