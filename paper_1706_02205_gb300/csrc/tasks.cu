// Tasks (1), (3) and (4) of Section 1 with the factor standing in for Theta:
// Theta v ~ L (L^T v), log det Theta ~ 2 sum_i log L_ii, and samples L z of
// N(0, L L^T).  Plus the covariance function on its own (the entries the
// factor evaluates).
//
// L z is a gather along the CSR rows of L (one warp per row, lanes over its
// entries, coalesced col/val reads); L^T v a gather along the columns through
// the CSC of the pattern (one warp per chunk of a column; rowidx and slot
// coalesced, the values fetched through slot).  No atomics: each output is a
// sum in a fixed order, so results repeat bit for bit.  Vectors are point-major
// inside (x[k * NS + r], NS = nrhs padded to a power of two), so one point's
// components share a 32-byte sector.
#include <algorithm>

#include "covariance.cuh"
#include "solver.cuh"

namespace kc {

constexpr int TK_THREADS = 256;
constexpr int TK_WARPS = TK_THREADS / 32;

template <int NS>
__device__ __forceinline__ void gather_fma(double (&acc)[NS], double w, const double* __restrict__ z, int64_t k) {
    const double* p = z + k * NS;
#pragma unroll
    for (int r = 0; r < NS; ++r) acc[r] = fma(w, __ldg(p + r), acc[r]);
}

// lanes 0..NS-1 write y[j*NS + r] = (warp total of acc[r]) + dj * z[j*NS + r]
template <int NS>
__device__ __forceinline__ void finish_row(double (&acc)[NS], double dj, const double* __restrict__ z, int64_t j,
                                           double* __restrict__ y) {
    const int lane = lane_id();
    double mine = 0.0;
#pragma unroll
    for (int r = 0; r < NS; ++r) {
        const double t = warp_sum(acc[r]);  // butterfly: every lane holds the same bits
        if (lane == r) mine = t;
    }
    if (lane < NS) y[j * NS + lane] = fma(dj, z[j * NS + lane], mine);
}

// y = L z: row j of L is col/val[rowptr[j] .. rowptr[j+1]-1), the diagonal last
// (taken from diag, the FP64 L_jj).
template <typename T, int NS>
__global__ void __launch_bounds__(TK_THREADS) l_rows_k(const int64_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ col, const T* __restrict__ val,
                                                       const double* __restrict__ diag, int64_t N,
                                                       const double* __restrict__ z, double* __restrict__ y) {
    const int64_t j = (int64_t)blockIdx.x * TK_WARPS + (threadIdx.x >> 5);
    if (j >= N) return;
    double acc[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) acc[r] = 0.0;
    const int64_t e1 = rowptr[j + 1] - 1;
#pragma unroll 4
    for (int64_t e = rowptr[j] + lane_id(); e < e1; e += 32) gather_fma<NS>(acc, (double)__ldg(&val[e]), z, __ldg(&col[e]));
    finish_row<NS>(acc, diag[j], z, j, y);
}

// y = L^T v: column i of L is rowidx[colptr[i] .. colptr[i+1]), the diagonal
// first; slot gives each entry's CSR position in val.  Maximin columns are
// very uneven (the first column holds every point), so each column is cut
// into chunks of at most LT_CHUNK entries below its diagonal, one warp per
// chunk; a column of one chunk writes its result directly, a longer one
// leaves per-chunk sums that lt_finish_k adds in chunk order.
constexpr int LT_CHUNK = 1024;

__global__ void lt_count_k(const int64_t* __restrict__ colptr, int64_t N, int32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t len = colptr[i + 1] - colptr[i] - 1;
    cnt[i] = len <= LT_CHUNK ? 1 : (int32_t)((len + LT_CHUNK - 1) / LT_CHUNK);
}

__global__ void lt_owner_k(const int64_t* __restrict__ off, int64_t N, int32_t* __restrict__ owner) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int64_t c = off[i]; c < off[i + 1]; ++c) owner[c] = (int32_t)i;
}

template <typename T, int NS>
__global__ void __launch_bounds__(TK_THREADS) lt_chunks_k(const int64_t* __restrict__ colptr,
                                                          const int32_t* __restrict__ rowidx,
                                                          const int64_t* __restrict__ slot, const T* __restrict__ val,
                                                          const double* __restrict__ diag,
                                                          const int64_t* __restrict__ off,
                                                          const int32_t* __restrict__ owner, int64_t N,
                                                          const double* __restrict__ v, double* __restrict__ y,
                                                          double* __restrict__ part) {
    const int64_t c = (int64_t)blockIdx.x * TK_WARPS + (threadIdx.x >> 5);
    if (c >= off[N]) return;
    const int i = owner[c];
    const int64_t k = c - off[i];
    const int64_t q0 = colptr[i] + 1 + k * LT_CHUNK;
    const int64_t q1 = min(colptr[i + 1], q0 + LT_CHUNK);
    double acc[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) acc[r] = 0.0;
#pragma unroll 4
    for (int64_t q = q0 + lane_id(); q < q1; q += 32)
        gather_fma<NS>(acc, (double)__ldg(&val[__ldg(&slot[q])]), v, __ldg(&rowidx[q]));
    if (off[i + 1] - off[i] == 1) {
        finish_row<NS>(acc, diag[i], v, i, y);
    } else {
        const int lane = lane_id();
        double mine = 0.0;
#pragma unroll
        for (int r = 0; r < NS; ++r) {
            const double t = warp_sum(acc[r]);
            if (lane == r) mine = t;
        }
        if (lane < NS) part[c * NS + lane] = mine;
    }
}

// y[i][r] of the columns cut into several chunks: the chunk sums in order
template <int NS>
__global__ void lt_finish_k(const int64_t* __restrict__ off, int64_t N, const double* __restrict__ diag,
                            const double* __restrict__ v, const double* __restrict__ part, double* __restrict__ y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * NS) return;
    const int64_t i = t / NS;
    const int r = (int)(t % NS);
    const int64_t c0 = off[i], c1 = off[i + 1];
    if (c1 - c0 == 1) return;
    double s = 0.0;
    for (int64_t c = c0; c < c1; ++c) s += part[c * NS + r];
    y[i * NS + r] = fma(diag[i], v[i * NS + r], s);
}

// Chunk layout of the columns (independent of the vectors): off[i] = first
// chunk of column i, off[N] = chunks in all; owner[c] = column of chunk c.
struct LtChunks {
    int64_t* off = nullptr;
    int32_t* owner = nullptr;
    int64_t cap = 0;  // chunks at most: N + (nnz - N) / LT_CHUNK
};

static kc_status lt_chunks_build(const kc_pattern* P, Arena& A, cudaStream_t s, LtChunks& C) {
    const int64_t N = P->N;
    C.cap = N + (P->nnz - N) / LT_CHUNK + 1;
    int32_t* cnt;
    KC_TRY(A.get(&cnt, N));
    KC_TRY(A.get(&C.off, N + 1));
    KC_TRY(A.get(&C.owner, C.cap));
    note_launch(), lt_count_k<<<blocks_for(N, 256), 256, 0, s>>>(P->colptr, N, cnt);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i32_to_i64(cnt, C.off, N, A, s));
    note_launch(), lt_owner_k<<<blocks_for(N, 256), 256, 0, s>>>(C.off, N, C.owner);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

template <typename T, int NS>
static kc_status mv_launch(const kc_pattern* P, bool transpose, const T* val, const double* diag, const double* in,
                           double* out, const LtChunks& C, double* part, cudaStream_t s) {
    if (transpose) {
        // the grid covers the most chunks there can be; surplus warps return
        note_launch(), lt_chunks_k<T, NS><<<blocks_for(C.cap, TK_WARPS), TK_THREADS, 0, s>>>(
            P->colptr, P->rowidx, P->slot, val, diag, C.off, C.owner, P->N, in, out, part);
        KC_CUDA(cudaGetLastError());
        note_launch(), lt_finish_k<NS><<<blocks_for(P->N * NS, 256), 256, 0, s>>>(C.off, P->N, diag, in, part, out);
    } else {
        note_launch(), l_rows_k<T, NS><<<blocks_for(P->N, TK_WARPS), TK_THREADS, 0, s>>>(P->rowptr, P->col, val, diag,
                                                                                         P->N, in, out);
    }
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

template <typename T>
static kc_status mv_dispatch(const kc_pattern* P, bool transpose, const T* val, const double* diag, const double* in,
                             double* out, int ns, const LtChunks& C, double* part, cudaStream_t s) {
    switch (ns) {
        case 1: return mv_launch<T, 1>(P, transpose, val, diag, in, out, C, part, s);
        case 2: return mv_launch<T, 2>(P, transpose, val, diag, in, out, C, part, s);
        case 4: return mv_launch<T, 4>(P, transpose, val, diag, in, out, C, part, s);
        case 8: return mv_launch<T, 8>(P, transpose, val, diag, in, out, C, part, s);
        default: return mv_launch<T, 16>(P, transpose, val, diag, in, out, C, part, s);
    }
}

// which: 0 = L, 1 = L^T, 2 = L L^T
kc_status factor_matvec_impl(const kc_pattern* P, int prec, const void* val, const double* diag, const int32_t* perm,
                             const double* in, int nrhs, double* out, int which, cudaStream_t s) {
    if (nrhs < 1 || nrhs > 16) return fail(KC_EINVAL, "nrhs must be in 1..16");
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
    if (in == out) return fail(KC_EINVAL, "the output must not alias the input");
    int ns = 1;
    while (ns < nrhs) ns <<= 1;
    Arena A(s);
    double *a, *b, *part = nullptr;
    KC_TRY(A.get(&a, P->N * ns));
    KC_TRY(A.get(&b, P->N * ns));
    LtChunks C;
    if (which != 0) {
        KC_TRY(lt_chunks_build(P, A, s, C));
        KC_TRY(A.get(&part, C.cap * ns));
    }
    KC_TRY(to_point_major(in, perm, P->N, nrhs, a, s, ns));
    auto step = [&](bool tr, const double* x, double* y) {
        return prec == KC_FP64 ? mv_dispatch<double>(P, tr, (const double*)val, diag, x, y, ns, C, part, s)
                               : mv_dispatch<float>(P, tr, (const float*)val, diag, x, y, ns, C, part, s);
    };
    const double* res = b;
    if (which == 0) KC_TRY(step(false, a, b));
    else if (which == 1) KC_TRY(step(true, a, b));
    else {
        KC_TRY(step(true, a, b));
        KC_TRY(step(false, b, a));
        res = a;
    }
    return from_point_major(res, perm, P->N, nrhs, out, s, ns);
}

// ------------------------------------------------------------------ logdet
// Block b sums log diag[i] over its fixed range (threads strided, then a
// fixed tree); one block then sums the block partials in order.
constexpr int LD_THREADS = 256;
constexpr int LD_MAX_BLOCKS = 1024;

__device__ __forceinline__ void block_sum2(double& s, long long& z, double* sh, long long* shz) {
    s = warp_sum(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) sh[w] = s, shz[w] = z;
    __syncthreads();
    if (threadIdx.x == 0) {
        s = 0.0;
        z = 0;
        for (int k = 0; k < LD_THREADS / 32; ++k) s += sh[k], z += shz[k];
    }
}

__global__ void __launch_bounds__(LD_THREADS) logdet_part_k(const double* __restrict__ diag, int64_t N, int64_t per,
                                                            double* __restrict__ part, long long* __restrict__ zpart) {
    __shared__ double sh[LD_THREADS / 32];
    __shared__ long long shz[LD_THREADS / 32];
    const int64_t a = (int64_t)blockIdx.x * per, e = min(N, a + per);
    double s = 0.0;
    long long z = 0;
    for (int64_t i = a + threadIdx.x; i < e; i += LD_THREADS) {
        const double d = diag[i];
        if (d > 0.0) s += log(d);
        else ++z;
    }
    block_sum2(s, z, sh, shz);
    if (threadIdx.x == 0) part[blockIdx.x] = s, zpart[blockIdx.x] = z;
}

__global__ void __launch_bounds__(LD_THREADS) logdet_final_k(const double* __restrict__ part,
                                                             const long long* __restrict__ zpart, int nb,
                                                             double* __restrict__ out, long long* __restrict__ zout) {
    __shared__ double sh[LD_THREADS / 32];
    __shared__ long long shz[LD_THREADS / 32];
    double s = 0.0;
    long long z = 0;
    for (int k = threadIdx.x; k < nb; k += LD_THREADS) s += part[k], z += zpart[k];
    block_sum2(s, z, sh, shz);
    if (threadIdx.x == 0) *out = 2.0 * s, *zout = z;
}

kc_status logdet_impl(const kc_pattern* P, const double* diag, double* logdet_out, int64_t* zero_out, cudaStream_t s) {
    const int64_t N = P->N;
    const int nb = (int)std::min<int64_t>(LD_MAX_BLOCKS, (N + LD_THREADS * 8 - 1) / (LD_THREADS * 8));
    const int64_t per = (N + nb - 1) / nb;
    Arena A(s);
    double* part;
    long long* zpart;
    double* res;
    long long* zres;
    KC_TRY(A.get(&part, nb));
    KC_TRY(A.get(&zpart, nb));
    KC_TRY(A.get(&res, 1));
    KC_TRY(A.get(&zres, 1));
    note_launch(), logdet_part_k<<<nb, LD_THREADS, 0, s>>>(diag, N, per, part, zpart);
    KC_CUDA(cudaGetLastError());
    note_launch(), logdet_final_k<<<1, LD_THREADS, 0, s>>>(part, zpart, nb, res, zres);
    KC_CUDA(cudaGetLastError());
    double h = 0.0;
    long long hz = 0;
    KC_CUDA(cudaMemcpyAsync(&h, res, sizeof(double), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaMemcpyAsync(&hz, zres, sizeof(long long), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    *logdet_out = h;
    if (zero_out) *zero_out = (int64_t)hz;
    return KC_OK;
}

// --------------------------------------------------------- kernel alone
__global__ void kernel_eval_k(KernelParams kp, int prec, const double* __restrict__ r, int64_t n,
                              double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = prec == KC_FP64 ? cov_f64(kp, r[i]) : (double)cov_f32(kp, (float)r[i]);
}

kc_status kernel_eval_impl(const kc_kernel* kern, int prec, const double* r, int64_t n, double* out, cudaStream_t s) {
    KernelParams kp;
    KC_TRY(kernel_params(kern, &kp));
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
    if (n == 0) return KC_OK;
    Arena A(s);
    KC_TRY(upload_coef(kp, A, s));
    note_launch(), kernel_eval_k<<<blocks_for(n, 256), 256, 0, s>>>(kp, prec, r, n, out);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

}  // namespace kc
