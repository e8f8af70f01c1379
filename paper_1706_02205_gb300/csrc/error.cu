// The sampled error estimator of a factor (Section 4.4), on the device.
//
//   E^2 = sum_t ((L L^T)_{i_t j_t} - Theta_{i_t j_t})^2 / sum_t Theta_{i_t j_t}^2
//
// over m index pairs (i_t, j_t) that the caller draws i.i.d. uniformly from
// I x I (original point numbering, the diagonal allowed), optionally only over
// the pairs a keep mask marks (the paper's filtered estimator).  The pairs are
// mapped to positions of the maximin order through the inverse of perm.
//
// (L L^T)_ab for positions a <= b is the sum over k <= a of L_ak L_bk: the
// entries of row a below its diagonal matched in row b, plus L_aa L_ba (the
// diagonal L_aa is the FP64 pivot).  One warp per pair: lanes take the entries
// of row a with stride 32 and find each in row b by binary search (rows are
// sorted); products and sums in FP64, the warp's sum in a fixed butterfly
// order.  Theta_ab is evaluated from the coordinates in FP64 by the same code
// as the FP64 factor's entries, the nugget on the diagonal.  The per-pair
// terms are then summed in a fixed order (block ranges, then the blocks in
// order), so the result repeats bit for bit.
#include <algorithm>

#include "covariance.cuh"

namespace kc {

constexpr int FE_THREADS = 256;
constexpr int FE_MAX_BLOCKS = 1024;

__device__ __forceinline__ int64_t find_in_row(const int32_t* __restrict__ col, int64_t lo, int64_t hi, int k) {
    int64_t end = hi;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(&col[mid]) < k) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && __ldg(&col[lo]) == k) ? lo : -1;
}

template <typename T>
__global__ void __launch_bounds__(FE_THREADS) frob_pairs_k(const int64_t* __restrict__ rowptr,
                                                            const int32_t* __restrict__ col,
                                                            const T* __restrict__ val, const double* __restrict__ diag,
                                                            const double* __restrict__ x, int d, KernelParams kp,
                                                            const int32_t* __restrict__ pos, int64_t N,
                                                            const int64_t* __restrict__ pi,
                                                            const int64_t* __restrict__ pj,
                                                            const int8_t* __restrict__ keep, int64_t m,
                                                            double* __restrict__ e2, double* __restrict__ th2,
                                                            int* __restrict__ bad) {
    const int lane = lane_id();
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = w0; t < m; t += nw) {
        const int64_t oi = pi[t], oj = pj[t];
        if (oi < 0 || oi >= N || oj < 0 || oj >= N) {  // reported, never used as an index
            if (lane == 0) {
                atomicExch(bad, 1);
                e2[t] = 0.0;
                th2[t] = 0.0;
            }
            continue;
        }
        if (keep && !keep[t]) {
            if (lane == 0) e2[t] = th2[t] = 0.0;
            continue;
        }
        int a = pos[oi], b = pos[oj];
        if (a > b) {
            const int u = a;
            a = b;
            b = u;
        }
        const int64_t a0 = rowptr[a], a1 = rowptr[a + 1] - 1;  // row a below the diagonal: [a0, a1)
        const int64_t b0 = rowptr[b], b1 = rowptr[b + 1] - 1;
        double s = 0.0;
        if (a == b) {
            for (int64_t e = a0 + lane; e < a1; e += 32) {
                const double v = (double)val[e];
                s = fma(v, v, s);
            }
        } else {
            for (int64_t e = a0 + lane; e < a1; e += 32) {
                const int64_t f = find_in_row(col, b0, b1, __ldg(&col[e]));
                if (f >= 0) s = fma((double)val[e], (double)val[f], s);
            }
        }
        s = warp_sum(s);
        if (lane == 0) {
            const double daa = diag[a];
            if (a == b) {
                s = fma(daa, daa, s);
            } else {
                const int64_t f = find_in_row(col, b0, b1, a);
                if (f >= 0) s = fma(daa, (double)val[f], s);
            }
            double r2 = 0.0;
            for (int q = 0; q < d; ++q) {
                const double u = x[(int64_t)a * d + q] - x[(int64_t)b * d + q];
                r2 = fma(u, u, r2);
            }
            double th = cov_f64(kp, sqrt(r2));
            if (a == b) th += kp.nugget;
            const double err = s - th;
            e2[t] = err * err;
            th2[t] = th * th;
        }
    }
}

__global__ void fe_inverse_k(const int32_t* __restrict__ perm, int64_t N, int32_t* __restrict__ pos) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < N) pos[perm[q]] = (int32_t)q;
}

__device__ __forceinline__ void block_sum3(double& u, double& v, long long& c, double* sh) {
    u = warp_sum(u);
    v = warp_sum(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if (lane_id() == 0) sh[3 * w] = u, sh[3 * w + 1] = v, sh[3 * w + 2] = (double)c;
    __syncthreads();
    if (threadIdx.x == 0) {
        u = v = 0.0;
        c = 0;
        for (int k = 0; k < FE_THREADS / 32; ++k) u += sh[3 * k], v += sh[3 * k + 1], c += (long long)sh[3 * k + 2];
    }
}

// Block b sums its fixed range of pairs (kept pairs counted); then one block
// sums the block partials in order.
__global__ void __launch_bounds__(FE_THREADS) fe_part_k(const double* __restrict__ e2, const double* __restrict__ th2,
                                                        const int8_t* __restrict__ keep, int64_t m, int64_t per,
                                                        double* __restrict__ part) {
    __shared__ double sh[3 * FE_THREADS / 32];
    const int64_t a = (int64_t)blockIdx.x * per, e = min(m, a + per);
    double u = 0.0, v = 0.0;
    long long c = 0;
    for (int64_t t = a + threadIdx.x; t < e; t += FE_THREADS) {
        u += e2[t];
        v += th2[t];
        c += (keep == nullptr || keep[t]) ? 1 : 0;
    }
    block_sum3(u, v, c, sh);
    if (threadIdx.x == 0) part[3 * blockIdx.x] = u, part[3 * blockIdx.x + 1] = v, part[3 * blockIdx.x + 2] = (double)c;
}

__global__ void __launch_bounds__(FE_THREADS) fe_final_k(const double* __restrict__ part, int nb,
                                                         double* __restrict__ out) {
    __shared__ double sh[3 * FE_THREADS / 32];
    double u = 0.0, v = 0.0;
    long long c = 0;
    for (int k = threadIdx.x; k < nb; k += FE_THREADS)
        u += part[3 * k], v += part[3 * k + 1], c += (long long)part[3 * k + 2];
    block_sum3(u, v, c, sh);
    if (threadIdx.x == 0) out[0] = u, out[1] = v, out[2] = (double)c;
}

kc_status frob_error_impl(const kc_pattern* P, int prec, const void* val, const double* diag, const double* x_ord,
                          int d, const kc_kernel* kern, const int32_t* perm, const int64_t* pi, const int64_t* pj,
                          int64_t m, const int8_t* keep, double* num2_out, double* den2_out, int64_t* kept_out,
                          cudaStream_t s) {
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
    KernelParams kp;
    KC_TRY(kernel_params(kern, &kp));
    const int64_t N = P->N;
    Arena A(s);
    KC_TRY(upload_coef(kp, A, s));
    int32_t* pos;
    double *e2, *th2, *part, *res;
    int* bad;
    const int nb = (int)std::min<int64_t>(FE_MAX_BLOCKS, std::max<int64_t>(1, (m + FE_THREADS * 8 - 1) /
                                                                                   (FE_THREADS * 8)));
    const int64_t per = (m + nb - 1) / nb;
    KC_TRY(A.get(&pos, N));
    KC_TRY(A.get(&e2, m));
    KC_TRY(A.get(&th2, m));
    KC_TRY(A.get(&part, 3 * nb));
    KC_TRY(A.get(&res, 3));
    KC_TRY(A.get(&bad, 1));
    KC_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    note_launch(), fe_inverse_k<<<blocks_for(N, 256), 256, 0, s>>>(perm, N, pos);
    KC_CUDA(cudaGetLastError());
    const int grid = sm_count() * 8;
    if (prec == KC_FP64)
        note_launch(), frob_pairs_k<double><<<grid, FE_THREADS, 0, s>>>(P->rowptr, P->col, (const double*)val, diag,
                                                                        x_ord, d, kp, pos, N, pi, pj, keep, m, e2,
                                                                        th2, bad);
    else
        note_launch(), frob_pairs_k<float><<<grid, FE_THREADS, 0, s>>>(P->rowptr, P->col, (const float*)val, diag,
                                                                       x_ord, d, kp, pos, N, pi, pj, keep, m, e2, th2,
                                                                       bad);
    KC_CUDA(cudaGetLastError());
    note_launch(), fe_part_k<<<nb, FE_THREADS, 0, s>>>(e2, th2, keep, m, per, part);
    KC_CUDA(cudaGetLastError());
    note_launch(), fe_final_k<<<1, FE_THREADS, 0, s>>>(part, nb, res);
    KC_CUDA(cudaGetLastError());
    double h[3];
    int hb = 0;
    KC_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (hb) return fail(KC_EINVAL, "kc_frob_error: a pair index is outside 0..N-1");
    *num2_out = h[0];
    *den2_out = h[1];
    if (kept_out) *kept_out = (int64_t)h[2];
    return KC_OK;
}

}  // namespace kc
