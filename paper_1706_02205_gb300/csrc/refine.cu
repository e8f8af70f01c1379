// a8: refinement of the solve, and the dense kernel-matrix products.
//
// The refined solve is CG on the dense Theta (task (2) of Section 1) with the
// factor as preconditioner, M = L L^T (Section 4.3 suggests CG preconditioned
// with the factor).  Theta is never stored: Theta v is evaluated from the
// coordinates, FP64 throughout, O(N^2) per product.  The masked matrix Theta
// restricted to S is not positive definite in general, so it is not used as
// the CG operator.
//
// a9's error check uses the same dense product with FP32 entries and
// compensated (Dot2) tile sums combined in FP64.
#include "solver.cuh"
#include "covariance.cuh"

namespace kc {

constexpr int DM_THREADS = 128;
constexpr int DM_MAXD = 32;

// y[j][r] = sum_k Theta(x_j, x_k) v[k][r], point-major, FP64.
template <int NRHS>
__global__ void __launch_bounds__(DM_THREADS) dense_theta_f64_k(const double* __restrict__ x, int64_t N, int d,
                                                              KernelParams kp, const double* __restrict__ v,
                                                              double* __restrict__ y) {
    extern __shared__ __align__(16) double sh[];
    double* sx = sh;                       // DM_THREADS * d
    double* sv = sh + DM_THREADS * d;      // DM_THREADS * NRHS
    const int64_t j = (int64_t)blockIdx.x * DM_THREADS + threadIdx.x;
    double xj[DM_MAXD];
    for (int t = 0; t < d; ++t) xj[t] = j < N ? x[j * d + t] : 0.0;
    double acc[NRHS];
#pragma unroll
    for (int r = 0; r < NRHS; ++r) acc[r] = 0.0;
    for (int64_t k0 = 0; k0 < N; k0 += DM_THREADS) {
        __syncthreads();
        for (int u = threadIdx.x; u < DM_THREADS * d; u += DM_THREADS) {
            int64_t k = k0 + u / d;
            sx[u] = k < N ? x[k0 * d + u] : 0.0;
        }
        for (int u = threadIdx.x; u < DM_THREADS * NRHS; u += DM_THREADS) {
            int64_t k = k0 + u / NRHS;
            sv[u] = k < N ? v[k0 * NRHS + u] : 0.0;
        }
        __syncthreads();
        const int kn = (int)min((int64_t)DM_THREADS, N - k0);
        for (int kk = 0; kk < kn; ++kk) {
            double s = 0.0;
            for (int t = 0; t < d; ++t) {
                double u = xj[t] - sx[kk * d + t];
                s = fma(u, u, s);
            }
            double th = cov_f64(kp, sqrt(s));
            if (k0 + kk == j) th += kp.nugget;
#pragma unroll
            for (int r = 0; r < NRHS; ++r) acc[r] = fma(th, sv[kk * NRHS + r], acc[r]);
        }
    }
    if (j < N)
#pragma unroll
        for (int r = 0; r < NRHS; ++r) y[j * NRHS + r] = acc[r];
}

template <int NRHS>
static kc_status dense_f64_launch(const double* x, int64_t N, int d, const KernelParams& kp, const double* v,
                                  double* y, cudaStream_t s) {
    size_t sm = sizeof(double) * DM_THREADS * (d + NRHS);
    KC_TRY(allow_dynamic_smem(dense_theta_f64_k<NRHS>));
    ::kc::note_launch(), dense_theta_f64_k<NRHS><<<blocks_for(N, DM_THREADS), DM_THREADS, sm, s>>>(x, N, d, kp, v, y);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

kc_status dense_theta_f64(const double* x, int64_t N, int d, const KernelParams& kp, const double* v, double* y,
                          int nrhs, cudaStream_t s) {
    if (d > DM_MAXD) return fail(KC_EINVAL, "dense product supports d <= 32");
    switch (nrhs) {
        case 1: return dense_f64_launch<1>(x, N, d, kp, v, y, s);
        case 2: return dense_f64_launch<2>(x, N, d, kp, v, y, s);
        case 4: return dense_f64_launch<4>(x, N, d, kp, v, y, s);
        case 8: return dense_f64_launch<8>(x, N, d, kp, v, y, s);
        case 16: return dense_f64_launch<16>(x, N, d, kp, v, y, s);
        default: return fail(KC_EINVAL, "internal: nrhs slot must be 1,2,4,8,16");
    }
}

// ------------------------------------------------- CG vector operations
constexpr int RED_BLOCKS = 256;

// partial[b * nrhs + r] = sum over block b's points of a[k][r] * c[k][r]
__global__ void dots_k(const double* __restrict__ a, const double* __restrict__ c, int64_t N, int nrhs,
                       double* __restrict__ partial) {
    __shared__ double sh[16][33];
    const int lane = lane_id(), w = threadIdx.x >> 5;  // 8 warps
    for (int r = 0; r < nrhs; ++r) {
        double s = 0.0;
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
            s = fma(a[k * nrhs + r], c[k * nrhs + r], s);
        s = warp_sum(s);
        if (lane == 0) sh[r][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < nrhs) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sh[threadIdx.x][q];
        partial[blockIdx.x * nrhs + threadIdx.x] = s;
    }
}
__global__ void dots_final_k(const double* __restrict__ partial, int nb, int nrhs, double* __restrict__ out) {
    int r = threadIdx.x;
    if (r < nrhs) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += partial[b * nrhs + r];
        out[r] = s;
    }
}

static kc_status dots(const double* a, const double* c, int64_t N, int nrhs, double* partial, double* out,
                      cudaStream_t s) {
    ::kc::note_launch(), dots_k<<<RED_BLOCKS, 256, 0, s>>>(a, c, N, nrhs, partial);
    ::kc::note_launch(), dots_final_k<<<1, 32, 0, s>>>(partial, RED_BLOCKS, nrhs, out);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// alpha = rz/pq per rhs (0 for a finished rhs); x += alpha p; r -= alpha q
__global__ void cg_update_xr_k(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                               const double* __restrict__ q, const double* __restrict__ rz,
                               const double* __restrict__ pq, const int* __restrict__ active, int64_t N, int nrhs) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * nrhs) {
        int c = (int)(t % nrhs);
        if (!active[c]) return;
        double al = rz[c] / pq[c];
        x[t] = fma(al, p[t], x[t]);
        r[t] = fma(-al, q[t], r[t]);
    }
}
// beta = rz_new/rz; p = z + beta p; rz = rz_new
__global__ void cg_update_p_k(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ rz,
                              const double* __restrict__ rz_new, const int* __restrict__ active, int64_t N,
                              int nrhs) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * nrhs) {
        int c = (int)(t % nrhs);
        if (!active[c]) return;
        double be = rz_new[c] / rz[c];
        p[t] = fma(be, p[t], z[t]);
    }
}
__global__ void copy_k(double* __restrict__ dst, const double* __restrict__ src, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = src[t];
}
__global__ void sub_k(double* __restrict__ dst, const double* __restrict__ a, const double* __restrict__ b,
                      int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = a[t] - b[t];
}

// y[k][r] = sum_m A(orig[k], orig[m]) v[m][r] in positions (point-major,
// stride NS): one warp per row, A given by CSR rows in original numbering,
// pos the inverse of orig.  Each output is one warp's sum in a fixed order.
template <int NS>
__global__ void __launch_bounds__(256) sparse_pos_mv_k(const int64_t* __restrict__ arp,
                                                       const int32_t* __restrict__ acol,
                                                       const double* __restrict__ aval,
                                                       const int32_t* __restrict__ orig, const int32_t* __restrict__ pos,
                                                       int64_t N, const double* __restrict__ v, double* __restrict__ y) {
    const int64_t k = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (k >= N) return;
    const int u = orig[k];
    double acc[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) acc[r] = 0.0;
    for (int64_t f = arp[u] + lane_id(); f < arp[u + 1]; f += 32) {
        const double a = __ldg(&aval[f]);
        const double* vm = v + (int64_t)__ldg(&pos[__ldg(&acol[f])]) * NS;
#pragma unroll
        for (int r = 0; r < NS; ++r) acc[r] = fma(a, __ldg(vm + r), acc[r]);
    }
    double mine = 0.0;
#pragma unroll
    for (int r = 0; r < NS; ++r) {
        const double t = warp_sum(acc[r]);
        if (lane_id() == r) mine = t;
    }
    if (lane_id() < NS) y[k * NS + lane_id()] = mine;
}

__global__ void inverse_index_k(const int32_t* __restrict__ orig, int64_t N, int32_t* __restrict__ pos) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < N) pos[orig[q]] = (int32_t)q;
}

struct SparseOp {
    const int64_t* arp;
    const int32_t* acol;
    const double* aval;
    const int32_t* orig;
    const int32_t* pos;
};

static kc_status sparse_pos_mv(const SparseOp& M, int64_t N, const double* v, double* y, int ns, cudaStream_t s) {
    const unsigned g = blocks_for(N, 8);
    switch (ns) {
        case 1: ::kc::note_launch(), sparse_pos_mv_k<1><<<g, 256, 0, s>>>(M.arp, M.acol, M.aval, M.orig, M.pos, N, v, y); break;
        case 2: ::kc::note_launch(), sparse_pos_mv_k<2><<<g, 256, 0, s>>>(M.arp, M.acol, M.aval, M.orig, M.pos, N, v, y); break;
        case 4: ::kc::note_launch(), sparse_pos_mv_k<4><<<g, 256, 0, s>>>(M.arp, M.acol, M.aval, M.orig, M.pos, N, v, y); break;
        case 8: ::kc::note_launch(), sparse_pos_mv_k<8><<<g, 256, 0, s>>>(M.arp, M.acol, M.aval, M.orig, M.pos, N, v, y); break;
        default: ::kc::note_launch(), sparse_pos_mv_k<16><<<g, 256, 0, s>>>(M.arp, M.acol, M.aval, M.orig, M.pos, N, v, y);
    }
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// The operator of the CG: the dense Theta from the coordinates (kernel given)
// or a given sparse matrix (M.arp given).
struct CgOperator {
    const double* x_ord = nullptr;
    int d = 0;
    KernelParams kp{};
    SparseOp M{};
    kc_status apply(int64_t N, const double* v, double* y, int ns, cudaStream_t s) const {
        if (M.arp) return sparse_pos_mv(M, N, v, y, ns, s);
        return dense_theta_f64(x_ord, N, d, kp, v, y, ns, s);
    }
};

static kc_status refine_core(const kc_pattern* P, CgOperator& op, double fb, int prec, const void* val,
                             const double* diag, const int32_t* perm, const double* b, int nrhs, double rtol,
                             int maxit, double* x_out, int32_t* iters_out, double* relres_out, const kc_opts* o,
                             Arena& A, cudaStream_t s);

kc_status refine_impl(const kc_pattern* P, const double* x_ord, int d, const kc_kernel* kern, int prec,
                      const void* val, const double* diag, const int32_t* perm, const double* b, int nrhs,
                      double rtol, int maxit, double* x_out, int32_t* iters_out, double* relres_out,
                      const kc_opts* o, cudaStream_t s) {
    CgOperator op;
    KC_TRY(kernel_params(kern, &op.kp));
    op.x_ord = x_ord;
    op.d = d;
    Arena A(s);
    KC_TRY(upload_coef(op.kp, A, s));
    return refine_core(P, op, sqrt(op.kp.sigma2 + op.kp.nugget), prec, val, diag, perm, b, nrhs, rtol, maxit, x_out,
                       iters_out, relres_out, o, A, s);
}

kc_status refine_sparse_impl(const kc_pattern* P, int prec, const void* val, const double* diag,
                             const int32_t* perm, const int64_t* arp, const int32_t* acol, const double* aval,
                             const double* b, int nrhs, double rtol, int maxit, double* x_out, int32_t* iters_out,
                             double* relres_out, const kc_opts* o, cudaStream_t s) {
    CgOperator op;
    Arena A(s);
    int32_t* pos;
    KC_TRY(A.get(&pos, P->N));
    ::kc::note_launch(), inverse_index_k<<<blocks_for(P->N, 256), 256, 0, s>>>(perm, P->N, pos);
    KC_CUDA(cudaGetLastError());
    op.M = SparseOp{arp, acol, aval, perm, pos};
    return refine_core(P, op, 1.0, prec, val, diag, perm, b, nrhs, rtol, maxit, x_out, iters_out, relres_out, o, A,
                       s);
}

static kc_status refine_core(const kc_pattern* P, CgOperator& op, double fb, int prec, const void* val,
                             const double* diag, const int32_t* perm, const double* b, int nrhs, double rtol,
                             int maxit, double* x_out, int32_t* iters_out, double* relres_out, const kc_opts* o,
                             Arena& A, cudaStream_t s) {
    if (nrhs < 1 || nrhs > 16) return fail(KC_EINVAL, "nrhs must be in 1..16");
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "bad prec");
    const int64_t N = P->N;
    int ns = 1;
    while (ns < nrhs) ns <<= 1;  // padded slot count (extra columns stay zero)
    Solver S;
    KC_TRY(solver_init(S, P, ns, o, A, s));
    const int64_t n = N * ns;
    double *bp, *xs, *r, *z, *p, *q, *partial, *sc;
    int* active;
    KC_TRY(A.get(&bp, n));
    KC_TRY(A.get(&xs, n));
    KC_TRY(A.get(&r, n));
    KC_TRY(A.get(&z, n));
    KC_TRY(A.get(&p, n));
    KC_TRY(A.get(&q, n));
    KC_TRY(A.get(&partial, RED_BLOCKS * 16));
    KC_TRY(A.get(&sc, 16 * 6));
    KC_TRY(A.get(&active, 16));
    double* rz = sc;
    double* rzn = sc + 16;
    double* pq = sc + 32;
    double* rr = sc + 48;
    double* bb = sc + 64;
    KC_CUDA(cudaMemsetAsync(bp, 0, sizeof(double) * n, s));
    KC_CUDA(cudaMemsetAsync(xs, 0, sizeof(double) * n, s));
    // scatter b into the padded point-major layout
    {
        double* tmp;
        KC_TRY(A.get(&tmp, N * nrhs));
        KC_TRY(to_point_major(b, perm, N, nrhs, tmp, s));
        KC_CUDA(cudaMemcpy2DAsync(bp, sizeof(double) * ns, tmp, sizeof(double) * nrhs, sizeof(double) * nrhs, N,
                                  cudaMemcpyDeviceToDevice, s));
    }
    auto precond = [&](const double* in, double* out) -> kc_status {
        if (prec == KC_FP64) return solver_apply<double>(S, (const double*)val, diag, fb, in, out, ns, s);
        return solver_apply<float>(S, (const float*)val, diag, fb, in, out, ns, s);
    };
    const unsigned gb = blocks_for(n, 256);
    ::kc::note_launch(), copy_k<<<gb, 256, 0, s>>>(r, bp, n);
    KC_TRY(dots(bp, bp, N, ns, partial, bb, s));
    KC_TRY(precond(r, z));
    ::kc::note_launch(), copy_k<<<gb, 256, 0, s>>>(p, z, n);
    KC_TRY(dots(r, z, N, ns, partial, rz, s));
    double h_bb[16], h_rr[16], h_pq[16];
    int h_active[16];
    KC_CUDA(cudaMemcpyAsync(h_bb, bb, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    KC_TRY(solver_check(S, s));
    for (int c = 0; c < ns; ++c) h_active[c] = (c < nrhs && h_bb[c] > 0.0) ? 1 : 0;
    int it = 0;
    kc_status result = KC_ENOTCONV;
    for (;;) {
        KC_TRY(dots(r, r, N, ns, partial, rr, s));
        KC_CUDA(cudaMemcpyAsync(h_rr, rr, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        bool all = true;
        for (int c = 0; c < nrhs; ++c) {
            if (h_active[c] && sqrt(h_rr[c]) <= rtol * sqrt(h_bb[c])) h_active[c] = 0;
            if (h_active[c]) all = false;
        }
        if (all) {
            result = KC_OK;
            break;
        }
        if (it >= maxit) break;
        KC_CUDA(cudaMemcpyAsync(active, h_active, sizeof(int) * ns, cudaMemcpyHostToDevice, s));
        KC_TRY(op.apply(N, p, q, ns, s));
        KC_TRY(dots(p, q, N, ns, partial, pq, s));
        KC_CUDA(cudaMemcpyAsync(h_pq, pq, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < nrhs; ++c)
            if (h_active[c] && !(h_pq[c] > 0.0)) {
                result = KC_EINDEF;
                h_active[c] = 0;
            }
        if (result == KC_EINDEF) break;
        ::kc::note_launch(), cg_update_xr_k<<<gb, 256, 0, s>>>(xs, r, p, q, rz, pq, active, N, ns);
        KC_TRY(precond(r, z));
        KC_TRY(dots(r, z, N, ns, partial, rzn, s));
        ::kc::note_launch(), cg_update_p_k<<<gb, 256, 0, s>>>(p, z, rz, rzn, active, N, ns);
        ::kc::note_launch(), copy_k<<<1, 32, 0, s>>>(rz, rzn, ns);
        KC_CUDA(cudaGetLastError());
        ++it;
    }
    KC_TRY(solver_check(S, s));
    // true residual b - (operator) x
    KC_TRY(op.apply(N, xs, q, ns, s));
    ::kc::note_launch(), sub_k<<<gb, 256, 0, s>>>(r, bp, q, n);
    KC_TRY(dots(r, r, N, ns, partial, rr, s));
    KC_CUDA(cudaMemcpyAsync(h_rr, rr, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    {
        double* tmp;
        KC_TRY(A.get(&tmp, N * nrhs));
        KC_CUDA(cudaMemcpy2DAsync(tmp, sizeof(double) * nrhs, xs, sizeof(double) * ns, sizeof(double) * nrhs, N,
                                  cudaMemcpyDeviceToDevice, s));
        KC_TRY(from_point_major(tmp, perm, N, nrhs, x_out, s));
    }
    KC_CUDA(cudaStreamSynchronize(s));
    if (iters_out) *iters_out = it;
    if (relres_out)
        for (int c = 0; c < nrhs; ++c) relres_out[c] = h_bb[c] > 0 ? sqrt(h_rr[c] / h_bb[c]) : 0.0;
    if (result == KC_ENOTCONV) return fail(KC_ENOTCONV, "refine: rtol not reached in maxit iterations");
    if (result == KC_EINDEF) return fail(KC_EINDEF, "refine: nonpositive curvature in CG");
    return KC_OK;
}

// ---------------------------------------------------------------- a9: PCA
__global__ void pca_scatter_k(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t N, int k,
                              const void* __restrict__ val, int is_f32, const int32_t* __restrict__ perm,
                              float* __restrict__ Lk) {
    int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = lane_id();
    if (j >= N) return;
    int64_t a = rowptr[j], b = rowptr[j + 1];
    int64_t orow = perm[j];
    for (int64_t e = a + lane; e < b; e += 32) {
        int c = col[e];
        if (c >= k) break;
        float v = is_f32 ? ((const float*)val)[e] : (float)((const double*)val)[e];
        Lk[(int64_t)c * N + orow] = v;
    }
}

kc_status pca_truncate_impl(const kc_pattern* P, int prec, const void* val, const int32_t* perm, int k, float* Lk,
                            cudaStream_t s) {
    if (k < 0 || k > P->N) return fail(KC_EINVAL, "k must be in 0..N");
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "bad prec");
    KC_CUDA(cudaMemsetAsync(Lk, 0, sizeof(float) * P->N * (size_t)k, s));
    if (k == 0) return KC_OK;
    ::kc::note_launch(), pca_scatter_k<<<blocks_for(P->N * 32, 256), 256, 0, s>>>(P->rowptr, P->col, P->N, k, val, prec == KC_FP32_FORM,
                                                             perm, Lk);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// w = Theta v (dense, FP32 entries, Dot2 tile sums combined in FP64), nrhs = 1
__global__ void __launch_bounds__(DM_THREADS) dense_theta_f32_k(const double* __restrict__ x, int64_t N, int d,
                                                              KernelParams kp, const double* __restrict__ v,
                                                              double* __restrict__ y) {
    __shared__ float sx[DM_THREADS * 4];
    __shared__ float sv[DM_THREADS];
    const int64_t j = (int64_t)blockIdx.x * DM_THREADS + threadIdx.x;
    float xj[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = 0; t < d; ++t) xj[t] = j < N ? (float)x[j * d + t] : 0.f;
    double acc = 0.0;
    for (int64_t k0 = 0; k0 < N; k0 += DM_THREADS) {
        __syncthreads();
        {
            int64_t k = k0 + threadIdx.x;
            for (int t = 0; t < 4; ++t) sx[threadIdx.x * 4 + t] = (k < N && t < d) ? (float)x[k * d + t] : 0.f;
            sv[threadIdx.x] = k < N ? (float)v[k] : 0.f;
        }
        __syncthreads();
        const int kn = (int)min((int64_t)DM_THREADS, N - k0);
        float s = 0.f, c = 0.f;
        for (int kk = 0; kk < kn; ++kk) {
            float u0 = xj[0] - sx[kk * 4], u1 = xj[1] - sx[kk * 4 + 1], u2 = xj[2] - sx[kk * 4 + 2],
                  u3 = xj[3] - sx[kk * 4 + 3];
            float rr = fmaf(u0, u0, fmaf(u1, u1, fmaf(u2, u2, u3 * u3)));
            float th = cov_f32(kp, sqrtf(rr));
            float a = th, b = sv[kk];
            float pr = a * b, ep = fmaf(a, b, -pr);
            float ns = s + pr, zz = ns - s;
            float es = (s - (ns - zz)) + (pr - zz);
            s = ns;
            c += ep + es;
        }
        acc += (double)s + (double)c;
    }
    if (j < N) y[j] = acc + kp.nugget * v[j];
}

// c[a] = sum_i Lk[a*N+i] v[i]
__global__ void lkt_v_k(const float* __restrict__ Lk, const double* __restrict__ v, int64_t N,
                        double* __restrict__ c) {
    __shared__ double sh[8];
    const int a = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s = fma((double)Lk[(int64_t)a * N + i], v[i], s);
    s = warp_sum(s);
    if (lane_id() == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
        c[a] = t;
    }
}
// w[i] -= sum_a Lk[a*N+i] c[a]
__global__ void w_minus_lk_c_k(const float* __restrict__ Lk, const double* __restrict__ c, int k, int64_t N,
                               double* __restrict__ w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        double s = 0.0;
        for (int a = 0; a < k; ++a) s = fma((double)Lk[(int64_t)a * N + i], c[a], s);
        w[i] -= s;
    }
}
__global__ void scale_k(const double* __restrict__ w, const double* __restrict__ nrm2, int64_t N,
                        double* __restrict__ v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        double n = sqrt(nrm2[0]);
        v[i] = n > 0.0 ? w[i] / n : 0.0;
    }
}

kc_status pca_error_impl(const double* x, int64_t N, int d, const kc_kernel* kern, int k, const float* Lk,
                         const double* v0, int iters, double* est_out, cudaStream_t s) {
    KernelParams kp;
    KC_TRY(kernel_params(kern, &kp));
    if (d > 4) return fail(KC_EINVAL, "kc_pca_error supports d <= 4");
    Arena A(s);
    KC_TRY(upload_coef(kp, A, s));
    double *v, *w, *c, *partial, *sc;
    KC_TRY(A.get(&v, N));
    KC_TRY(A.get(&w, N));
    KC_TRY(A.get(&c, k > 0 ? k : 1));
    KC_TRY(A.get(&partial, RED_BLOCKS));
    KC_TRY(A.get(&sc, 2));
    KC_CUDA(cudaMemcpyAsync(v, v0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    for (int it = 0; it < iters; ++it) {
        ::kc::note_launch(), dense_theta_f32_k<<<blocks_for(N, DM_THREADS), DM_THREADS, 0, s>>>(x, N, d, kp, v, w);
        if (k > 0) {
            ::kc::note_launch(), lkt_v_k<<<k, 256, 0, s>>>(Lk, v, N, c);
            ::kc::note_launch(), w_minus_lk_c_k<<<blocks_for(N, 256), 256, 0, s>>>(Lk, c, k, N, w);
        }
        KC_TRY(dots(v, w, N, 1, partial, sc, s));
        KC_TRY(dots(w, w, N, 1, partial, sc + 1, s));
        ::kc::note_launch(), scale_k<<<blocks_for(N, 256), 256, 0, s>>>(w, sc + 1, N, v);
        KC_CUDA(cudaGetLastError());
    }
    double h[2] = {0, 0};
    KC_CUDA(cudaMemcpyAsync(h, sc, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (est_out) *est_out = fabs(h[0]);
    return KC_OK;
}

}  // namespace kc
