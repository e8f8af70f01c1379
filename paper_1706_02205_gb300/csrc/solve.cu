// a7: L L^T x = b with the sparse factor (task (2) of Section 1), as two
// sync-free level-scheduled triangular solves in one persistent launch each.
//
// Forward  L y = b:   y_j = (b_j - sum_{k in R_j} L_jk y_k) / L_jj, one warp per
//                     row, rows in (level, index) order; row j waits for the
//                     ready flags of its R_j.
// Backward L^T x = y: x_i = (y_i - sum_{j in C_i} L_ji x_j) / L_ii, over the
//                     CSC columns in reverse level order; wide columns are cut
//                     into the same chunks as the factor's tasks, each chunk
//                     adds its partial sum atomically and the last chunk of a
//                     column finishes x_i.
// Vectors are point-major inside (v[k * nrhs + r]) so one entry's right-hand
// sides are contiguous; lanes map to (entry, rhs) pairs.  Sums are FP64 for
// both value types.  A dropped pivot (L_ii = 0) uses sqrt(Theta_ii).
#include "solver.cuh"

namespace kc {

template <typename T>
struct SolveArgs {
    int64_t N;
    int nrhs, NR;  // NR = nrhs rounded up to a power of two (<= 16)
    const int64_t* __restrict__ rowptr;
    const int32_t* __restrict__ col;
    const int64_t* __restrict__ colptr;
    const int32_t* __restrict__ rowidx;
    const int64_t* __restrict__ slot;
    const int32_t* __restrict__ order;
    const int2* __restrict__ tasks;
    int64_t ntasks;
    int rpt;
    const T* __restrict__ val;
    const double* __restrict__ diag;
    double diag_fallback;
    const double* b;  // point-major input
    double* y;        // point-major output of the forward solve / input of backward
    double* x;        // point-major output of the backward solve
    double* acc;      // point-major partial sums of wide columns
    unsigned* cnt;    // finished chunks per column (backward)
    int* ready;       // per point flag
    unsigned long long* ticket;
    int* status;
    long long spin_limit;
};

__device__ __forceinline__ bool wait_flag(const int* f, const int* status, long long limit) {
    if (ld_acquire_s32(f) != 0) return true;
    long long t0 = clock64();
    unsigned ns = 32;
    while (ld_acquire_s32(f) == 0) {
        if (clock64() - t0 > limit || ld_volatile_s32(status) != 0) return false;
        __nanosleep(ns);  // back off so waiting warps do not flood L2 with polls
        if (ns < 512) ns <<= 1;
    }
    return true;
}

template <typename T>
__global__ void __launch_bounds__(256) fwd_solve_k(SolveArgs<T> A) {
    const int lane = lane_id();
    const unsigned FULL = 0xffffffffu;
    const int per = 32 / A.NR;  // entries per warp step
    const int r = lane % A.NR, eo = lane / A.NR;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(A.ticket, 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= A.N) return;
        if (ld_volatile_s32(A.status) != 0) return;
        const int j = A.order[t];
        const int64_t a = A.rowptr[j], b = A.rowptr[j + 1] - 1;
        bool ok = true;
        for (int64_t e = a + lane; e < b && ok; e += 32) ok = wait_flag(&A.ready[__ldg(&A.col[e])], A.status, A.spin_limit);
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
            return;
        }
        __threadfence();
        __syncwarp();
        double s = 0.0;
        if (r < A.nrhs) {
            // four independent (col, val, y) loads in flight per lane
            double s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int64_t e = a + eo;
            for (; e + 3 * per < b; e += 4 * per) {
                const int k0 = __ldg(&A.col[e]), k1 = __ldg(&A.col[e + per]);
                const int k2 = __ldg(&A.col[e + 2 * per]), k3 = __ldg(&A.col[e + 3 * per]);
                const double v0 = (double)__ldg(&A.val[e]), v1 = (double)__ldg(&A.val[e + per]);
                const double v2 = (double)__ldg(&A.val[e + 2 * per]), v3 = (double)__ldg(&A.val[e + 3 * per]);
                s = fma(v0, __ldcg(&A.y[(int64_t)k0 * A.nrhs + r]), s);
                s1 = fma(v1, __ldcg(&A.y[(int64_t)k1 * A.nrhs + r]), s1);
                s2 = fma(v2, __ldcg(&A.y[(int64_t)k2 * A.nrhs + r]), s2);
                s3 = fma(v3, __ldcg(&A.y[(int64_t)k3 * A.nrhs + r]), s3);
            }
            for (; e < b; e += per) s = fma((double)__ldg(&A.val[e]), __ldcg(&A.y[(int64_t)__ldg(&A.col[e]) * A.nrhs + r]), s);
            s = (s + s1) + (s2 + s3);
        }
        for (int o = 16; o >= A.NR; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (eo == 0 && r < A.nrhs) {
            double dj = A.diag[j];
            if (!(dj > 0.0)) dj = A.diag_fallback;
            A.y[(int64_t)j * A.nrhs + r] = (A.b[(int64_t)j * A.nrhs + r] - s) / dj;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_s32(&A.ready[j], 1);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) bwd_solve_k(SolveArgs<T> A) {
    const int lane = lane_id();
    const unsigned FULL = 0xffffffffu;
    const int per = 32 / A.NR;
    const int r = lane % A.NR, eo = lane / A.NR;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(A.ticket, 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= A.ntasks) return;
        if (ld_volatile_s32(A.status) != 0) return;
        const int2 tk = A.tasks[A.ntasks - 1 - (int64_t)t];
        const int i = tk.x, c = tk.y;
        const int64_t c0 = A.colptr[i], c1 = A.colptr[i + 1];
        const int64_t m = c1 - c0 - 1;
        const unsigned nch = m <= 0 ? 1u : (unsigned)((m + A.rpt - 1) / A.rpt);
        const int64_t qs = c0 + 1 + (int64_t)c * A.rpt;
        const int64_t qe = min(c1, qs + A.rpt);
        bool ok = true;
        for (int64_t q = qs + lane; q < qe && ok; q += 32)
            ok = wait_flag(&A.ready[__ldg(&A.rowidx[q])], A.status, A.spin_limit);
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
            return;
        }
        __threadfence();
        __syncwarp();
        double s = 0.0;
        if (r < A.nrhs) {
            double s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int64_t q = qs + eo;
            for (; q + 3 * per < qe; q += 4 * per) {
                const int j0 = __ldg(&A.rowidx[q]), j1 = __ldg(&A.rowidx[q + per]);
                const int j2 = __ldg(&A.rowidx[q + 2 * per]), j3 = __ldg(&A.rowidx[q + 3 * per]);
                const int64_t p0 = __ldg(&A.slot[q]), p1 = __ldg(&A.slot[q + per]);
                const int64_t p2 = __ldg(&A.slot[q + 2 * per]), p3 = __ldg(&A.slot[q + 3 * per]);
                s = fma((double)__ldg(&A.val[p0]), __ldcg(&A.x[(int64_t)j0 * A.nrhs + r]), s);
                s1 = fma((double)__ldg(&A.val[p1]), __ldcg(&A.x[(int64_t)j1 * A.nrhs + r]), s1);
                s2 = fma((double)__ldg(&A.val[p2]), __ldcg(&A.x[(int64_t)j2 * A.nrhs + r]), s2);
                s3 = fma((double)__ldg(&A.val[p3]), __ldcg(&A.x[(int64_t)j3 * A.nrhs + r]), s3);
            }
            for (; q < qe; q += per) {
                const int j = __ldg(&A.rowidx[q]);
                s = fma((double)__ldg(&A.val[__ldg(&A.slot[q])]), __ldcg(&A.x[(int64_t)j * A.nrhs + r]), s);
            }
            s = (s + s1) + (s2 + s3);
        }
        for (int o = 16; o >= A.NR; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        bool finish = true;
        if (nch > 1) {
            if (eo == 0 && r < A.nrhs) atomicAdd(&A.acc[(int64_t)i * A.nrhs + r], s);
            __threadfence();
            __syncwarp();
            unsigned prev = 0;
            if (lane == 0) prev = atomicAdd(&A.cnt[i], 1u);
            prev = __shfl_sync(FULL, prev, 0);
            finish = (prev == nch - 1);
            if (finish) {
                __threadfence();
                s = __ldcg(&A.acc[(int64_t)i * A.nrhs + (r < A.nrhs ? r : 0)]);
            }
        }
        if (finish) {
            if (eo == 0 && r < A.nrhs) {
                double di = A.diag[i];
                if (!(di > 0.0)) di = A.diag_fallback;
                A.x[(int64_t)i * A.nrhs + r] = (A.y[(int64_t)i * A.nrhs + r] - s) / di;
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_s32(&A.ready[i], 1);
        }
    }
}

__global__ void to_point_major_k(const double* __restrict__ b, const int32_t* __restrict__ perm, int64_t N, int nrhs,
                                 double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * nrhs) {
        int64_t k = t / nrhs;
        int r = (int)(t % nrhs);
        out[t] = b[(int64_t)r * N + perm[k]];
    }
}
__global__ void from_point_major_k(const double* __restrict__ xp, const int32_t* __restrict__ perm, int64_t N,
                                   int nrhs, double* __restrict__ x) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * nrhs) {
        int64_t k = t / nrhs;
        int r = (int)(t % nrhs);
        x[(int64_t)r * N + perm[k]] = xp[t];
    }
}

kc_status solver_init(Solver& S, const kc_pattern* P, int nrhs_cap, const kc_opts* o, Arena& A, cudaStream_t s) {
    S.P = P;
    S.rpt = (o && o->rows_per_task > 0) ? o->rows_per_task : 64;
    if (o && o->spin_limit_cycles > 0) S.spin = o->spin_limit_cycles;
    KC_TRY(build_tasks(P, S.rpt, A, s, &S.tasks, &S.ntasks, &S.maxr));
    S.nrhs_cap = nrhs_cap;
    KC_TRY(A.get(&S.ready, P->N));
    KC_TRY(A.get(&S.cnt, P->N));
    KC_TRY(A.get(&S.acc, P->N * nrhs_cap));
    KC_TRY(A.get(&S.ticket, 2));
    KC_TRY(A.get(&S.status, 1));
    KC_TRY(A.get(&S.y, P->N * nrhs_cap));
    return KC_OK;
}

// z = (L L^T)^{-1} rhs, point-major, positions order.  Does not synchronise;
// the status word is checked by solver_check.
template <typename T>
kc_status solver_apply(Solver& S, const T* val, const double* diag, double diag_fallback, const double* rhs,
                       double* z, int nrhs, cudaStream_t s) {
    const kc_pattern* P = S.P;
    int NR = 1;
    while (NR < nrhs) NR <<= 1;
    SolveArgs<T> a;
    a.N = P->N;
    a.nrhs = nrhs;
    a.NR = NR;
    a.rowptr = P->rowptr;
    a.col = P->col;
    a.colptr = P->colptr;
    a.rowidx = P->rowidx;
    a.slot = P->slot;
    a.order = P->order;
    a.tasks = S.tasks;
    a.ntasks = S.ntasks;
    a.rpt = S.rpt;
    a.val = val;
    a.diag = diag;
    a.diag_fallback = diag_fallback;
    a.b = rhs;
    a.y = S.y;
    a.x = z;
    a.acc = S.acc;
    a.cnt = S.cnt;
    a.ready = S.ready;
    a.status = S.status;
    a.spin_limit = S.spin;
    int grid = sm_count() * 8;
    KC_CUDA(cudaMemsetAsync(S.ready, 0, sizeof(int) * P->N, s));
    KC_CUDA(cudaMemsetAsync(S.ticket, 0, 2 * sizeof(unsigned long long), s));
    KC_CUDA(cudaMemsetAsync(S.status, 0, sizeof(int), s));
    a.ticket = S.ticket;
    ::kc::note_launch(), fwd_solve_k<T><<<grid, 256, 0, s>>>(a);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaMemsetAsync(S.ready, 0, sizeof(int) * P->N, s));
    KC_CUDA(cudaMemsetAsync(S.cnt, 0, sizeof(unsigned) * P->N, s));
    KC_CUDA(cudaMemsetAsync(S.acc, 0, sizeof(double) * P->N * nrhs, s));
    a.ticket = S.ticket + 1;
    ::kc::note_launch(), bwd_solve_k<T><<<grid, 256, 0, s>>>(a);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}
template kc_status solver_apply<double>(Solver&, const double*, const double*, double, const double*, double*, int,
                                        cudaStream_t);
template kc_status solver_apply<float>(Solver&, const float*, const double*, double, const double*, double*, int,
                                       cudaStream_t);

kc_status solver_check(Solver& S, cudaStream_t s) {
    int h = 0;
    KC_CUDA(cudaMemcpyAsync(&h, S.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (h == DEV_TIMEOUT) return fail(KC_ETIMEOUT, "solve: a dependency wait ran out");
    if (h != 0) return fail(KC_ECUDA, "solve: device status " + std::to_string(h));
    return KC_OK;
}

kc_status to_point_major(const double* b, const int32_t* perm, int64_t N, int nrhs, double* out, cudaStream_t s) {
    ::kc::note_launch(), to_point_major_k<<<blocks_for(N * nrhs, 256), 256, 0, s>>>(b, perm, N, nrhs, out);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}
kc_status from_point_major(const double* xp, const int32_t* perm, int64_t N, int nrhs, double* x, cudaStream_t s) {
    ::kc::note_launch(), from_point_major_k<<<blocks_for(N * nrhs, 256), 256, 0, s>>>(xp, perm, N, nrhs, x);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

kc_status solve_impl(const kc_pattern* P, int prec, const void* val, const double* diag, const kc_kernel* kern,
                     const int32_t* perm, const double* b, int nrhs, double* x, const kc_opts* o, cudaStream_t s) {
    KernelParams kp;
    KC_TRY(kernel_params(kern, &kp));
    if (nrhs < 1 || nrhs > 16) return fail(KC_EINVAL, "nrhs must be in 1..16");
    Arena A(s);
    Solver S;
    KC_TRY(solver_init(S, P, nrhs, o, A, s));
    double *bp, *zp;
    KC_TRY(A.get(&bp, P->N * nrhs));
    KC_TRY(A.get(&zp, P->N * nrhs));
    KC_TRY(to_point_major(b, perm, P->N, nrhs, bp, s));
    double fb = sqrt(kp.sigma2 + kp.nugget);
    if (prec == KC_FP64) KC_TRY(solver_apply<double>(S, (const double*)val, diag, fb, bp, zp, nrhs, s));
    else if (prec == KC_FP32_FORM) KC_TRY(solver_apply<float>(S, (const float*)val, diag, fb, bp, zp, nrhs, s));
    else return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
    KC_TRY(from_point_major(zp, perm, P->N, nrhs, x, s));
    return solver_check(S, s);
}

}  // namespace kc
