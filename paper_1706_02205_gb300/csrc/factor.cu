// a5+a6: ICHOL(0) of the Matern kernel matrix restricted to S (Algorithm 2,
// "Incomplete Cholesky factorization with sparsity pattern S"), in its
// left-looking form, as one persistent sync-free kernel.
//
//   for each column i (in dependency order):
//     p    = Theta_ii - sum_{k in R_i} L_ik^2              (FP64)
//     p <= 0  ->  the whole column i is zero (Section 4.4)
//     L_ii = sqrt(p)
//     L_ji = (Theta_ji - sum_{k in R_j cap R_i} L_jk L_ik) / L_ii,  j in C_i
//
// Work units ("tasks") are (column, chunk of up to `rows_per_task` rows of
// C_i), listed in (level, index) order and handed out by an atomic ticket.  A
// warp that takes a task waits (bounded spin, acquire loads) until every
// column k in R_i has published all its tasks, stages row i (indices and
// values) in shared memory, recomputes the pivot, and then for each row j of
// its chunk merges the prefix of row j (entries k < i) against the staged
// row: lanes split into groups of G; each lane walks the prefix with stride G
// and binary-searches its k in the staged row.  Theta_ji is evaluated from the
// coordinates in the kernel (entries are never stored).  The task publishes
// by a release increment of done[i].
//
// Forward progress: a task only waits on columns of lower level, whose tasks
// have smaller ticket numbers and were claimed by running warps, so the
// earliest unfinished task can always proceed.  Every wait is bounded: when it
// runs out the kernel records DEV_TIMEOUT in the status word and returns.
#include "common.cuh"

namespace kc {

template <typename T>
struct FactorArgs {
    int64_t N;
    int d;
    const double* __restrict__ x;
    const int64_t* __restrict__ rowptr;
    const int32_t* __restrict__ col;
    const int64_t* __restrict__ colptr;
    const int32_t* __restrict__ rowidx;
    const int64_t* __restrict__ slot;
    const int2* __restrict__ tasks;
    int64_t ntasks;
    int rpt;  // rows per task
    T* val;
    double* diag;
    unsigned* done;
    unsigned long long* ticket;
    int* status;
    unsigned long long* zero_piv;
    KernelParams kp;
    long long spin_limit;
    int hold_col;
    int cap;  // staged entries per warp
};

__device__ __forceinline__ unsigned n_tasks_of(const int64_t* __restrict__ colptr, int k, int rpt) {
    int64_t m = colptr[k + 1] - colptr[k] - 1;  // rows below the diagonal
    return m <= 0 ? 1u : (unsigned)((m + rpt - 1) / rpt);
}

// position of key k in sorted a[0..n), or -1
__device__ __forceinline__ int bsearch_smem(const int* a, int n, int k) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && a[lo] == k) ? lo : -1;
}
__device__ __forceinline__ int64_t bsearch_glob(const int32_t* __restrict__ a, int64_t lo, int64_t hi, int k) {
    int64_t end = hi;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(&a[mid]) < k) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && __ldg(&a[lo]) == k) ? lo : -1;
}

// Compensated accumulation (Dot2 of Ogita, Rump and Oishi, 2005):
// TwoProduct by fma, TwoSum of the running sum, errors summed separately.
struct Dot2 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        float p = a * b;
        float ep = fmaf(a, b, -p);
        float ns = s + p;
        float z = ns - s;
        float es = (s - (ns - z)) + (p - z);
        s = ns;
        c += ep + es;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
    Dot2 d;
    __device__ __forceinline__ void add(float a, float b) { d.add(a, b); }
    __device__ __forceinline__ double value() const { return d.value(); }
};

template <typename T>
__device__ __forceinline__ double theta_off(const FactorArgs<T>& A, const double* xj, const double* xi);

template <>
__device__ __forceinline__ double theta_off<double>(const FactorArgs<double>& A, const double* xj,
                                                    const double* xi) {
    double s = 0.0;
    for (int t = 0; t < A.d; ++t) {
        double u = xj[t] - xi[t];
        s = fma(u, u, s);
    }
    return matern_f64(sqrt(s), A.kp.nu_code, A.kp.scale, A.kp.sigma2);
}
template <>
__device__ __forceinline__ double theta_off<float>(const FactorArgs<float>& A, const double* xj, const double* xi) {
    float s = 0.f;
    for (int t = 0; t < A.d; ++t) {
        float u = (float)(xj[t] - xi[t]);
        s = fmaf(u, u, s);
    }
    return (double)matern_f32(sqrtf(s), A.kp.nu_code, (float)A.kp.scale, (float)A.kp.sigma2);
}

template <typename T>
__global__ void __launch_bounds__(256) ichol_persistent_k(FactorArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    int* s_idx = (int*)(smem + (size_t)w * A.cap * (sizeof(int) + sizeof(T)));
    T* s_val = (T*)(s_idx + A.cap);
    const unsigned FULL = 0xffffffffu;

    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(A.ticket, 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= A.ntasks) return;
        if (ld_volatile_s32(A.status) != 0) return;
        const int2 tk = A.tasks[t];
        const int i = tk.x, c = tk.y;
        const int64_t a0 = A.rowptr[i], a1 = A.rowptr[i + 1] - 1;  // R_i = col[a0..a1)
        const int nr = (int)(a1 - a0);

        // ---- wait until every column k in R_i is complete
        bool ok = true;
        for (int e = lane; e < nr && ok; e += 32) {
            const int k = __ldg(&A.col[a0 + e]);
            const unsigned need = n_tasks_of(A.colptr, k, A.rpt);
            const unsigned* f = &A.done[k];
            if (ld_acquire_u32(f) < need) {
                long long t0 = clock64();
                while (ld_acquire_u32(f) < need) {
                    if (clock64() - t0 > A.spin_limit || ld_volatile_s32(A.status) != 0) {
                        ok = false;
                        break;
                    }
                }
            }
        }
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
            return;
        }
        __threadfence();
        __syncwarp();

        // ---- stage row i, pivot in FP64
        const bool staged = nr <= A.cap;
        double ps = 0.0;
        for (int e = lane; e < nr; e += 32) {
            const T v = ldcg(&A.val[a0 + e]);
            if (staged) {
                s_idx[e] = __ldg(&A.col[a0 + e]);
                s_val[e] = v;
            }
            ps += (double)v * (double)v;
        }
        ps = warp_sum(ps);
        __syncwarp();
        const double p = (A.kp.sigma2 + A.kp.nugget) - ps;
        const bool zero = !(p > 0.0);
        const double Lii = zero ? 0.0 : sqrt(p);
        if (c == 0 && lane == 0) {
            A.val[a1] = (T)Lii;
            A.diag[i] = Lii;
            if (zero) atomicAdd(A.zero_piv, 1ULL);
        }
        const double* xi = A.x + (int64_t)i * A.d;

        // ---- rows of this chunk
        int G = 1;
        while (G < 32 && 2 * G <= nr) G <<= 1;
        const int ng = 32 / G, g = lane / G, sub = lane % G;
        const int64_t qs = A.colptr[i] + 1 + (int64_t)c * A.rpt;
        const int64_t qe = min(A.colptr[i + 1], qs + A.rpt);
        for (int64_t q0 = qs; q0 < qe; q0 += ng) {
            const int64_t q = q0 + g;
            const bool act = q < qe;
            Acc<T> acc;
            int j = 0;
            int64_t bij = 0;
            if (act) {
                j = __ldg(&A.rowidx[q]);
                bij = __ldg(&A.slot[q]);
                const int64_t b0 = __ldg(&A.rowptr[j]);
                if (!zero) {
                    for (int64_t e = b0 + sub; e < bij; e += G) {
                        const int k = __ldg(&A.col[e]);
                        if (staged) {
                            const int pos = bsearch_smem(s_idx, nr, k);
                            if (pos >= 0) acc.add(ldcg(&A.val[e]), s_val[pos]);
                        } else {
                            const int64_t pos = bsearch_glob(A.col, a0, a1, k);
                            if (pos >= 0) acc.add(ldcg(&A.val[e]), ldcg(&A.val[pos]));
                        }
                    }
                }
            }
            double s = acc.value();
            for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
            if (act && sub == 0) {
                double v = 0.0;
                if (!zero) {
                    const double th = theta_off<T>(A, A.x + (int64_t)j * A.d, xi);
                    v = (th - s) / Lii;
                }
                A.val[bij] = (T)v;
            }
        }

        // ---- publish
        __threadfence();
        __syncwarp();
        if (lane == 0 && i != A.hold_col) red_release_add_u32(&A.done[i], 1u);
    }
}

// tasks of column order[p]: n_tasks_of(order[p])
__global__ void task_count_k(const int32_t* __restrict__ order, const int64_t* __restrict__ colptr, int64_t N,
                             int rpt, int64_t* __restrict__ cnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) cnt[p] = n_tasks_of(colptr, order[p], rpt);
}
__global__ void task_fill_k(const int32_t* __restrict__ order, const int64_t* __restrict__ toff, int64_t N,
                            int2* __restrict__ tasks) {
    int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = lane_id();
    if (p < N) {
        int64_t a = toff[p], b = toff[p + 1];
        int i = order[p];
        for (int64_t t = a + lane; t < b; t += 32) tasks[t] = make_int2(i, (int)(t - a));
    }
}
__global__ void max_row_k(const int64_t* __restrict__ rowptr, int64_t N, int* __restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int m = 0;
    if (j < N) m = (int)(rowptr[j + 1] - rowptr[j] - 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane_id() == 0) atomicMax(out, m);
}

// Build the task list (level order) of a pattern; returns count on the host.
kc_status build_tasks(const kc_pattern* P, int rpt, Arena& A, cudaStream_t s, int2** tasks_out, int64_t* ntasks_out,
                      int* max_row_out) {
    int64_t N = P->N;
    int64_t* cnt;
    int64_t* toff;
    int* mr;
    KC_TRY(A.get(&cnt, N));
    KC_TRY(A.get(&toff, N + 1));
    KC_TRY(A.get(&mr, 1));
    ::kc::note_launch(), task_count_k<<<blocks_for(N, 256), 256, 0, s>>>(P->order, P->colptr, N, rpt, cnt);
    KC_TRY(exclusive_scan_i64(cnt, toff, N, A, s));
    KC_CUDA(cudaMemsetAsync(mr, 0, sizeof(int), s));
    ::kc::note_launch(), max_row_k<<<blocks_for(N, 256), 256, 0, s>>>(P->rowptr, N, mr);
    KC_CUDA(cudaGetLastError());
    int64_t nt = 0;
    int hmr = 0;
    KC_CUDA(cudaMemcpyAsync(&nt, toff + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaMemcpyAsync(&hmr, mr, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    int2* tasks;
    KC_TRY(A.get(&tasks, nt));
    ::kc::note_launch(), task_fill_k<<<blocks_for(N * 32, 256), 256, 0, s>>>(P->order, toff, N, tasks);
    KC_CUDA(cudaGetLastError());
    *tasks_out = tasks;
    *ntasks_out = nt;
    *max_row_out = hmr;
    return KC_OK;
}

template <typename T>
static kc_status factor_run(const kc_pattern* P, const double* x, int d, const KernelParams& kp, T* val,
                            double* diag, int64_t* zero_out, const kc_opts* o, cudaStream_t s) {
    Arena A(s);
    const int rpt = (o && o->rows_per_task > 0) ? o->rows_per_task : 64;
    const int warps = (o && o->warps_per_cta > 0) ? o->warps_per_cta : 8;
    if (warps > 8) return fail(KC_EINVAL, "warps_per_cta must be <= 8");
    int2* tasks;
    int64_t nt;
    int maxr;
    KC_TRY(build_tasks(P, rpt, A, s, &tasks, &nt, &maxr));

    unsigned* done;
    unsigned long long* ticket;
    unsigned long long* zp;
    int* status;
    KC_TRY(A.get(&done, P->N));
    KC_TRY(A.get(&ticket, 1));
    KC_TRY(A.get(&zp, 1));
    KC_TRY(A.get(&status, 1));
    KC_CUDA(cudaMemsetAsync(done, 0, sizeof(unsigned) * P->N, s));
    KC_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s));
    KC_CUDA(cudaMemsetAsync(zp, 0, sizeof(unsigned long long), s));
    KC_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));

    FactorArgs<T> a;
    a.N = P->N;
    a.d = d;
    a.x = x;
    a.rowptr = P->rowptr;
    a.col = P->col;
    a.colptr = P->colptr;
    a.rowidx = P->rowidx;
    a.slot = P->slot;
    a.tasks = tasks;
    a.ntasks = nt;
    a.rpt = rpt;
    a.val = val;
    a.diag = diag;
    a.done = done;
    a.ticket = ticket;
    a.status = status;
    a.zero_piv = zp;
    a.kp = kp;
    a.spin_limit = (o && o->spin_limit_cycles > 0) ? o->spin_limit_cycles : 4000000000LL;
    a.hold_col = (o && o->test_hold_column > 0) ? o->test_hold_column - 1 : -1;
    int cap = 64;
    while (cap < maxr && cap < 1024) cap *= 2;
    a.cap = cap;
    size_t smem = (size_t)warps * cap * (sizeof(int) + sizeof(T));
    KC_CUDA(cudaFuncSetAttribute(ichol_persistent_k<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ichol_persistent_k<T>, warps * 32, smem));
    if (o && o->ctas_per_sm > 0 && o->ctas_per_sm < per_sm) per_sm = o->ctas_per_sm;
    if (per_sm < 1) per_sm = 1;
    int grid = sm_count() * per_sm;
    cudaEvent_t e0, e1;
    KC_CUDA(cudaEventCreate(&e0));
    KC_CUDA(cudaEventCreate(&e1));
    KC_CUDA(cudaEventRecord(e0, s));
    ::kc::note_launch(), ichol_persistent_k<T><<<grid, warps * 32, smem, s>>>(a);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaEventRecord(e1, s));
    int h_status = 0;
    unsigned long long h_zp = 0;
    KC_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaMemcpyAsync(&h_zp, zp, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    KC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_factor_kernel_ms(ms);
    if (zero_out) *zero_out = (int64_t)h_zp;
    if (h_status == DEV_TIMEOUT) return fail(KC_ETIMEOUT, "factor: a dependency wait ran out");
    if (h_status != 0) return fail(KC_ECUDA, "factor: device status " + std::to_string(h_status));
    return KC_OK;
}

kc_status factor_impl(const kc_pattern* P, const double* x, int d, const kc_kernel* kern, int prec, void* val,
                      double* diag, int64_t* zero_out, const kc_opts* o, cudaStream_t s) {
    KernelParams kp;
    KC_TRY(kernel_params(kern, &kp));
    if (prec == KC_FP64) return factor_run<double>(P, x, d, kp, (double*)val, diag, zero_out, o, s);
    if (prec == KC_FP32_FORM) return factor_run<float>(P, x, d, kp, (float*)val, diag, zero_out, o, s);
    return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
}

}  // namespace kc
