// The C ABI of libkchol (declared in include/kchol.h): argument checks and
// dispatch to the device implementations.  No torch types cross it.  Every
// entry point is an NVTX range of its own name (header-only NVTX: inert unless
// a profiler is attached).
#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace
#define KC_RANGE(name) NvtxRange kc_nvtx_range_(name)

namespace kc {
kc_status order_impl(const double* x, int64_t N, int d, int32_t* perm, double* l, double* x_ord, cudaStream_t s);
kc_status pattern_count_impl(const double* x_ord, const double* l, int64_t N, int d, double rho, int rule,
                             int64_t* rowptr, int64_t* nnz_out, cudaStream_t s);
kc_status pattern_fill_impl(const double* x_ord, const double* l, int64_t N, int d, double rho, int rule,
                            const int64_t* rowptr, int32_t* col, cudaStream_t s);
kc_status pattern_begin_impl(const double* x_ord, const double* l, int64_t N, int d, double rho, int rule,
                             int64_t* rowptr, int64_t* nnz_out, void** out, cudaStream_t s);
kc_status pattern_end_impl(void* h, int32_t* col);
void pattern_abort_impl(void* h);
kc_status schedule_impl(int64_t N, const int64_t* rowptr, const int32_t* col, int64_t nnz, const double* x, int d,
                        int64_t* colptr, int32_t* rowidx, int64_t* slot, int32_t* level, int32_t* order,
                        int32_t* depth_out, cudaStream_t s);
kc_status factor_impl(const kc_pattern* P, const double* x, int d, const kc_kernel* kern, int prec, void* val,
                      double* diag, int64_t* zero_out, const kc_opts* o, cudaStream_t s);
kc_status solve_impl(const kc_pattern* P, int prec, const void* val, const double* diag, const kc_kernel* kern,
                     const int32_t* perm, const double* b, int nrhs, double* x, const kc_opts* o, cudaStream_t s);
kc_status refine_impl(const kc_pattern* P, const double* x_ord, int d, const kc_kernel* kern, int prec,
                      const void* val, const double* diag, const int32_t* perm, const double* b, int nrhs,
                      double rtol, int maxit, double* x_out, int32_t* iters_out, double* relres_out,
                      const kc_opts* o, cudaStream_t s);
kc_status solve_noalloc_impl(const kc_pattern* P, int prec, const void* val, const double* diag,
                             const kc_kernel* kern, const int32_t* perm, const double* b, int nrhs, double* x,
                             cudaStream_t s);
kc_status plan_create_impl(const kc_pattern* P, const double* x, int d, const kc_kernel* kerns, int nsets,
                           const int32_t* col_set, int prec, const kc_opts* o, kc_factor_plan** out, cudaStream_t s);
kc_status plan_launch_impl(kc_factor_plan* pl, void* val, double* diag, cudaStream_t s);
kc_status plan_finish_impl(kc_factor_plan* pl, int64_t* zero_out, cudaStream_t s);
kc_status plan_tune_impl(kc_factor_plan* pl, void* val, double* diag, int32_t* lanes_out, int32_t* unroll_out,
                         double* best_ms_out, cudaStream_t s);
void plan_destroy_impl(kc_factor_plan* pl);
kc_status pattern_concat_impl(int nsets, const int64_t* const* rowptrs, const int32_t* const* cols, const int64_t* Ns,
                              int64_t* rowptr_out, int32_t* col_out, int32_t* set_out, cudaStream_t s);
kc_status points_concat_impl(int nsets, const double* const* xs, const int64_t* Ns, const int32_t* ds, int dout,
                             double* out, cudaStream_t s);
kc_status index_concat_impl(int nsets, const int32_t* const* idx, const int64_t* Ns, int32_t* out, cudaStream_t s);
kc_status pca_truncate_impl(const kc_pattern* P, int prec, const void* val, const int32_t* perm, int k, float* Lk,
                            cudaStream_t s);
kc_status pca_error_impl(const double* x, int64_t N, int d, const kc_kernel* kern, int k, const float* Lk,
                         const double* v0, int iters, double* est_out, cudaStream_t s);
kc_status factor_matvec_impl(const kc_pattern* P, int prec, const void* val, const double* diag, const int32_t* perm,
                             const double* in, int nrhs, double* out, int which, cudaStream_t s);
kc_status logdet_impl(const kc_pattern* P, const double* diag, double* logdet_out, int64_t* zero_out, cudaStream_t s);
kc_status factor_blocked_impl(const kc_pattern* P, const double* x, int d, const kc_kernel* kern, int prec, void* val,
                              double* diag, int64_t* zero_out, const kc_opts* o, cudaStream_t s);
kc_status frob_error_impl(const kc_pattern* P, int prec, const void* val, const double* diag, const double* x_ord,
                          int d, const kc_kernel* kern, const int32_t* perm, const int64_t* pi, const int64_t* pj,
                          int64_t m, const int8_t* keep, double* num2_out, double* den2_out, int64_t* kept_out,
                          cudaStream_t s);
kc_status kernel_eval_impl(const kc_kernel* kern, int prec, const double* r, int64_t n, double* out, cudaStream_t s);
kc_status factor_given_impl(const kc_pattern* P, const double* aval, int prec, void* val, double* diag,
                            int64_t* zero_out, const kc_opts* o, cudaStream_t s);
kc_status pattern_validate_impl(const kc_pattern* P, cudaStream_t s);
kc_status supernodal_impl(const double* x_ord, const double* l, int d, double rho, const kc_pattern* P,
                          int32_t* newm, int32_t* level, int32_t* node_out, int32_t* color_out, double* x_new,
                          int64_t* rowptr, int64_t* nnz_out, int32_t* col, int64_t col_cap, cudaStream_t s);
kc_status refine_sparse_impl(const kc_pattern* P, int prec, const void* val, const double* diag,
                             const int32_t* perm, const int64_t* arp, const int32_t* acol, const double* aval,
                             const double* b, int nrhs, double rtol, int maxit, double* x_out, int32_t* iters_out,
                             double* relres_out, const kc_opts* o, cudaStream_t s);
kc_status pattern_reverse_impl(int64_t N, const int64_t* colptr, const int32_t* rowidx, int64_t* rowptr, int32_t* col,
                               cudaStream_t s);
kc_status gather_impl(int64_t N, const int64_t* rowptr, const int32_t* col, const int32_t* orig, const int64_t* arp,
                      const int32_t* acol, const double* aval_in, double* aval, int64_t* outside_out,
                      cudaStream_t s);
}  // namespace kc

using namespace kc;

static kc_status check_pattern(const kc_pattern* P) {
    if (!P) return fail(KC_EINVAL, "pattern is NULL");
    if (P->N < 1) return fail(KC_EINVAL, "pattern N must be >= 1");
    if (P->N > INT32_MAX) return fail(KC_EINVAL, "N must fit in int32");
    if (P->nnz < P->N) return fail(KC_EINVAL, "pattern nnz must be >= N (every row holds its diagonal)");
    if (!P->rowptr || !P->col || !P->colptr || !P->rowidx || !P->slot || !P->order)
        return fail(KC_EINVAL, "pattern has a NULL array (run kc_schedule first)");
    return KC_OK;
}

static kc_status check_points(const void* x, int64_t N, int32_t d) {
    if (!x) return fail(KC_EINVAL, "points are NULL");
    if (N < 1 || N > INT32_MAX) return fail(KC_EINVAL, "N must be in 1..2^31-1");
    if (d < 1 || d > 32) return fail(KC_EINVAL, "d must be in 1..32");
    return KC_OK;
}

extern "C" {

const char* kc_last_error(void) { return last_error_cstr(); }

int32_t kc_abi_version(void) { return KC_ABI_VERSION; }

int64_t kc_launch_count(void) { return launch_count(); }

kc_status kc_scratch_trim(int64_t keep_bytes) {
    KC_RANGE("kc_scratch_trim");
    return scratch_trim(keep_bytes);
}

double kc_last_factor_kernel_ms(void) { return factor_kernel_ms(); }

kc_status kc_order_points(const double* x, int64_t N, int32_t d, int32_t* perm, double* l, double* x_ord,
                          void* stream) {
    KC_RANGE("kc_order_points");
    KC_TRY(check_points(x, N, d));
    if (!perm || !l || !x_ord) return fail(KC_EINVAL, "output arrays must be non-NULL");
    return order_impl(x, N, d, perm, l, x_ord, (cudaStream_t)stream);
}

kc_status kc_pattern_count(const double* x_ord, const double* l, int64_t N, int32_t d, double rho, int32_t rule,
                           int64_t* rowptr, int64_t* nnz_out, void* stream) {
    KC_RANGE("kc_pattern_count");
    KC_TRY(check_points(x_ord, N, d));
    if (!l || !rowptr) return fail(KC_EINVAL, "l and rowptr must be non-NULL");
    if (!(rho > 0.0)) return fail(KC_EINVAL, "rho must be > 0");
    if (rule != KC_RULE_MAX && rule != KC_RULE_MIN) return fail(KC_EINVAL, "rule must be KC_RULE_MAX or KC_RULE_MIN");
    return pattern_count_impl(x_ord, l, N, d, rho, rule, rowptr, nnz_out, (cudaStream_t)stream);
}

kc_status kc_pattern_fill(const double* x_ord, const double* l, int64_t N, int32_t d, double rho, int32_t rule,
                          const int64_t* rowptr, int32_t* col, void* stream) {
    KC_RANGE("kc_pattern_fill");
    KC_TRY(check_points(x_ord, N, d));
    if (!l || !rowptr || !col) return fail(KC_EINVAL, "l, rowptr and col must be non-NULL");
    if (!(rho > 0.0)) return fail(KC_EINVAL, "rho must be > 0");
    if (rule != KC_RULE_MAX && rule != KC_RULE_MIN) return fail(KC_EINVAL, "rule must be KC_RULE_MAX or KC_RULE_MIN");
    return pattern_fill_impl(x_ord, l, N, d, rho, rule, rowptr, col, (cudaStream_t)stream);
}

kc_status kc_pattern_begin(const double* x_ord, const double* l, int64_t N, int32_t d, double rho, int32_t rule,
                           int64_t* rowptr, int64_t* nnz_out, kc_pattern_builder** builder_out, void* stream) {
    KC_RANGE("kc_pattern_begin");
    if (!builder_out) return fail(KC_EINVAL, "builder_out must be non-NULL");
    *builder_out = nullptr;
    KC_TRY(check_points(x_ord, N, d));
    if (!l || !rowptr) return fail(KC_EINVAL, "l and rowptr must be non-NULL");
    if (!(rho > 0.0)) return fail(KC_EINVAL, "rho must be > 0");
    if (rule != KC_RULE_MAX && rule != KC_RULE_MIN) return fail(KC_EINVAL, "rule must be KC_RULE_MAX or KC_RULE_MIN");
    void* h = nullptr;
    KC_TRY(pattern_begin_impl(x_ord, l, N, d, rho, rule, rowptr, nnz_out, &h, (cudaStream_t)stream));
    *builder_out = (kc_pattern_builder*)h;
    return KC_OK;
}

kc_status kc_pattern_end(kc_pattern_builder* builder, int32_t* col) {
    KC_RANGE("kc_pattern_end");
    if (!builder) return fail(KC_EINVAL, "builder must be non-NULL");
    if (!col) {
        pattern_abort_impl(builder);
        return fail(KC_EINVAL, "col must be non-NULL (the builder was released)");
    }
    return pattern_end_impl(builder, col);
}

void kc_pattern_abort(kc_pattern_builder* builder) { pattern_abort_impl(builder); }

kc_status kc_schedule(int64_t N, const int64_t* rowptr, const int32_t* col, const double* x_ord, int32_t d,
                      int64_t* colptr, int32_t* rowidx, int64_t* slot, int32_t* level, int32_t* order,
                      int32_t* depth_out, void* stream) {
    KC_RANGE("kc_schedule");
    if (N < 1 || N > INT32_MAX) return fail(KC_EINVAL, "N must be in 1..2^31-1");
    if (!rowptr || !col || !colptr || !rowidx || !slot || !level || !order)
        return fail(KC_EINVAL, "arrays must be non-NULL");
    if (x_ord && d < 1) return fail(KC_EINVAL, "d must be >= 1 when x_ord is given");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t nnz = 0;
    KC_CUDA(cudaMemcpyAsync(&nnz, rowptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (nnz < N) return fail(KC_EINVAL, "rowptr[N] must be >= N");
    return schedule_impl(N, rowptr, col, nnz, x_ord, d, colptr, rowidx, slot, level, order, depth_out, s);
}

kc_status kc_factor(const kc_pattern* pat, const double* x_ord, int32_t d, const kc_kernel* kern, int32_t prec,
                    void* val, double* diag, int64_t* zero_pivots_out, const kc_opts* opts, void* stream) {
    KC_RANGE("kc_factor");
    KC_TRY(check_pattern(pat));
    KC_TRY(check_points(x_ord, pat->N, d));
    if (!val || !diag) return fail(KC_EINVAL, "val and diag must be non-NULL");
    return factor_impl(pat, x_ord, d, kern, prec, val, diag, zero_pivots_out, opts, (cudaStream_t)stream);
}

kc_status kc_factor_blocked(const kc_pattern* pat, const double* x_ord, int32_t d, const kc_kernel* kern,
                            int32_t prec, void* val, double* diag, int64_t* zero_pivots_out, const kc_opts* opts,
                            void* stream) {
    KC_RANGE("kc_factor_blocked");
    KC_TRY(check_pattern(pat));
    KC_TRY(check_points(x_ord, pat->N, d));
    if (!val || !diag) return fail(KC_EINVAL, "val and diag must be non-NULL");
    return factor_blocked_impl(pat, x_ord, d, kern, prec, val, diag, zero_pivots_out, opts, (cudaStream_t)stream);
}

kc_status kc_solve(const kc_pattern* pat, int32_t prec, const void* val, const double* diag, const kc_kernel* kern,
                   const int32_t* perm, const double* b, int32_t nrhs, double* x, const kc_opts* opts, void* stream) {
    KC_RANGE("kc_solve");
    KC_TRY(check_pattern(pat));
    if (!val || !diag || !perm || !b || !x) return fail(KC_EINVAL, "arrays must be non-NULL");
    return solve_impl(pat, prec, val, diag, kern, perm, b, nrhs, x, opts, (cudaStream_t)stream);
}

kc_status kc_factor_plan_create(const kc_pattern* pat, const double* x_ord, int32_t d, const kc_kernel* kerns,
                                int32_t nsets, const int32_t* col_set, int32_t prec, const kc_opts* opts,
                                kc_factor_plan** out, void* stream) {
    KC_RANGE("kc_factor_plan_create");
    KC_TRY(check_pattern(pat));
    KC_TRY(check_points(x_ord, pat->N, d));
    if (!kerns || !out) return fail(KC_EINVAL, "kerns and out must be non-NULL");
    return plan_create_impl(pat, x_ord, d, kerns, nsets, col_set, prec, opts, out, (cudaStream_t)stream);
}

kc_status kc_factor_plan_launch(kc_factor_plan* plan, void* val, double* diag, void* stream) {
    KC_RANGE("kc_factor_plan_launch");
    if (!plan || !val || !diag) return fail(KC_EINVAL, "plan, val and diag must be non-NULL");
    return plan_launch_impl(plan, val, diag, (cudaStream_t)stream);
}

kc_status kc_factor_plan_finish(kc_factor_plan* plan, int64_t* zero_pivots_out, void* stream) {
    KC_RANGE("kc_factor_plan_finish");
    if (!plan) return fail(KC_EINVAL, "plan is NULL");
    return plan_finish_impl(plan, zero_pivots_out, (cudaStream_t)stream);
}

kc_status kc_factor_plan_tune(kc_factor_plan* plan, void* val, double* diag, int32_t* lanes_out, int32_t* unroll_out,
                              double* best_ms_out, void* stream) {
    KC_RANGE("kc_factor_plan_tune");
    if (!plan || !val || !diag) return fail(KC_EINVAL, "plan, val and diag must be non-NULL");
    return plan_tune_impl(plan, val, diag, lanes_out, unroll_out, best_ms_out, (cudaStream_t)stream);
}

void kc_factor_plan_destroy(kc_factor_plan* plan) { plan_destroy_impl(plan); }

kc_status kc_pattern_concat(int32_t nsets, const int64_t* const* rowptrs, const int32_t* const* cols, const int64_t* Ns,
                            int64_t* rowptr_out, int32_t* col_out, int32_t* set_out, void* stream) {
    KC_RANGE("kc_pattern_concat");
    if (nsets < 1 || !rowptrs || !cols || !Ns || !rowptr_out || !col_out) return fail(KC_EINVAL, "bad concat arguments");
    return pattern_concat_impl(nsets, rowptrs, cols, Ns, rowptr_out, col_out, set_out, (cudaStream_t)stream);
}

kc_status kc_points_concat(int32_t nsets, const double* const* xs, const int64_t* Ns, const int32_t* ds, int32_t dout,
                           double* out, void* stream) {
    KC_RANGE("kc_points_concat");
    if (nsets < 1 || !xs || !Ns || !ds || !out || dout < 1) return fail(KC_EINVAL, "bad concat arguments");
    return points_concat_impl(nsets, xs, Ns, ds, dout, out, (cudaStream_t)stream);
}

kc_status kc_index_concat(int32_t nsets, const int32_t* const* idx, const int64_t* Ns, int32_t* out, void* stream) {
    KC_RANGE("kc_index_concat");
    if (nsets < 1 || !idx || !Ns || !out) return fail(KC_EINVAL, "bad concat arguments");
    return index_concat_impl(nsets, idx, Ns, out, (cudaStream_t)stream);
}

kc_status kc_solve_noalloc(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                           const kc_kernel* kern, const int32_t* perm, const double* b, int32_t nrhs, double* x,
                           void* stream) {
    KC_RANGE("kc_solve_noalloc");
    KC_TRY(check_pattern(pat));
    if (!val || !diag || !perm || !b || !x) return fail(KC_EINVAL, "arrays must be non-NULL");
    return solve_noalloc_impl(pat, prec, val, diag, kern, perm, b, nrhs, x, (cudaStream_t)stream);
}

kc_status kc_refine(const kc_pattern* pat, const double* x_ord, int32_t d, const kc_kernel* kern, int32_t prec,
                    const void* val, const double* diag, const int32_t* perm, const double* b, int32_t nrhs,
                    double rtol, int32_t maxit, double* x, int32_t* iters_out, double* relres_out,
                    const kc_opts* opts, void* stream) {
    KC_RANGE("kc_refine");
    KC_TRY(check_pattern(pat));
    KC_TRY(check_points(x_ord, pat->N, d));
    if (!val || !diag || !perm || !b || !x) return fail(KC_EINVAL, "arrays must be non-NULL");
    if (!(rtol > 0.0) || maxit < 0) return fail(KC_EINVAL, "need rtol > 0 and maxit >= 0");
    return refine_impl(pat, x_ord, d, kern, prec, val, diag, perm, b, nrhs, rtol, maxit, x, iters_out, relres_out,
                       opts, (cudaStream_t)stream);
}

kc_status kc_pca_truncate(const kc_pattern* pat, int32_t prec, const void* val, const int32_t* perm, int32_t k,
                          float* Lk, void* stream) {
    KC_RANGE("kc_pca_truncate");
    KC_TRY(check_pattern(pat));
    if (!val || !perm || (!Lk && k > 0)) return fail(KC_EINVAL, "arrays must be non-NULL");
    return pca_truncate_impl(pat, prec, val, perm, k, Lk, (cudaStream_t)stream);
}

kc_status kc_pca_error(const double* x, int64_t N, int32_t d, const kc_kernel* kern, int32_t k, const float* Lk,
                       const double* v0, int32_t iters, double* estimate_out, void* stream) {
    KC_RANGE("kc_pca_error");
    KC_TRY(check_points(x, N, d));
    if (k < 0 || k > N || (k > 0 && !Lk) || !v0 || iters < 1) return fail(KC_EINVAL, "bad PCA error arguments");
    return pca_error_impl(x, N, d, kern, k, Lk, v0, iters, estimate_out, (cudaStream_t)stream);
}

kc_status kc_kernel_eval(const kc_kernel* kern, int32_t prec, const double* r, int64_t n, double* out,
                         void* stream) {
    KC_RANGE("kc_kernel_eval");
    if (n < 0 || (n > 0 && (!r || !out))) return fail(KC_EINVAL, "bad kernel evaluation arguments");
    return kernel_eval_impl(kern, prec, r, n, out, (cudaStream_t)stream);
}

static kc_status matvec_entry(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                              const int32_t* perm, const double* in, int32_t nrhs, double* out, int which,
                              void* stream) {
    KC_TRY(check_pattern(pat));
    if (!val || !diag || !perm || !in || !out) return fail(KC_EINVAL, "arrays must be non-NULL");
    return factor_matvec_impl(pat, prec, val, diag, perm, in, nrhs, out, which, (cudaStream_t)stream);
}

kc_status kc_l_matvec(const kc_pattern* pat, int32_t prec, const void* val, const double* diag, const int32_t* perm,
                      const double* z, int32_t nrhs, double* y, void* stream) {
    KC_RANGE("kc_l_matvec");
    return matvec_entry(pat, prec, val, diag, perm, z, nrhs, y, 0, stream);
}

kc_status kc_lt_matvec(const kc_pattern* pat, int32_t prec, const void* val, const double* diag, const int32_t* perm,
                       const double* v, int32_t nrhs, double* y, void* stream) {
    KC_RANGE("kc_lt_matvec");
    return matvec_entry(pat, prec, val, diag, perm, v, nrhs, y, 1, stream);
}

kc_status kc_llt_matvec(const kc_pattern* pat, int32_t prec, const void* val, const double* diag, const int32_t* perm,
                        const double* v, int32_t nrhs, double* y, void* stream) {
    KC_RANGE("kc_llt_matvec");
    return matvec_entry(pat, prec, val, diag, perm, v, nrhs, y, 2, stream);
}

kc_status kc_logdet(const kc_pattern* pat, const double* diag, double* logdet_out, int64_t* zero_pivots_out,
                    void* stream) {
    KC_RANGE("kc_logdet");
    KC_TRY(check_pattern(pat));
    if (!diag || !logdet_out) return fail(KC_EINVAL, "diag and logdet_out must be non-NULL");
    return logdet_impl(pat, diag, logdet_out, zero_pivots_out, (cudaStream_t)stream);
}

kc_status kc_frob_error(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                        const double* x_ord, int32_t d, const kc_kernel* kern, const int32_t* perm, const int64_t* pi,
                        const int64_t* pj, int64_t m, const int8_t* keep, double* num2_out, double* den2_out,
                        int64_t* kept_out, void* stream) {
    KC_RANGE("kc_frob_error");
    KC_TRY(check_pattern(pat));
    KC_TRY(check_points(x_ord, pat->N, d));
    if (m < 0 || (m > 0 && (!pi || !pj))) return fail(KC_EINVAL, "kc_frob_error: bad pair arrays");
    if (!val || !diag || !perm || !num2_out || !den2_out) return fail(KC_EINVAL, "arrays must be non-NULL");
    return frob_error_impl(pat, prec, val, diag, x_ord, d, kern, perm, pi, pj, m, keep, num2_out, den2_out, kept_out,
                           (cudaStream_t)stream);
}

kc_status kc_pattern_reverse(int64_t N, const int64_t* colptr, const int32_t* rowidx, int64_t* rowptr_out,
                             int32_t* col_out, void* stream) {
    KC_RANGE("kc_pattern_reverse");
    if (N < 1 || N > INT32_MAX) return fail(KC_EINVAL, "N must be in 1..2^31-1");
    if (!colptr || !rowidx || !rowptr_out || !col_out) return fail(KC_EINVAL, "arrays must be non-NULL");
    return pattern_reverse_impl(N, colptr, rowidx, rowptr_out, col_out, (cudaStream_t)stream);
}

kc_status kc_gather_entries(int64_t N, const int64_t* rowptr, const int32_t* col, const int32_t* orig,
                            const int64_t* a_rowptr, const int32_t* a_col, const double* a_val, double* aval_out,
                            int64_t* outside_out, void* stream) {
    KC_RANGE("kc_gather_entries");
    if (N < 1 || N > INT32_MAX) return fail(KC_EINVAL, "N must be in 1..2^31-1");
    if (!rowptr || !col || !orig || !a_rowptr || !a_col || !a_val || !aval_out)
        return fail(KC_EINVAL, "arrays must be non-NULL");
    return gather_impl(N, rowptr, col, orig, a_rowptr, a_col, a_val, aval_out, outside_out, (cudaStream_t)stream);
}

kc_status kc_factor_given(const kc_pattern* pat, const double* aval, int32_t prec, void* val, double* diag,
                          int64_t* zero_pivots_out, const kc_opts* opts, void* stream) {
    KC_RANGE("kc_factor_given");
    KC_TRY(check_pattern(pat));
    if (!aval || !val || !diag) return fail(KC_EINVAL, "arrays must be non-NULL");
    return factor_given_impl(pat, aval, prec, val, diag, zero_pivots_out, opts, (cudaStream_t)stream);
}

kc_status kc_refine_sparse(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                           const int32_t* perm, const int64_t* a_rowptr, const int32_t* a_col, const double* a_val,
                           const double* b, int32_t nrhs, double rtol, int32_t maxit, double* x, int32_t* iters_out,
                           double* relres_out, const kc_opts* opts, void* stream) {
    KC_RANGE("kc_refine_sparse");
    KC_TRY(check_pattern(pat));
    if (!val || !diag || !perm || !a_rowptr || !a_col || !a_val || !b || !x)
        return fail(KC_EINVAL, "arrays must be non-NULL");
    if (!(rtol > 0.0) || maxit < 0) return fail(KC_EINVAL, "rtol must be > 0 and maxit >= 0");
    return refine_sparse_impl(pat, prec, val, diag, perm, a_rowptr, a_col, a_val, b, nrhs, rtol, maxit, x,
                              iters_out, relres_out, opts, (cudaStream_t)stream);
}

kc_status kc_supernodal_count(const double* x_ord, const double* l, int32_t d, double rho, const kc_pattern* pat,
                              int32_t* newm, int32_t* level, int32_t* node, int32_t* color, double* x_new,
                              int64_t* rowptr, int64_t* nnz_out, void* stream) {
    KC_RANGE("kc_supernodal_count");
    KC_TRY(check_pattern(pat));
    KC_TRY(check_points(x_ord, pat->N, d));
    if (!l || !newm || !x_new || !rowptr || !nnz_out) return fail(KC_EINVAL, "arrays must be non-NULL");
    if (!(rho >= 1.0)) return fail(KC_EINVAL, "the supernodal construction needs rho >= 1");
    return supernodal_impl(x_ord, l, d, rho, pat, newm, level, node, color, x_new, rowptr, nnz_out, nullptr, 0,
                           (cudaStream_t)stream);
}

kc_status kc_supernodal(const double* x_ord, const double* l, int32_t d, double rho, const kc_pattern* pat,
                        int32_t* newm, int32_t* level, int32_t* node, int32_t* color, double* x_new, int64_t* rowptr,
                        int32_t* col, int64_t col_capacity, int64_t* nnz_out, void* stream) {
    KC_RANGE("kc_supernodal");
    KC_TRY(check_pattern(pat));
    KC_TRY(check_points(x_ord, pat->N, d));
    if (!l || !newm || !x_new || !rowptr || !nnz_out || (col_capacity > 0 && !col))
        return fail(KC_EINVAL, "arrays must be non-NULL");
    if (!(rho >= 1.0)) return fail(KC_EINVAL, "the supernodal construction needs rho >= 1");
    return supernodal_impl(x_ord, l, d, rho, pat, newm, level, node, color, x_new, rowptr, nnz_out, col,
                           col_capacity, (cudaStream_t)stream);
}

kc_status kc_supernodal_fill(const double* x_ord, const double* l, int32_t d, double rho, const kc_pattern* pat,
                             const int64_t* rowptr, int32_t* col, void* stream) {
    KC_RANGE("kc_supernodal_fill");
    KC_TRY(check_pattern(pat));
    KC_TRY(check_points(x_ord, pat->N, d));
    if (!l || !rowptr || !col) return fail(KC_EINVAL, "arrays must be non-NULL");
    if (!(rho >= 1.0)) return fail(KC_EINVAL, "the supernodal construction needs rho >= 1");
    return supernodal_impl(x_ord, l, d, rho, pat, nullptr, nullptr, nullptr, nullptr, nullptr,
                           const_cast<int64_t*>(rowptr), nullptr, col, 0, (cudaStream_t)stream);
}

kc_status kc_pattern_validate(const kc_pattern* pat, void* stream) {
    KC_RANGE("kc_pattern_validate");
    KC_TRY(check_pattern(pat));
    return pattern_validate_impl(pat, (cudaStream_t)stream);
}

}  // extern "C"
