/*
 * libkchol -- sparse Cholesky factorisation of dense Matern kernel matrices
 * on one GB300 (sm_103a), following Schaefer, Sullivan and Owhadi,
 * "Compression, inversion, and approximate PCA of dense kernel matrices at
 * near-linear computational complexity" (arXiv:1706.02205).
 *
 * The method: order the points x_1..x_N by the maximin ordering (Section 2.3),
 * keep the sparsity pattern S_rho = {(i,j): dist(x_i,x_j) <= rho max(l_i,l_j)}
 * (Section 2.3), and run zero fill-in incomplete Cholesky ICHOL(0) (Algorithm 2)
 * on the kernel matrix Theta restricted to S, with Theta_ij evaluated from the
 * coordinates.  The factor L then serves the tasks of Section 1: solves with
 * Theta (task (2)) and rank-k PCA (task (5), Section 2.5).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Plain C ABI.  Pointers marked "device" are CUDA device pointers owned by
 *    the caller; pointers marked "host" are ordinary host memory.  The library
 *    never frees caller memory.  Internal scratch is taken stream-ordered on
 *    the given stream from a private memory pool per device (created on the
 *    library's first call on that device; the device's default pool, which
 *    cudaMallocAsync uses for everyone else in the process, is not touched)
 *    and released before the call returns.  The private pool keeps up to
 *    16 GiB of released scratch mapped for the next call, so repeated calls do
 *    not map GBs afresh; kc_scratch_trim hands it back to the driver.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Kernels are enqueued on it.  A call that returns a size to the host
 *    (marked "synchronises") waits for the stream.
 *  - Points: double x[N*d], row-major, original order.  After ordering,
 *    "position" k means the k-th point of the maximin order; perm[k] is its
 *    original index and x_ord[k*d+t] its coordinates.
 *  - The pattern of L is CSR by rows in positions: rowptr[N+1] (int64),
 *    col[nnz] (int32) ascending in each row, the diagonal last in each row.
 *  - Every call returns a kc_status; KC_OK is 0.  kc_last_error() gives a
 *    message for the calling thread's last failure.
 *  - Squared distances are summed coordinate by coordinate, each operation
 *    rounded separately (no fused multiply-add), so ordering and pattern are
 *    bit-identical to a CPU implementation of their definitions.
 */
#ifndef KCHOL_H
#define KCHOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KC_OK = 0,
    KC_EINVAL = 1,     /* bad argument */
    KC_ENOMEM = 2,     /* scratch allocation failed */
    KC_ECUDA = 3,      /* a CUDA runtime call failed */
    KC_ETIMEOUT = 4,   /* a bounded device-side wait ran out (no hang, no trap) */
    KC_ENOTCONV = 5,   /* iterative refinement did not reach rtol */
    KC_ERANKDEF = 6,   /* informational: some pivots were dropped */
    KC_EINDEF = 7      /* CG met nonpositive curvature */
} kc_status;

/* Covariance function (Section 4.4); nugget is added on the diagonal only
 * (Section 4.3), and Theta_ii = sigma2 + nugget for every family.
 * KC_MATERN (Eq. (Matern)): sigma2 2^{1-nu}/Gamma(nu) t^nu K_nu(t) with
 *   t = sqrt(2 nu) r / ell, nu in (0, 50].  nu = 0.5, 1.5, 2.5 use the
 *   closed forms (K of half-integer order is elementary); other nu evaluate
 *   K_nu by Temme's series (t <= 2) or Steed's continued fraction (t > 2) and
 *   the upward recurrence, in double (the FP32 form rounds that value).
 * KC_CAUCHY (the Cauchy class of Gneiting, Section 4.4):
 *   sigma2 (1 + (r/ell)^alpha)^{-beta/alpha}, 0 < alpha <= 2, beta > 0
 *   (nu is ignored); the FP32 form evaluates it in float.
 * A struct zero-initialised past nugget is a Matern kernel. */
typedef enum { KC_MATERN = 0, KC_CAUCHY = 1 } kc_family;
typedef struct {
    double nu;
    double ell;
    double sigma2;
    double nugget;
    int32_t family;  /* kc_family */
    double alpha;    /* KC_CAUCHY */
    double beta;     /* KC_CAUCHY */
} kc_kernel;

typedef enum { KC_RULE_MAX = 0, KC_RULE_MIN = 1 } kc_rule;
/* KC_RULE_MAX: (j,i), i before j, is in S iff dist <= rho*l[i] (Section 2.3).
 * KC_RULE_MIN: iff dist <= rho*l[j] (the pattern of Section 6). */

typedef enum { KC_FP64 = 0, KC_FP32_FORM = 1 } kc_prec;
/* KC_FP64: values, entries and sums in double; val is double[nnz].
 * KC_FP32_FORM: val is float[nnz]; dot products in float with compensated
 * (Dot2, Ogita-Rump-Oishi) accumulation, combined in double; the pivot
 * Theta_ii - sum L_ik^2 and its square root in double (diag[] keeps it). */

/* Device view of a pattern and its schedule (all pointers device, caller-owned). */
typedef struct {
    int64_t N;
    int64_t nnz;
    const int64_t* rowptr;   /* [N+1] CSR rows of L */
    const int32_t* col;      /* [nnz] */
    const int64_t* colptr;   /* [N+1] CSC columns of L (from kc_schedule) */
    const int32_t* rowidx;   /* [nnz] rows of each column, ascending, diagonal first */
    const int64_t* slot;     /* [nnz] CSR position of each CSC entry */
    const int32_t* order;    /* [N]   columns sorted by dependency level (kc_schedule): the order
                                the factor and the solves take them in */
    int32_t depth;           /* number of dependency levels */
    const int32_t* level;    /* [N]   dependency level of every column (informational; may be NULL) */
} kc_pattern;

/* Options of the persistent kernels (zero-initialise for defaults). */
typedef struct {
    int64_t spin_limit_cycles;     /* bound of every device wait; 0 -> ~4e9 cycles */
    int32_t rows_per_task;         /* rows of a column per task; 0 -> factor: about (nnz - N) / (depth x
                                      resident warps), a power of two in 16..128; factor by column groups:
                                      see kc_factor_blocked; backward solve: 128 */
    int32_t ctas_per_sm;           /* persistent grid = SMs x this; 0 -> occupancy; < 0 (factor) ->
                                      occupancy + this (at least 1): leaves that many CTA slots per
                                      SM to kernels on other streams (latency of concurrent solves) */
    int32_t warps_per_cta;         /* 0 -> the CTA size (8, 4, 2 or 1 warps) with the most resident warps */
    int32_t test_hold_column;      /* test hook: 0 = off; c+1 makes column c never signal
                                      ready, so a wait on it runs out (KC_ETIMEOUT) */
    int32_t lanes_per_row;         /* factor: lanes merging one row (1,2,4,..,32); 0 -> 8 (FP32 form) or
                                      4 (FP64): one 32-byte sector of values per group load */
    int32_t unroll;                /* factor: (col, val) loads staged ahead per lane, 4, 8 or 16 (16: FP32
                                      form only; FP64 takes 8); 0 -> FP32 form: 16 when the mean row
                                      holds >= 400 entries, else 8; FP64: 4 */
    int32_t adaptive_chunks;       /* factor: nonzero -> a task takes at least |R_i|/4 rows */
    int32_t stage_bytes;           /* factor: <= 0 -> row prefixes loaded into registers (the default);
                                      > 0 -> bulk form: each warp fills two shared-memory stage buffers of
                                      this many bytes (<= 65536) with bulk (TMA) copies of row prefixes */
} kc_opts;

const char* kc_last_error(void);
/* Version of this interface (structs and signatures); a binding built for
 * another version must not call the library.  2: kc_schedule takes the points,
 * kc_opts has stage_bytes.  3: kc_kernel has family, alpha, beta;
 * kc_kernel_eval, kc_l_matvec, kc_lt_matvec, kc_llt_matvec, kc_logdet,
 * kc_pattern_reverse, kc_gather_entries, kc_factor_given, kc_refine_sparse,
 * kc_supernodal_count, kc_supernodal_fill, kc_supernodal, kc_pattern_validate.
 * 4: kc_scratch_trim, kc_frob_error, kc_factor_blocked; scratch from a private pool per device.
 * 5: kc_pattern_begin, kc_pattern_end, kc_pattern_abort; kc_opts.ctas_per_sm < 0. */
#define KC_ABI_VERSION 5
int32_t kc_abi_version(void);

/* Number of kernels this library has launched in the process so far
 * (monotone; take differences around a region of interest). */
int64_t kc_launch_count(void);

/* Device time in ms of the persistent factor kernel of the calling thread's
 * last kc_factor, measured with CUDA events on the launching stream (the
 * task-list build before it is excluded). */
double kc_last_factor_kernel_ms(void);

/* Releases the memory the current device's private scratch pool keeps mapped
 * between calls, down to keep_bytes (0 = all of it).  Memory still in use by
 * work enqueued on some stream is not released.  KC_EINVAL if keep_bytes < 0;
 * KC_OK (nothing to do) before the library's first call on the device. */
kc_status kc_scratch_trim(int64_t keep_bytes);

/* ---- a2: maximin ordering (Section 2.3) -------------------------------- *
 * x: device double[N*d].  Outputs (device): perm int32[N] (position ->
 * original index), l double[N] (l[0] = +inf; first point = original index 0;
 * ties of the squared distance go to the smaller original index), x_ord
 * double[N*d] (x permuted).  d >= 1, N >= 1.  Exact: equals the greedy
 * definition bit for bit.  Synchronises. */
kc_status kc_order_points(const double* x, int64_t N, int32_t d, int32_t* perm, double* l,
                          double* x_ord, void* stream);

/* ---- a3: sparsity pattern S_rho (Section 2.3), two phases --------------- *
 * kc_pattern_count fills rowptr (device int64[N+1]) and returns nnz through
 * nnz_out (host); synchronises.  kc_pattern_fill writes col (device
 * int32[nnz]), ascending per row, diagonal last.  rho > 0. */
kc_status kc_pattern_count(const double* x_ord, const double* l, int64_t N, int32_t d, double rho,
                           int32_t rule, int64_t* rowptr, int64_t* nnz_out, void* stream);
kc_status kc_pattern_fill(const double* x_ord, const double* l, int64_t N, int32_t d, double rho,
                          int32_t rule, const int64_t* rowptr, int32_t* col, void* stream);

/* The same pattern with one search instead of two: kc_pattern_begin runs the
 * search once, fills rowptr (device int64[N+1]) and nnz_out (host) as
 * kc_pattern_count does, and keeps the bucketing grid and one membership bit
 * per candidate in scratch owned by *builder_out (synchronises).  x_ord, l and
 * rowptr must stay valid and unchanged until the builder is released.
 * kc_pattern_end writes col (device int32[nnz], ascending per row, diagonal
 * last: the same array as kc_pattern_fill) from those bits on the stream
 * given to kc_pattern_begin, synchronises, and releases the builder, whatever
 * its status (col NULL: KC_EINVAL, released).  kc_pattern_abort releases a
 * builder without filling (NULL: nothing).  On an error kc_pattern_begin
 * leaves *builder_out NULL.  A builder is used by one thread at a time. */
typedef struct kc_pattern_builder kc_pattern_builder;
kc_status kc_pattern_begin(const double* x_ord, const double* l, int64_t N, int32_t d, double rho,
                           int32_t rule, int64_t* rowptr, int64_t* nnz_out, kc_pattern_builder** builder_out,
                           void* stream);
kc_status kc_pattern_end(kc_pattern_builder* builder, int32_t* col);
void kc_pattern_abort(kc_pattern_builder* builder);

/* ---- a4: schedule ------------------------------------------------------ *
 * From the CSR rows: CSC (colptr int64[N+1], rowidx int32[nnz], slot
 * int64[nnz]), dependency levels level int32[N] with level(i) = 1 + max over
 * k in row i of level(k), and order int32[N] = the columns sorted by level;
 * within a level by index, or, when x_ord (device double[N*d], the points in
 * the pattern's order; may be NULL) is given, by the Morton code of each
 * column's point, so that the factor's and the solves' consecutive work items
 * touch neighbouring points (better L2 reuse).  depth_out (host) = number of
 * levels.  Synchronises. */
kc_status kc_schedule(int64_t N, const int64_t* rowptr, const int32_t* col, const double* x_ord, int32_t d,
                      int64_t* colptr, int32_t* rowidx, int64_t* slot, int32_t* level, int32_t* order,
                      int32_t* depth_out, void* stream);

/* Check a pattern and its schedule (all device arrays of pat): rowptr from 0
 * to nnz with every row nonempty, columns in range and ascending with the
 * diagonal last; colptr likewise, row indices ascending with the diagonal
 * first, each slot pointing at the same entry in the rows; order a
 * permutation.  Every index is range-checked before it is used, so a corrupt
 * pattern is reported (KC_EINVAL, naming the array and index) rather than
 * read out of bounds.  The other entry points trust their pattern; run this
 * on patterns that did not come from this library.  Synchronises. */
kc_status kc_pattern_validate(const kc_pattern* pat, void* stream);

/* ---- a5+a6: ICHOL(0) factor (Algorithm 2, left-looking form) ------------ *
 * For each column i in dependency order: p = Theta_ii - sum_k L_ik^2; if
 * p <= 0 the whole column is zero (Section 4.4); else L_ii = sqrt(p) and
 * L_ji = (Theta_ji - sum_{k in R_j and R_i} L_jk L_ik) / L_ii.  Theta is
 * evaluated from x_ord (device double[N*d]) inside the kernel.
 * val: device double[nnz] (KC_FP64) or float[nnz] (KC_FP32_FORM), CSR layout.
 * diag: device double[N], the FP64 L_ii (0 for a dropped pivot).
 * zero_pivots_out (host, may be NULL): dropped pivots.  One persistent launch.
 * Returns KC_ETIMEOUT if a dependency wait ran out.  Synchronises. */
kc_status kc_factor(const kc_pattern* pat, const double* x_ord, int32_t d, const kc_kernel* kern,
                    int32_t prec, void* val, double* diag, int64_t* zero_pivots_out,
                    const kc_opts* opts, void* stream);

/* ---- the same factor by column groups (the supernodal block factorisation)  *
 * Same arguments and result as kc_factor (up to the order of the sums), for
 * entries from the covariance function.  Runs of consecutive columns whose
 * rows share one list of earlier columns and whose columns share one set of
 * later rows -- the supernodes of the supernodal multicolour ordering of the
 * stability section -- are factored as blocks of at most 8 columns: the
 * group's diagonal block by a small dense Cholesky with the zero-column rule,
 * and every row below it with one pass over the row's prefix for all the
 * group's columns, then a forward substitution (the block algorithm of the
 * stability appendix, equal to Algorithm 2 on such a pattern).  On a pattern
 * without such runs (the maximin pattern) every group is one column.  opts:
 * spin_limit_cycles, rows_per_task (rows of one task; 0 -> (nnz - N) / (depth x
 * resident CTAs) as the nearest power of two in 64..512), lanes_per_row (>= 8).
 * One persistent launch.  Synchronises. */
kc_status kc_factor_blocked(const kc_pattern* pat, const double* x_ord, int32_t d, const kc_kernel* kern,
                            int32_t prec, void* val, double* diag, int64_t* zero_pivots_out, const kc_opts* opts,
                            void* stream);

/* ---- factor plans: many point sets in one launch, capturable ------------ *
 * A plan keeps the task list and counters of one pattern, so that each
 * factorisation is a single persistent launch with no allocation and no host
 * synchronisation (it can be recorded in a CUDA graph).  Independent point
 * sets are factored together by concatenating their patterns
 * block-diagonally (positions of set s shifted by its offset, coordinates
 * padded to a common d with zeros): col_set (device int32[N]) gives the set of
 * every column and kerns[set] (host, nsets entries) its covariance function;
 * with nsets == 1, col_set may be NULL.  x_ord must stay valid while the plan
 * is used.  kc_factor_plan_finish synchronises and reports a timeout or the
 * dropped pivots of the last launch.  kc_factor_plan_tune times every
 * combination of lanes per row {2,4,8,16} and staging depth {8,16} once on the
 * plan's own problem and keeps the fastest (it overwrites val and diag). */
typedef struct kc_factor_plan kc_factor_plan;
kc_status kc_factor_plan_create(const kc_pattern* pat, const double* x_ord, int32_t d, const kc_kernel* kerns,
                                int32_t nsets, const int32_t* col_set, int32_t prec, const kc_opts* opts,
                                kc_factor_plan** out, void* stream);
kc_status kc_factor_plan_launch(kc_factor_plan* plan, void* val, double* diag, void* stream);
kc_status kc_factor_plan_finish(kc_factor_plan* plan, int64_t* zero_pivots_out, void* stream);
kc_status kc_factor_plan_tune(kc_factor_plan* plan, void* val, double* diag, int32_t* lanes_out,
                              int32_t* unroll_out, double* best_ms_out, void* stream);
void kc_factor_plan_destroy(kc_factor_plan* plan);

/* Concatenate nsets patterns block-diagonally (host arrays of device
 * pointers): rowptr_out int64[sum N + 1], col_out int32[sum nnz], and
 * set_out int32[sum N] (set of every position).  Synchronises. */
kc_status kc_pattern_concat(int32_t nsets, const int64_t* const* rowptrs, const int32_t* const* cols,
                            const int64_t* Ns, int64_t* rowptr_out, int32_t* col_out, int32_t* set_out, void* stream);

/* Concatenate point arrays (host array of device pointers, set s has Ns[s]
 * points of dimension ds[s]) into out double[sum N * dout], padding missing
 * coordinates with 0 (dout >= every ds). */
kc_status kc_points_concat(int32_t nsets, const double* const* xs, const int64_t* Ns, const int32_t* ds,
                           int32_t dout, double* out, void* stream);

/* Concatenate index arrays (host array of device pointers) shifting set s by
 * its offset sum_{t<s} Ns[t]: for permutations of the concatenated sets. */
kc_status kc_index_concat(int32_t nsets, const int32_t* const* idx, const int64_t* Ns, int32_t* out, void* stream);

/* ---- a7: solve L L^T x = b (task (2) with the factor) ------------------- *
 * b, x: device double[nrhs*N], column-major (rhs r at offset r*N), original
 * point order.  perm: device int32[N].  A dropped pivot uses
 * sqrt(Theta_ii) = sqrt(sigma2 + nugget) on the diagonal (kern gives it).
 * 1 <= nrhs <= 16.  Level-scheduled sparse triangular solves, FP64 sums. */
kc_status kc_solve(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                   const kc_kernel* kern, const int32_t* perm, const double* b, int32_t nrhs,
                   double* x, const kc_opts* opts, void* stream);

/* ---- kc_solve without device allocation ---------------------------------- *
 * The paper has no counterpart: this is an operational variant of kc_solve.
 * It is for callers that cannot allocate device memory while they run -- a
 * server whose device memory is handed out up front to another framework's
 * pool, a plugin that its host application forbids to allocate, a
 * latency-critical loop where an allocation could block on driver locks or
 * synchronise the device.  Same arguments and result as kc_solve (no opts);
 * the scratch comes from one fixed file-scope device array of 28 MiB + 256 B
 * that every GPU loading this library keeps until the process exits, so it
 * needs N <= 2^20 and N*nrhs <= 2^20 (larger sizes return KC_EINVAL).  The
 * caller passes every input and output.  All calls on a device share the one
 * array: calls that overlap on the GPU race and corrupt each other, so
 * serialise them.  The first call on a device, with that device current,
 * looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  The address is kept per device together
 * with the unique id of the CUDA context it belongs to: after a
 * cudaDeviceReset (a new context) the next call looks it up again, so that
 * call too should come before any stream capture.  Synchronises. */
kc_status kc_solve_noalloc(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                           const kc_kernel* kern, const int32_t* perm, const double* b, int32_t nrhs, double* x,
                           void* stream);

/* ---- a8: refinement: CG on the dense Theta preconditioned by L L^T ------ *
 * (task (2); CG with the factor as preconditioner, Section 4.3).  The
 * matrix-vector product with Theta is evaluated from the coordinates in
 * FP64, O(N^2) per iteration.  Starts from x = 0; stops when every rhs has
 * ||b - Theta x||_2 <= rtol ||b||_2 or after maxit iterations.
 * iters_out (host int32[1]), relres_out (host double[nrhs]): recursive
 * relative residuals.  Returns KC_ENOTCONV or KC_EINDEF on failure. */
kc_status kc_refine(const kc_pattern* pat, const double* x_ord, int32_t d, const kc_kernel* kern,
                    int32_t prec, const void* val, const double* diag, const int32_t* perm,
                    const double* b, int32_t nrhs, double rtol, int32_t maxit, double* x,
                    int32_t* iters_out, double* relres_out, const kc_opts* opts, void* stream);

/* ---- a9: rank-k PCA (Section 2.5) --------------------------------------- *
 * Lk: device float[k*N] column-major (column a at offset a*N), the first k
 * columns of L with rows scattered back to original order. */
kc_status kc_pca_truncate(const kc_pattern* pat, int32_t prec, const void* val, const int32_t* perm,
                          int32_t k, float* Lk, void* stream);

/* Power iteration estimate of ||Theta - Lk Lk^T||_2 on original-order points
 * x (device double[N*d]): iters steps from the unit vector v0 (device
 * double[N]); estimate_out (host) = |v^T B v|.  Theta v is evaluated on the
 * fly (FP32 entries, FP64 sums). */
kc_status kc_pca_error(const double* x, int64_t N, int32_t d, const kc_kernel* kern, int32_t k,
                       const float* Lk, const double* v0, int32_t iters, double* estimate_out,
                       void* stream);

/* ---- the covariance function alone ------------------------------------- *
 * out[i] = G(r[i]) for n distances (device double[n] each, n >= 0), without
 * the nugget, evaluated exactly as the factor evaluates its entries:
 * KC_FP64 in double; KC_FP32_FORM with r rounded to float first and the
 * result widened.  Stream-ordered (no synchronisation). */
kc_status kc_kernel_eval(const kc_kernel* kern, int32_t prec, const double* r, int64_t n, double* out,
                         void* stream);

/* ---- tasks (1), (3) and (4) of Section 1 with the factor ---------------- *
 * L is a factor from kc_factor: val in prec (CSR layout of pat), diag its
 * FP64 diagonal (0 for a dropped column, which stays zero).  perm (device
 * int32[N]) is the ordering: position k holds original point perm[k].
 * Vectors are device double[nrhs*N], column-major (vector r at offset r*N),
 * in original point order; 1 <= nrhs <= 16; outputs must not alias inputs.
 *   kc_l_matvec:   y = P L P^T z   (task (4): for z ~ N(0, I), y is a sample
 *                                   of N(0, P L L^T P^T), L L^T ~ Theta)
 *   kc_lt_matvec:  y = P L^T P^T v
 *   kc_llt_matvec: y = P L L^T P^T v   (task (1): approximates Theta v)
 * Products and sums in FP64.  L z gathers along the rows of L, L^T v along
 * its columns (the CSC of pat): no atomics, every sum in a fixed order, so
 * the result is the same bits on every run.  Stream-ordered. */
kc_status kc_l_matvec(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                      const int32_t* perm, const double* z, int32_t nrhs, double* y, void* stream);
kc_status kc_lt_matvec(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                       const int32_t* perm, const double* v, int32_t nrhs, double* y, void* stream);
kc_status kc_llt_matvec(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                        const int32_t* perm, const double* v, int32_t nrhs, double* y, void* stream);

/* Task (3): logdet_out (host) = log det(L L^T) = 2 sum_i log diag[i] over
 * the kept pivots (diag: device double[N]); zero_pivots_out (host, may be
 * NULL) = the dropped ones (then L L^T is singular and the sum covers the
 * rest).  A fixed reduction order: the same bits on every run.
 * Synchronises. */
kc_status kc_logdet(const kc_pattern* pat, const double* diag, double* logdet_out, int64_t* zero_pivots_out,
                    void* stream);

/* ---- the sampled error estimator of Section 4.4 -------------------------- *
 * E^2 = num2 / den2 with num2 = sum_t ((L L^T)_{pi[t],pj[t]} - Theta_{pi[t],pj[t]})^2
 * and den2 = sum_t Theta_{pi[t],pj[t]}^2 over the m pairs (device int64[m]
 * each, original point numbering, 0..N-1: the caller draws them i.i.d.
 * uniformly from I x I with replacement), or over the pairs with keep[t] != 0
 * (device int8[m], may be NULL: every pair).  L is a factor from kc_factor
 * (val in prec, CSR layout of pat, diag its FP64 pivots), perm the ordering
 * and x_ord (device double[N*d]) the points in positions; kern the
 * covariance function, evaluated in FP64 as the FP64 factor does, nugget on
 * the diagonal.  (L L^T)_ij is a sparse row merge in FP64.  The sums run in a
 * fixed order (same bits on every run).  Outputs (host): num2, den2 and the
 * number of pairs kept (may be NULL).  A pair index outside 0..N-1 gives
 * KC_EINVAL (detected on the device, never used as an index).
 * Synchronises. */
kc_status kc_frob_error(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                        const double* x_ord, int32_t d, const kc_kernel* kern, const int32_t* perm, const int64_t* pi,
                        const int64_t* pj, int64_t m, const int8_t* keep, double* num2_out, double* den2_out,
                        int64_t* kept_out, void* stream);

/* ---- Section 6: factors of a given sparse matrix, reverse order ---------- *
 * The precision matrix A = Theta^{-1} (a discretised elliptic operator) has
 * near-sparse Cholesky factors in the reverse maximin order on the pattern
 * of the min rule, dist(i, j) <= rho min(l[i], l[j]) (kc_pattern_count with
 * KC_RULE_MIN); so has sigma^2 A + I, which gives Theta + sigma^2 I =
 * Theta (sigma^2 A + I) for a nugget sigma^2.
 *
 * kc_pattern_reverse: from the CSC (colptr int64[N+1], rowidx int32[nnz],
 * device; kc_schedule's output) of a maximin-order lower-triangular pattern,
 * the CSR rows (rowptr_out int64[N+1], col_out int32[nnz], device) of the
 * same symmetric pattern in the reversed order, where position q is maximin
 * position N-1-q: columns ascending, diagonal last.  Stream-ordered.
 *
 * kc_gather_entries: aval_out[e] (device double[nnz]) = A(orig[j], orig[i])
 * for every entry e = (j, i) of the pattern (rowptr, col, device), where
 * orig (device int32[N]) maps a position to the original index and A is
 * N x N, given by CSR rows in original numbering (a_rowptr int64[N+1],
 * a_col int32, a_val double, device; columns ascending within each row,
 * both triangles stored); 0 where A has no entry.  outside_out (host, may be
 * NULL; synchronises when given) = the number of A's off-diagonal entries
 * (u, v) whose positions are not in the pattern: ICHOL(0) drops them
 * (Algorithm 2), so a nonzero count means the pattern is too small for A.
 *
 * kc_factor_given: ICHOL(0) (Algorithm 2, left-looking form, as kc_factor)
 * of the symmetric matrix whose lower triangle on pat is aval (device
 * double[nnz], CSR layout of pat).  val, diag, zero_pivots_out, opts and the
 * errors as for kc_factor; the FP32 form rounds the entries to float.  A
 * dropped pivot leaves diag 0: kc_solve then divides by
 * sqrt(kern->sigma2 + kern->nugget), so pass a kernel whose sigma2 is of the
 * size of A's diagonal.  Synchronises. */
kc_status kc_pattern_reverse(int64_t N, const int64_t* colptr, const int32_t* rowidx, int64_t* rowptr_out,
                             int32_t* col_out, void* stream);
kc_status kc_gather_entries(int64_t N, const int64_t* rowptr, const int32_t* col, const int32_t* orig,
                            const int64_t* a_rowptr, const int32_t* a_col, const double* a_val, double* aval_out,
                            int64_t* outside_out, void* stream);
kc_status kc_factor_given(const kc_pattern* pat, const double* aval, int32_t prec, void* val, double* diag,
                          int64_t* zero_pivots_out, const kc_opts* opts, void* stream);

/* CG on A x = b for the given sparse symmetric positive-definite A (CSR in
 * original numbering as for kc_gather_entries), preconditioned by L L^T, the
 * factor of kc_factor_given on pat (val in prec, diag; perm: position ->
 * original index).  A is applied in positions by a sparse product (one warp
 * per row, FP64, a fixed summation order).  b, x, nrhs, rtol, maxit,
 * iters_out, relres_out and the errors as for kc_refine; a dropped pivot
 * divides by 1.  Synchronises. */
kc_status kc_refine_sparse(const kc_pattern* pat, int32_t prec, const void* val, const double* diag,
                           const int32_t* perm, const int64_t* a_rowptr, const int32_t* a_col, const double* a_val,
                           const double* b, int32_t nrhs, double rtol, int32_t maxit, double* x, int32_t* iters_out,
                           double* relres_out, const kc_opts* opts, void* stream);

/* ---- supernodal multicolour ordering and pattern ------------------------ *
 * The Construction of the paper's stability section, from the maximin order
 * (x_ord, l of kc_order_points) and its max-rule pattern S_rho of the same
 * rho >= 1 (pat, scheduled; every pair the construction tests lies in it).
 * Hierarchy: h = 1/2 and the largest finite length scale l[1] as the unit,
 * so maximin position m is on level k(m) = the smallest k >= 1 with
 * l[m] >= l[1] 2^-k (position 0 on level 1); d(a, b) = dist(a, b) /
 * (l[1] 2^-min(k(a), k(b))).  Supernodes of a level are taken greedily in
 * maximin order (unless an earlier supernode of the level is within d <=
 * rho); each point joins the nearest supernode of its level (ties to the
 * smaller index); supernodes A, B pair when members a, b have d(a, b) <=
 * rho; colours are greedy per level in maximin order; the new order sorts
 * by level, colour, supernode, maximin position; the pattern S holds (q, p),
 * p <= q, whenever the supernodes of q and p pair.  Algorithm 2 on this
 * order and pattern is the supernodal block factorisation.
 * kc_supernodal_count: newm int32[N] (maximin position of every new
 * position), level, node (maximin position of the supernode), colour
 * (int32[N] each, may be NULL), x_new double[N*d] (the points in the new
 * order), rowptr int64[N+1] of S, nnz_out (host).  kc_supernodal_fill: col
 * int32[nnz] (ascending, diagonal last), from the same inputs and rowptr.
 * kc_supernodal does both in one pass when col (device int32[col_capacity])
 * holds nnz entries; otherwise it leaves col alone and the caller, seeing
 * *nnz_out > col_capacity, completes with kc_supernodal_fill.  All
 * synchronise; KC_EINVAL if a level needs more than 64 colours. */
kc_status kc_supernodal_count(const double* x_ord, const double* l, int32_t d, double rho, const kc_pattern* pat,
                              int32_t* newm, int32_t* level, int32_t* node, int32_t* color, double* x_new,
                              int64_t* rowptr, int64_t* nnz_out, void* stream);
kc_status kc_supernodal_fill(const double* x_ord, const double* l, int32_t d, double rho, const kc_pattern* pat,
                             const int64_t* rowptr, int32_t* col, void* stream);
kc_status kc_supernodal(const double* x_ord, const double* l, int32_t d, double rho, const kc_pattern* pat,
                        int32_t* newm, int32_t* level, int32_t* node, int32_t* color, double* x_new, int64_t* rowptr,
                        int32_t* col, int64_t col_capacity, int64_t* nnz_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KCHOL_H */
