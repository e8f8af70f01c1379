/*
 * CPU FP64 oracle for the sparse Cholesky factorisation of dense kernel
 * matrices (Schaefer, Sullivan, Owhadi, "Compression, inversion, and
 * approximate PCA of dense kernel matrices at near-linear computational
 * complexity").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * bench's CPU-baseline leg may load this library; the product path never does.
 *
 * Plain, slow, single-threaded C in IEEE double precision.  It must be
 * compiled with -O2 -ffp-contract=off so that no multiply-add is fused: the
 * squared distance of two points is then the same bit pattern on every
 * machine, which the exact (bit-identical) comparisons of orderings and
 * patterns rely on.
 *
 * Conventions (readings of the paper where it is silent):
 *  - Points are row-major x[i*d + t], i in original order.
 *  - d2(a,b) = sum_{t=0}^{d-1} (x_a,t - x_b,t)^2, each operation rounded
 *    separately, summed in t order; dist = sqrt(d2) (correctly rounded).
 *  - Maximin ordering (Section 2.3): the first point is original index 0
 *    (the whole-space case lets it be arbitrary); each next point maximises the
 *    squared distance to the points already chosen; ties go to the smallest
 *    original index.  l[k] = sqrt(that squared distance), l[0] = +inf.
 *  - Positions in the ordering are the indices of the factor: "i" below is the
 *    i-th point of the maximin order.
 *  - Pattern S_rho (Section 2.3): for positions i < j, (j,i) is in S iff
 *    dist(i,j) <= rho * l[i] (the max rule, since l is non-increasing); the
 *    min rule (used in Section 6 for the reverse-order factor of the inverse)
 *    takes rho * l[j] instead.  The diagonal is always in S.
 *  - The factor L is stored as CSR by rows in ordered positions, column
 *    indices ascending, the diagonal last in each row.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;
typedef int32_t i32;

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

static double d2_of(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        double u = a[t] - b[t];
        double v = u * u;
        s = s + v;
    }
    return s;
}

double ko_d2(const double* a, const double* b, i32 d) { return d2_of(a, b, d); }

/* ------------------------------------------------------------------------ */
/* Maximin ordering by its definition, O(N^2) (Section 2.3, Eq. for i_{k+1})  */
/* ------------------------------------------------------------------------ */

/* perm[k] = original index of the k-th point; l[k] its length scale. */
void ko_maximin_brute(const double* x, i64 N, i32 d, i32* perm, double* l) {
    if (N <= 0) return;
    double* cur = (double*)malloc(sizeof(double) * (size_t)N);
    char* taken = (char*)calloc((size_t)N, 1);
    perm[0] = 0;
    l[0] = INFINITY;
    taken[0] = 1;
    for (i64 i = 0; i < N; ++i) cur[i] = d2_of(x + i * d, x, d);
    for (i64 k = 1; k < N; ++k) {
        i64 best = -1;
        for (i64 i = 0; i < N; ++i) {
            if (taken[i]) continue;
            if (best < 0 || cur[i] > cur[best]) best = i; /* strict: ties keep the smaller index */
        }
        perm[k] = (i32)best;
        l[k] = sqrt(cur[best]);
        taken[best] = 1;
        const double* xb = x + best * d;
        for (i64 i = 0; i < N; ++i) {
            if (taken[i]) continue;
            double v = d2_of(x + i * d, xb, d);
            if (v < cur[i]) cur[i] = v;
        }
    }
    free(cur);
    free(taken);
}

/* ------------------------------------------------------------------------ */
/* Ordering and pattern by the paper's heap algorithm (Algorithm 3,          */
/* "Ordering and sparsity pattern algorithm", Section 4.1).                  */
/* Readings: the symmetric entry pushed in the final aggregation is (j,i);    */
/* c[i] is sorted once after the loop that fills it.  The two pruning tests   */
/* get a relative slack of 1e-12 so that rounding in the triangle inequality  */
/* can only widen the candidate set, never drop a point.                     */
/* ------------------------------------------------------------------------ */

typedef struct { i32 j; double dist; } child_t;
typedef struct { child_t* a; i64 n, cap; } childvec;
typedef struct { i32* a; i64 n, cap; } intvec;

static void cv_push(childvec* v, i32 j, double dist) {
    if (v->n == v->cap) { v->cap = v->cap ? 2 * v->cap : 8; v->a = (child_t*)realloc(v->a, sizeof(child_t) * (size_t)v->cap); }
    v->a[v->n].j = j; v->a[v->n].dist = dist; v->n++;
}
static void iv_push(intvec* v, i32 j) {
    if (v->n == v->cap) { v->cap = v->cap ? 2 * v->cap : 8; v->a = (i32*)realloc(v->a, sizeof(i32) * (size_t)v->cap); }
    v->a[v->n++] = j;
}
static int child_cmp(const void* pa, const void* pb) {
    const child_t* a = (const child_t*)pa; const child_t* b = (const child_t*)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->j < b->j) ? -1 : (a->j > b->j);
}

/* mutable max-heap of original indices keyed by (key desc, index asc) */
typedef struct { i32* h; i64* where; double* key; i64 n; } heap_t;
static int h_above(const heap_t* H, i32 a, i32 b) {
    return H->key[a] > H->key[b] || (H->key[a] == H->key[b] && a < b);
}
static void h_swap(heap_t* H, i64 p, i64 q) {
    i32 a = H->h[p], b = H->h[q];
    H->h[p] = b; H->h[q] = a; H->where[b] = p; H->where[a] = q;
}
static void h_down(heap_t* H, i64 p) {
    for (;;) {
        i64 c1 = 2 * p + 1, c2 = c1 + 1, m = p;
        if (c1 < H->n && h_above(H, H->h[c1], H->h[m])) m = c1;
        if (c2 < H->n && h_above(H, H->h[c2], H->h[m])) m = c2;
        if (m == p) return;
        h_swap(H, p, m); p = m;
    }
}
static i32 h_pop(heap_t* H) {
    i32 top = H->h[0];
    h_swap(H, 0, H->n - 1);
    H->n--;
    H->where[top] = -1;
    if (H->n > 0) h_down(H, 0);
    return top;
}
/* lower the key of j to v if j is still in the heap and v is smaller */
static void h_decrease(heap_t* H, i32 j, double v) {
    i64 p = H->where[j];
    if (p < 0 || !(v < H->key[j])) return;
    H->key[j] = v;
    h_down(H, p);
}

typedef struct {
    i64 N;
    i32* perm;        /* ordered -> original */
    double* l;
    i64 nnz;          /* entries of L incl. diagonal */
    i64* rowptr;      /* CSR of L in ordered positions */
    i32* col;
} ko_sortsparse_result;

/* Returns a heap-allocated result; free with ko_sortsparse_free. */
ko_sortsparse_result* ko_sortsparse(const double* x, i64 N, i32 d, double rho, i32 rule_min) {
    ko_sortsparse_result* R = (ko_sortsparse_result*)calloc(1, sizeof(ko_sortsparse_result));
    R->N = N;
    if (N <= 0) { R->rowptr = (i64*)calloc(1, sizeof(i64)); return R; }
    R->perm = (i32*)malloc(sizeof(i32) * (size_t)N);
    R->l = (double*)malloc(sizeof(double) * (size_t)N);
    double* lo = (double*)malloc(sizeof(double) * (size_t)N); /* l by original index */
    i64* pos = (i64*)malloc(sizeof(i64) * (size_t)N);          /* original -> ordered */
    childvec* c = (childvec*)calloc((size_t)N, sizeof(childvec));
    intvec* p = (intvec*)calloc((size_t)N, sizeof(intvec));
    heap_t H;
    H.h = (i32*)malloc(sizeof(i32) * (size_t)N);
    H.where = (i64*)malloc(sizeof(i64) * (size_t)N);
    H.key = (double*)malloc(sizeof(double) * (size_t)N);
    H.n = N;
    for (i64 i = 0; i < N; ++i) { H.h[i] = (i32)i; H.where[i] = i; H.key[i] = INFINITY; lo[i] = INFINITY; }
    /* all keys equal: index order already satisfies the heap property */

    const double slack_lo = 1.0 - 1e-12, slack_hi = 1.0 + 1e-12;
    i64 k_ord = 0;
    /* first index: every point is its child */
    {
        i32 i = h_pop(&H);
        lo[i] = INFINITY;
        for (i64 j = 0; j < N; ++j) {
            double dd2 = d2_of(x + (i64)i * d, x + j * d, d);
            cv_push(&c[i], (i32)j, sqrt(dd2));
            iv_push(&p[j], i);
            h_decrease(&H, (i32)j, dd2);
        }
        qsort(c[i].a, (size_t)c[i].n, sizeof(child_t), child_cmp);
        R->perm[k_ord] = i; R->l[k_ord] = INFINITY; pos[i] = k_ord; k_ord++;
    }
    while (H.n > 0) {
        double key = H.key[H.h[0]];
        i32 i = h_pop(&H);
        double li = sqrt(key);
        lo[i] = li;
        double rli = rho * li;
        /* parent k: the closest earlier point whose children cover B(x_i, rho l[i]) */
        i32 k = -1; double dk = INFINITY;
        for (i64 t = 0; t < p[i].n; ++t) {
            i32 j = p[i].a[t];
            double dij = sqrt(d2_of(x + (i64)i * d, x + (i64)j * d, d));
            double rlj = rho * lo[j];
            if ((dij + rli) <= rlj * slack_lo || isinf(rlj)) {
                if (dij < dk || (dij == dk && j < k)) { dk = dij; k = j; }
            }
        }
        double dik = dk;
        double reach = (dik + rli) * slack_hi;
        for (i64 t = 0; t < c[k].n; ++t) {
            if (c[k].a[t].dist > reach) break; /* c[k] is sorted by distance to k */
            i32 j = c[k].a[t].j;
            double dd2 = d2_of(x + (i64)i * d, x + (i64)j * d, d);
            h_decrease(&H, j, dd2);
            double dij = sqrt(dd2);
            if (dij <= rli) { cv_push(&c[i], j, dij); iv_push(&p[j], i); }
        }
        qsort(c[i].a, (size_t)c[i].n, sizeof(child_t), child_cmp);
        R->perm[k_ord] = i; R->l[k_ord] = li; pos[i] = k_ord; k_ord++;
    }

    /* aggregate: column pos[i] of L holds the later children j of i */
    i64* cnt = (i64*)calloc((size_t)N + 1, sizeof(i64));
    if (!rule_min) {
        for (i64 i = 0; i < N; ++i)
            for (i64 t = 0; t < c[i].n; ++t) {
                i32 j = c[i].a[t].j;
                if (pos[j] >= pos[i]) cnt[pos[j] + 1]++;   /* includes the diagonal j == i */
            }
    } else {
        /* min rule: (j,i), i before j, iff dist <= rho * l[j]; children lists
           of i hold dist <= rho l[i] >= rho l[j], so they are a superset */
        for (i64 i = 0; i < N; ++i)
            for (i64 t = 0; t < c[i].n; ++t) {
                i32 j = c[i].a[t].j;
                if (pos[j] > pos[i] && c[i].a[t].dist <= rho * lo[j]) cnt[pos[j] + 1]++;
                else if (j == i) cnt[pos[j] + 1]++;
            }
    }
    R->rowptr = (i64*)malloc(sizeof(i64) * ((size_t)N + 1));
    R->rowptr[0] = 0;
    for (i64 r = 0; r < N; ++r) R->rowptr[r + 1] = R->rowptr[r] + cnt[r + 1];
    R->nnz = R->rowptr[N];
    R->col = (i32*)malloc(sizeof(i32) * (size_t)(R->nnz > 0 ? R->nnz : 1));
    i64* fill = (i64*)malloc(sizeof(i64) * (size_t)N);
    for (i64 r = 0; r < N; ++r) fill[r] = R->rowptr[r];
    /* visit columns in ordered position so that each row's entries come ascending */
    for (i64 q = 0; q < N; ++q) {
        i32 i = R->perm[q];
        for (i64 t = 0; t < c[i].n; ++t) {
            i32 j = c[i].a[t].j;
            int keep;
            if (!rule_min) keep = pos[j] >= pos[i];
            else keep = (j == i) || (pos[j] > pos[i] && c[i].a[t].dist <= rho * lo[j]);
            if (keep) R->col[fill[pos[j]]++] = (i32)q;
        }
    }
    free(fill); free(cnt);
    for (i64 i = 0; i < N; ++i) { free(c[i].a); free(p[i].a); }
    free(c); free(p); free(H.h); free(H.where); free(H.key); free(lo); free(pos);
    return R;
}

void ko_sortsparse_free(ko_sortsparse_result* R) {
    if (!R) return;
    free(R->perm); free(R->l); free(R->rowptr); free(R->col); free(R);
}

/* ------------------------------------------------------------------------ */
/* Pattern S_rho by its definition, O(N^2) (Section 2.3)                     */
/* xo: coordinates in ordered positions.  Two passes: count, then fill.      */
/* ------------------------------------------------------------------------ */

static int in_pattern(const double* xo, const double* l, i64 i, i64 j, i32 d, double rho, i32 rule_min) {
    /* i < j */
    double dist = sqrt(d2_of(xo + i * d, xo + j * d, d));
    double r = rule_min ? l[j] : l[i];
    if (isinf(r)) return 1;
    return dist <= rho * r;
}

void ko_pattern_count(const double* xo, const double* l, i64 N, i32 d, double rho, i32 rule_min, i64* rowptr) {
    rowptr[0] = 0;
    for (i64 j = 0; j < N; ++j) {
        i64 c = 1;
        for (i64 i = 0; i < j; ++i) c += in_pattern(xo, l, i, j, d, rho, rule_min);
        rowptr[j + 1] = rowptr[j] + c;
    }
}

void ko_pattern_fill(const double* xo, const double* l, i64 N, i32 d, double rho, i32 rule_min,
                     const i64* rowptr, i32* col) {
    for (i64 j = 0; j < N; ++j) {
        i64 w = rowptr[j];
        for (i64 i = 0; i < j; ++i)
            if (in_pattern(xo, l, i, j, d, rho, rule_min)) col[w++] = (i32)i;
        col[w++] = (i32)j;
    }
}

/* ------------------------------------------------------------------------ */
/* Covariance functions of Section 4.4.                                      */
/*                                                                          */
/* Matern, Eq. (Matern):                                                    */
/*   G(r) = sigma2 2^{1-nu} / Gamma(nu) t^nu K_nu(t),  t = sqrt(2 nu) r / ell */
/* with closed forms for nu = 1/2, 3/2, 5/2 (K of half-integer order is     */
/* elementary):  1/2: sigma2 e^{-t};  3/2: sigma2 (1+t) e^{-t};             */
/*   5/2: sigma2 (1 + t + t^2/3) e^{-t}.                                    */
/* Other nu > 0 use K_nu from its integral representation                   */
/*   K_nu(x) = int_0^inf exp(-x cosh s) cosh(nu s) ds     (x > 0)           */
/* (Abramowitz & Stegun 9.6.24), by the trapezoidal rule: the integrand is  */
/* entire and decays double-exponentially, so a fixed small step converges  */
/* to working precision.  G takes e^x K_nu(x) (the factor inside the        */
/* integral) and e^{-t} with its other factors, so it stays accurate where  */
/* K_nu alone would underflow.  G(0) = sigma2.                              */
/*                                                                          */
/* Cauchy class (Gneiting), Section 4.4:                                    */
/*   G(r) = sigma2 (1 + (r/ell)^alpha)^{-beta/alpha}.                        */
/*                                                                          */
/* The nugget is added on the diagonal only.                                */
/* ------------------------------------------------------------------------ */

/* e^x K_nu(x): the same integral with the factor e^x taken inside,
   exp(-x (cosh s - 1)) = exp(-2 x sinh^2(s/2)), so that no term underflows
   where K_nu itself leaves the double range.  ko_bessel_k is this times
   e^{-x}. */
double ko_bessel_k_scaled(double nu, double x) {
    if (!(x > 0.0)) return INFINITY;
    /* the trapezoidal error falls like exp(-pi^2/(2h)) but the integrand's
       size off the real axis grows with x: the step shrinks like 1/x */
    const double h = x > 512.0 ? 8.0 / x : 1.0 / 64.0;
    double sum = 0.5; /* s = 0 */
    double prev = sum;
    for (i64 k = 1;; ++k) {
        double s = h * (double)k;
        double u = sinh(0.5 * s);
        double f = exp(-2.0 * x * u * u) * cosh(nu * s);
        sum += f;
        if (f < prev && f <= 1e-18 * sum) break;
        if (!(f > 0.0) && k > 1) break;
        prev = f;
    }
    return h * sum;
}

double ko_bessel_k(double nu, double x) { return exp(-x) * ko_bessel_k_scaled(nu, x); }

double ko_matern(double r, double nu, double ell, double sigma2) {
    if (nu == 0.5) {
        double t = r / ell;
        return sigma2 * exp(-t);
    } else if (nu == 1.5) {
        double t = sqrt(3.0) * r / ell;
        return sigma2 * (1.0 + t) * exp(-t);
    } else if (nu == 2.5) {
        double t = sqrt(5.0) * r / ell;
        return sigma2 * (1.0 + t + t * t / 3.0) * exp(-t);
    }
    if (!(nu > 0.0)) return NAN;
    double t = sqrt(2.0 * nu) * r / ell;
    if (t == 0.0) return sigma2;
    double k = ko_bessel_k_scaled(nu, t);
    return sigma2 * exp((1.0 - nu) * log(2.0) - lgamma(nu) + nu * log(t) - t) * k;
}

double ko_cauchy(double r, double ell, double alpha, double beta, double sigma2) {
    return sigma2 * pow(1.0 + pow(r / ell, alpha), -beta / alpha);
}

/* family 0: Matern (nu, ell, sigma2); 1: Cauchy (ell, alpha, beta, sigma2) */
typedef struct { i32 family; double nu, ell, sigma2, nugget, alpha, beta; } ko_kernel;

double ko_cov(double r, const ko_kernel* K) {
    if (K->family == 1) return ko_cauchy(r, K->ell, K->alpha, K->beta, K->sigma2);
    return ko_matern(r, K->nu, K->ell, K->sigma2);
}

static double theta_pos(const double* xo, i32 d, i64 a, i64 b, const ko_kernel* K) {
    double r = sqrt(d2_of(xo + a * d, xo + b * d, d));
    double v = ko_cov(r, K);
    if (a == b) v += K->nugget;
    return v;
}

double ko_theta(const double* xo, i32 d, i64 a, i64 b, const ko_kernel* K) {
    return theta_pos(xo, d, a, b, K);
}

/* ------------------------------------------------------------------------ */
/* CSC (columns of L) from the CSR rows: colptr, rowidx ascending, and the   */
/* CSR slot of every CSC entry.                                              */
/* ------------------------------------------------------------------------ */

void ko_csr_to_csc(i64 N, const i64* rowptr, const i32* col, i64* colptr, i32* rowidx, i64* slot) {
    i64 nnz = rowptr[N];
    for (i64 i = 0; i <= N; ++i) colptr[i] = 0;
    for (i64 e = 0; e < nnz; ++e) colptr[col[e] + 1]++;
    for (i64 i = 0; i < N; ++i) colptr[i + 1] += colptr[i];
    i64* fill = (i64*)malloc(sizeof(i64) * (size_t)(N > 0 ? N : 1));
    for (i64 i = 0; i < N; ++i) fill[i] = colptr[i];
    for (i64 j = 0; j < N; ++j)
        for (i64 e = rowptr[j]; e < rowptr[j + 1]; ++e) {
            i64 w = fill[col[e]]++;
            rowidx[w] = (i32)j;
            slot[w] = e;
        }
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* ICHOL(0), Algorithm 2 ("Incomplete Cholesky factorization with sparsity   */
/* pattern S"), written in its left-looking form:                            */
/*   for i ascending:  p = Theta_ii - sum_{k in R_i} L_ik^2                  */
/*     if p <= 0 the whole column i is set to zero (Section 4.4: a           */
/*     nonpositive pivot zeroes that column of L);                           */
/*     else L_ii = sqrt(p) and for j in C_i:                                 */
/*       L_ji = (Theta_ji - sum_{k in R_j cap R_i} L_jk L_ik) / L_ii          */
/* where R_i = {k < i : (i,k) in S} and C_i = {j > i : (j,i) in S}.  In       */
/* exact arithmetic this is the same as the algorithm's right-looking update  */
/* A_kj -= A_ki A_ji / A_ii applied iff (i,j),(k,i),(k,j) in S.              */
/* Sums run in ascending k (rev=1: descending, the same arithmetic in the   */
/* other order, used only to measure how much FP64 rounding order moves the */
/* result).  val[] follows the CSR layout; piv (optional) receives every     */
/* pivot p before the test.  store_f32=1 rounds every off-diagonal Theta_ji */
/* and every off-diagonal entry of L to float as soon as it is computed      */
/* (later columns then use the rounded values; pivots and L_ii stay double): */
/* the roundings of a factor with float entries kept in float, used only to  */
/* size test tolerances.  Returns the number of zeroed columns.              */
/* ------------------------------------------------------------------------ */

/* Entries of the matrix being factored, by CSR position e of (j, i) in the  */
/* pattern: from the covariance function (xo, K) or, when aval is given,    */
/* aval[e] (the matrix given on the pattern, Section 6).                    */
static double entry_at(const double* xo, i32 d, const ko_kernel* K, const double* aval, i64 e, i64 j, i64 i) {
    return aval ? aval[e] : theta_pos(xo, d, j, i, K);
}

static i64 ichol_any(const double* xo, i64 N, i32 d, const ko_kernel* K, const double* aval,
                     const i64* rowptr, const i32* col, double* val, char* zero_col, i32 rev, double* piv,
                     i32 store_f32) {
    i64 nnz = rowptr[N];
    i64* colptr = (i64*)malloc(sizeof(i64) * ((size_t)N + 1));
    i32* rowidx = (i32*)malloc(sizeof(i32) * (size_t)(nnz > 0 ? nnz : 1));
    i64* slot = (i64*)malloc(sizeof(i64) * (size_t)(nnz > 0 ? nnz : 1));
    ko_csr_to_csc(N, rowptr, col, colptr, rowidx, slot);
    for (i64 e = 0; e < nnz; ++e) val[e] = 0.0;
    i64 zeroed = 0;
    for (i64 i = 0; i < N; ++i) {
        i64 a0 = rowptr[i], a1 = rowptr[i + 1] - 1; /* row i without its diagonal: [a0, a1) */
        double p = entry_at(xo, d, K, aval, a1, i, i);
        if (!rev) for (i64 e = a0; e < a1; ++e) p -= val[e] * val[e];
        else for (i64 e = a1 - 1; e >= a0; --e) p -= val[e] * val[e];
        if (piv) piv[i] = p;
        if (!(p > 0.0)) {
            zero_col[i] = 1; zeroed++;
            continue; /* column stays zero, diagonal included */
        }
        zero_col[i] = 0;
        double Lii = sqrt(p);
        val[a1] = Lii;
        for (i64 q = colptr[i] + 1; q < colptr[i + 1]; ++q) { /* skip the diagonal entry (first) */
            i64 j = rowidx[q];
            i64 b0 = rowptr[j];
            i64 bij = slot[q];                 /* position of (j,i) in row j */
            /* merge row j (k < i) with row i (k < i) */
            double s = entry_at(xo, d, K, aval, bij, j, i);
            if (store_f32) s = (double)(float)s;
            if (!rev) {
                i64 u = a0, v = b0;
                while (u < a1 && v < bij) {
                    i32 ku = col[u], kv = col[v];
                    if (ku == kv) { s -= val[v] * val[u]; ++u; ++v; }
                    else if (ku < kv) ++u;
                    else ++v;
                }
            } else {
                i64 u = a1 - 1, v = bij - 1;
                while (u >= a0 && v >= b0) {
                    i32 ku = col[u], kv = col[v];
                    if (ku == kv) { s -= val[v] * val[u]; --u; --v; }
                    else if (ku > kv) --u;
                    else --v;
                }
            }
            double q = s / Lii;
            val[bij] = store_f32 ? (double)(float)q : q;
        }
    }
    free(colptr); free(rowidx); free(slot);
    return zeroed;
}

i64 ko_ichol(const double* xo, i64 N, i32 d, const ko_kernel* K,
             const i64* rowptr, const i32* col, double* val, char* zero_col, i32 rev, double* piv,
             i32 store_f32) {
    return ichol_any(xo, N, d, K, NULL, rowptr, col, val, zero_col, rev, piv, store_f32);
}

/* ICHOL(0) of a given symmetric matrix A: aval[e] is A_ji for the CSR entry */
/* e = (j, i), i <= j, of the pattern (Section 6: the reverse-order factor    */
/* of the precision matrix, or of sigma^2 A + I for a nugget).               */
i64 ko_ichol_given(i64 N, const i64* rowptr, const i32* col, const double* aval, double* val, char* zero_col,
                   i32 rev, i32 store_f32) {
    return ichol_any(NULL, N, 0, NULL, aval, rowptr, col, val, zero_col, rev, NULL, store_f32);
}

/* ------------------------------------------------------------------------ */
/* Supernodal multicolour ordering and sparsity pattern (the Construction of */
/* the stability section).  Readings: h = 1/2; the scale l[1] (the largest  */
/* finite length scale) normalises the hierarchy, so point m of the maximin  */
/* order is on level k(m) = the smallest k >= 1 with l[m] >= l[1] 2^-k (the  */
/* first point, l = inf, on level 1), and the hierarchical pseudometric is   */
/* d(a, b) = dist(a, b) / (l[1] 2^-min(k(a), k(b))), so d <= rho reads      */
/* dist <= R_min(k(a),k(b)) with R_k = (rho l[1]) 2^-k.                      */
/*  - supernodes of level k: greedily in maximin order, a point becomes one  */
/*    unless an earlier supernode of its level lies within d <= rho (so two  */
/*    supernodes are farther apart than rho, their rho/2-balls are disjoint,  */
/*    and every point lies within rho of one);                               */
/*  - every point goes to the nearest supernode of its level (squared        */
/*    distance, ties to the smaller index);                                 */
/*  - supernode pattern: (A, B) whenever members a of A and b of B have      */
/*    d(a, b) <= rho (A with itself included);                              */
/*  - colours: per level, greedy in maximin order of the supernodes, the     */
/*    smallest colour no earlier same-level neighbour in the pattern has;    */
/*  - ordering: by level, colour, supernode (maximin index of the supernode),  */
/*    then maximin index;                                                   */
/*  - pattern S: (q, p), p <= q in the new order, whenever the supernodes of  */
/*    q and p are a pattern pair.                                           */
/* Inputs: x (original order), the maximin perm and l (ko_maximin_brute).    */
/* Outputs: order[q] (original index at new position q), level, node (the    */
/* maximin index of the supernode) and colour of every new position, and    */
/* the CSR rows of S (rowptr[N+1]; col through *col_out, malloc'd; free it   */
/* with ko_free).                                                            */
/* ------------------------------------------------------------------------ */

static double R_of(double rl1, i32 k) { return ldexp(rl1, -k); }

typedef struct { i32 level, color, node, m; } sn_key;

static int sn_cmp(const void* pa, const void* pb) {
    const sn_key* a = (const sn_key*)pa;
    const sn_key* b = (const sn_key*)pb;
    if (a->level != b->level) return a->level < b->level ? -1 : 1;
    if (a->color != b->color) return a->color < b->color ? -1 : 1;
    if (a->node != b->node) return a->node < b->node ? -1 : 1;
    return a->m < b->m ? -1 : (a->m > b->m);
}

void ko_free(void* p) { free(p); }

i64 ko_supernodal(const double* x, i64 N, i32 d, const i32* perm, const double* l, double rho, i32* order,
                  i32* level_out, i32* node_out, i32* color_out, i64* rowptr, i32** col_out) {
    double* xo = (double*)malloc(sizeof(double) * (size_t)(N * d));
    for (i64 m = 0; m < N; ++m)
        for (i32 t = 0; t < d; ++t) xo[m * d + t] = x[(i64)perm[m] * d + t];
    const double l1 = N > 1 ? l[1] : 1.0;
    const double rl1 = rho * l1;
    i32* lev = (i32*)malloc(sizeof(i32) * (size_t)N);
    for (i64 m = 0; m < N; ++m) {
        i32 k = 1;
        if (m > 0)
            while (!(l[m] >= ldexp(l1, -k))) ++k;
        lev[m] = k;
    }
    /* supernodes, greedy per level in maximin order */
    char* sup = (char*)calloc((size_t)N, 1);
    for (i64 m = 0; m < N; ++m) {
        int take = 1;
        const double R = R_of(rl1, lev[m]);
        for (i64 s = 0; s < m && take; ++s)
            if (sup[s] && lev[s] == lev[m] && sqrt(d2_of(xo + m * d, xo + s * d, d)) <= R) take = 0;
        sup[m] = (char)take;
    }
    /* nearest supernode of the same level */
    i32* node = (i32*)malloc(sizeof(i32) * (size_t)N);
    for (i64 m = 0; m < N; ++m) {
        double best = INFINITY;
        i32 bs = -1;
        for (i64 s = 0; s < N; ++s)
            if (sup[s] && lev[s] == lev[m]) {
                double e = d2_of(xo + m * d, xo + s * d, d);
                if (e < best) { best = e; bs = (i32)s; }
            }
        node[m] = bs;
    }
    /* supernode pattern as a dense N x N bit set over supernode indices */
    char* adj = (char*)calloc((size_t)(N * N), 1);
    if (!adj) { /* too large for the dense set: report it instead of writing through NULL */
        free(xo); free(lev); free(sup); free(node);
        *col_out = NULL;
        return -1;
    }
    for (i64 a = 0; a < N; ++a)
        for (i64 b = 0; b <= a; ++b) {
            i32 kmin = lev[a] < lev[b] ? lev[a] : lev[b];
            if (a == b || sqrt(d2_of(xo + a * d, xo + b * d, d)) <= R_of(rl1, kmin)) {
                adj[(i64)node[a] * N + node[b]] = 1;
                adj[(i64)node[b] * N + node[a]] = 1;
            }
        }
    /* greedy colours per level in supernode (maximin) order */
    i32* colr = (i32*)malloc(sizeof(i32) * (size_t)N);
    char* used = (char*)malloc((size_t)N + 1);
    for (i64 s = 0; s < N; ++s) {
        colr[s] = -1;
        if (!sup[s]) continue;
        memset(used, 0, (size_t)N + 1);
        for (i64 t = 0; t < s; ++t)
            if (sup[t] && lev[t] == lev[s] && adj[s * N + t] && colr[t] >= 0) used[colr[t]] = 1;
        i32 c = 0;
        while (used[c]) ++c;
        colr[s] = c;
    }
    /* the ordering */
    sn_key* keys = (sn_key*)malloc(sizeof(sn_key) * (size_t)N);
    for (i64 m = 0; m < N; ++m) keys[m] = (sn_key){lev[m], colr[node[m]], node[m], (i32)m};
    qsort(keys, (size_t)N, sizeof(sn_key), sn_cmp);
    i32* pos = (i32*)malloc(sizeof(i32) * (size_t)N);
    for (i64 q = 0; q < N; ++q) {
        i32 m = keys[q].m;
        order[q] = perm[m];
        level_out[q] = lev[m];
        node_out[q] = node[m];
        color_out[q] = colr[node[m]];
        pos[m] = (i32)q;
    }
    /* the pattern in the new order */
    i32* mat = (i32*)malloc(sizeof(i32) * (size_t)N); /* maximin index at new position */
    for (i64 q = 0; q < N; ++q) mat[q] = keys[q].m;
    rowptr[0] = 0;
    for (i64 q = 0; q < N; ++q) {
        i64 c = 0;
        for (i64 p = 0; p <= q; ++p)
            if (adj[(i64)node[mat[q]] * N + node[mat[p]]]) ++c;
        rowptr[q + 1] = rowptr[q] + c;
    }
    i32* col = (i32*)malloc(sizeof(i32) * (size_t)(rowptr[N] > 0 ? rowptr[N] : 1));
    for (i64 q = 0; q < N; ++q) {
        i64 w = rowptr[q];
        for (i64 p = 0; p <= q; ++p)
            if (adj[(i64)node[mat[q]] * N + node[mat[p]]]) col[w++] = (i32)p;
    }
    *col_out = col;
    free(xo); free(lev); free(sup); free(node); free(adj); free(colr); free(used); free(keys); free(pos); free(mat);
    return rowptr[N];
}

/* ------------------------------------------------------------------------ */
/* Reverse elimination order (Section 6): position q of the reversed order   */
/* is position N-1-q of the maximin order.  The lower triangle of a          */
/* symmetric pattern in reversed positions is the upper one in maximin      */
/* positions: row q lists N-1-b for the rows b of maximin column a = N-1-q   */
/* (b >= a), ascending, so the diagonal comes last.  colptr/rowidx: the CSC  */
/* of the maximin-order lower triangle.                                      */
/* ------------------------------------------------------------------------ */

void ko_pattern_reverse(i64 N, const i64* colptr, const i32* rowidx, i64* rowptr_out, i32* col_out) {
    rowptr_out[0] = 0;
    for (i64 q = 0; q < N; ++q) {
        i64 a = N - 1 - q;
        rowptr_out[q + 1] = rowptr_out[q] + (colptr[a + 1] - colptr[a]);
    }
    for (i64 q = 0; q < N; ++q) {
        i64 a = N - 1 - q, w = rowptr_out[q];
        for (i64 e = colptr[a + 1] - 1; e >= colptr[a]; --e) col_out[w++] = (i32)(N - 1 - rowidx[e]);
    }
}

/* aval[e] = A(orig[j], orig[i]) for each CSR entry e = (j, i) of the        */
/* pattern, where orig maps a position to its original index and A is given  */
/* by CSR rows in original numbering (columns ascending); 0 where A has no   */
/* entry.  Returns the number of A's entries (u, v), u != v, whose position   */
/* pair is not in the pattern (ICHOL(0) drops them, Algorithm 2).           */
i64 ko_gather_entries(i64 N, const i64* rowptr, const i32* col, const i32* orig, const i64* arp, const i32* acol,
                      const double* aval_in, double* aval) {
    for (i64 j = 0; j < N; ++j)
        for (i64 e = rowptr[j]; e < rowptr[j + 1]; ++e) {
            i64 u = orig[j], v = orig[col[e]];
            double a = 0.0;
            for (i64 f = arp[u]; f < arp[u + 1]; ++f)
                if (acol[f] == v) { a = aval_in[f]; break; }
            aval[e] = a;
        }
    i32* pos = (i32*)malloc(sizeof(i32) * (size_t)(N > 0 ? N : 1));
    for (i64 q = 0; q < N; ++q) pos[orig[q]] = (i32)q;
    i64 outside = 0;
    for (i64 u = 0; u < N; ++u)
        for (i64 f = arp[u]; f < arp[u + 1]; ++f) {
            i64 v = acol[f];
            if (v == u) continue;
            i64 j = pos[u] > pos[v] ? pos[u] : pos[v], i = pos[u] > pos[v] ? pos[v] : pos[u];
            int found = 0;
            for (i64 e = rowptr[j]; e < rowptr[j + 1]; ++e)
                if (col[e] == i) { found = 1; break; }
            if (!found) outside++;
        }
    free(pos);
    return outside;
}

/* ------------------------------------------------------------------------ */
/* Triangular solves with L (task (2), Section 1): y = L^{-1} b, x = L^{-T} y.*/
/* A zeroed column i uses diag[i] supplied by the caller.                    */
/* ------------------------------------------------------------------------ */

void ko_solve_lower(i64 N, const i64* rowptr, const i32* col, const double* val, const double* diag,
                    const double* b, double* y) {
    for (i64 j = 0; j < N; ++j) {
        double s = b[j];
        for (i64 e = rowptr[j]; e < rowptr[j + 1] - 1; ++e) s -= val[e] * y[col[e]];
        y[j] = s / diag[j];
    }
}

void ko_solve_upper(i64 N, const i64* rowptr, const i32* col, const double* val, const double* diag,
                    const double* y, double* x) {
    for (i64 i = 0; i < N; ++i) x[i] = y[i];
    for (i64 j = N - 1; j >= 0; --j) {
        x[j] = x[j] / diag[j];
        for (i64 e = rowptr[j]; e < rowptr[j + 1] - 1; ++e) x[col[e]] -= val[e] * x[j];
    }
}

/* ------------------------------------------------------------------------ */
/* Tasks (1), (3), (4) of Section 1 with the factor standing in for Theta:  */
/*   (1) Theta v ~ L (L^T v);  (3) logdet Theta ~ 2 sum_i log L_ii;          */
/*   (4) a sample of N(0, L L^T) is L z for z ~ N(0, I).                     */
/* All in ordered positions; L is the CSR factor with its diagonal last in   */
/* each row (zero for a dropped column).                                     */
/* ------------------------------------------------------------------------ */

/* y = L z */
void ko_l_matvec(i64 N, const i64* rowptr, const i32* col, const double* val, const double* z, double* y) {
    for (i64 j = 0; j < N; ++j) {
        double s = 0.0;
        for (i64 e = rowptr[j]; e < rowptr[j + 1]; ++e) s += val[e] * z[col[e]];
        y[j] = s;
    }
}

/* w = L^T v: entry (j, k) of L adds L_jk v_j to w_k */
void ko_lt_matvec(i64 N, const i64* rowptr, const i32* col, const double* val, const double* v, double* w) {
    for (i64 k = 0; k < N; ++k) w[k] = 0.0;
    for (i64 j = 0; j < N; ++j)
        for (i64 e = rowptr[j]; e < rowptr[j + 1]; ++e) w[col[e]] += val[e] * v[j];
}

/* 2 sum log L_ii over the kept columns; *zeroed = number of dropped ones
   (then L L^T is singular and its log-determinant is -infinity) */
double ko_logdet(i64 N, const i64* rowptr, const double* val, i64* zeroed) {
    double s = 0.0;
    i64 z = 0;
    for (i64 i = 0; i < N; ++i) {
        double Lii = val[rowptr[i + 1] - 1];
        if (Lii > 0.0) s += log(Lii);
        else z++;
    }
    *zeroed = z;
    return 2.0 * s;
}

/* ------------------------------------------------------------------------ */
/* y = Theta^S v: the kernel matrix restricted to the symmetric pattern S,   */
/* entries from the coordinates (the sparse matrix the factorisation sees).  */
/* ------------------------------------------------------------------------ */

void ko_theta_s_matvec(const double* xo, i64 N, i32 d, const ko_kernel* K,
                       const i64* rowptr, const i32* col, const double* v, double* y) {
    for (i64 j = 0; j < N; ++j) y[j] = 0.0;
    for (i64 j = 0; j < N; ++j) {
        for (i64 e = rowptr[j]; e < rowptr[j + 1] - 1; ++e) {
            i64 k = col[e];
            double t = theta_pos(xo, d, j, k, K);
            y[j] += t * v[k];
            y[k] += t * v[j];
        }
        y[j] += theta_pos(xo, d, j, j, K) * v[j];
    }
}

/* y = Theta v with the dense kernel matrix (O(N^2)). */
void ko_theta_dense_matvec(const double* xo, i64 N, i32 d, const ko_kernel* K, const double* v, double* y) {
    for (i64 j = 0; j < N; ++j) {
        double s = 0.0;
        for (i64 k = 0; k < N; ++k) s += theta_pos(xo, d, j, k, K) * v[k];
        y[j] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Preconditioned CG on A x = b with A = Theta^S (op=1) or dense Theta       */
/* (op=2), preconditioner M = L L^T (Section 4.3: CG preconditioned with the */
/* factor).  Starts from x = 0.  Returns iterations; relres gets the final   */
/* ||b - A x|| / ||b||; status 0 converged, 1 not converged, 2 p^T A p <= 0.   */
/* ------------------------------------------------------------------------ */

static double dotv(i64 n, const double* a, const double* b) {
    double s = 0.0;
    for (i64 i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

i32 ko_pcg(const double* xo, i64 N, i32 d, const ko_kernel* K,
           const i64* rowptr, const i32* col, const double* val, const double* diag, i32 op,
           const double* b, double rtol, i32 maxit, double* x, double* relres, i32* status) {
    double* r = (double*)malloc(sizeof(double) * (size_t)N);
    double* z = (double*)malloc(sizeof(double) * (size_t)N);
    double* p = (double*)malloc(sizeof(double) * (size_t)N);
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    double* t = (double*)malloc(sizeof(double) * (size_t)N);
    for (i64 i = 0; i < N; ++i) { x[i] = 0.0; r[i] = b[i]; }
    double bn = sqrt(dotv(N, b, b));
    *status = 1;
    i32 it = 0;
    double rn = bn;
    if (bn == 0.0) { *relres = 0.0; *status = 0; goto done; }
    ko_solve_lower(N, rowptr, col, val, diag, r, t);
    ko_solve_upper(N, rowptr, col, val, diag, t, z);
    for (i64 i = 0; i < N; ++i) p[i] = z[i];
    double rz = dotv(N, r, z);
    for (it = 0; it < maxit; ++it) {
        if (rn / bn <= rtol) { *status = 0; break; }
        if (op == 2) ko_theta_dense_matvec(xo, N, d, K, p, q);
        else ko_theta_s_matvec(xo, N, d, K, rowptr, col, p, q);
        double pq = dotv(N, p, q);
        if (!(pq > 0.0)) { *status = 2; break; }
        double alpha = rz / pq;
        for (i64 i = 0; i < N; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        rn = sqrt(dotv(N, r, r));
        ko_solve_lower(N, rowptr, col, val, diag, r, t);
        ko_solve_upper(N, rowptr, col, val, diag, t, z);
        double rz2 = dotv(N, r, z);
        double beta = rz2 / rz;
        rz = rz2;
        for (i64 i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    if (it == maxit && rn / bn <= rtol) *status = 0;
    /* true residual */
    if (op == 2) ko_theta_dense_matvec(xo, N, d, K, x, q);
    else ko_theta_s_matvec(xo, N, d, K, rowptr, col, x, q);
    for (i64 i = 0; i < N; ++i) q[i] = b[i] - q[i];
    *relres = sqrt(dotv(N, q, q)) / bn;
done:
    free(r); free(z); free(p); free(q); free(t);
    return it;
}

/* ------------------------------------------------------------------------ */
/* Sampled relative Frobenius error E (Section 4.4):                          */
/*   E ~ sqrt(sum_k ((L L^T)_{ik jk} - Theta_{ik jk})^2) / sqrt(sum_k Theta^2) */
/* over given index pairs in ORIGINAL numbering; pos maps original ->       */
/* ordered.  (L L^T)_ij is the merge of rows i and j of L.                    */
/* ------------------------------------------------------------------------ */

static double llt_entry(const i64* rowptr, const i32* col, const double* val, i64 a, i64 b) {
    i64 u = rowptr[a], ue = rowptr[a + 1], v = rowptr[b], ve = rowptr[b + 1];
    double s = 0.0;
    while (u < ue && v < ve) {
        if (col[u] == col[v]) { s += val[u] * val[v]; ++u; ++v; }
        else if (col[u] < col[v]) ++u;
        else ++v;
    }
    return s;
}

double ko_llt_entry(const i64* rowptr, const i32* col, const double* val, i64 a, i64 b) {
    return llt_entry(rowptr, col, val, a, b);
}

void ko_frob_error(const double* xo, i64 N, i32 d, const ko_kernel* K,
                   const i64* rowptr, const i32* col, const double* val, const i64* pos,
                   i64 m, const i64* pi, const i64* pj, const char* keep,
                   double* num2, double* den2, i64* kept) {
    double a = 0.0, b = 0.0; i64 c = 0;
    (void)N;
    for (i64 t = 0; t < m; ++t) {
        if (keep && !keep[t]) continue;
        i64 i = pos[pi[t]], j = pos[pj[t]];
        double th = theta_pos(xo, d, i, j, K);
        double e = llt_entry(rowptr, col, val, i, j) - th;
        a += e * e; b += th * th; c++;
    }
    *num2 = a; *den2 = b; *kept = c;
}

/* ------------------------------------------------------------------------ */
/* Approximate PCA (Section 2.5, Theorem on rank-k approximation): the first  */
/* k columns of L, rows scattered back to original order, column-major.      */
/* ------------------------------------------------------------------------ */

void ko_pca_truncate(i64 N, const i64* rowptr, const i32* col, const double* val, const i32* perm,
                     i32 k, double* Lk) {
    for (i64 e = 0; e < N * (i64)k; ++e) Lk[e] = 0.0;
    for (i64 j = 0; j < N; ++j)
        for (i64 e = rowptr[j]; e < rowptr[j + 1]; ++e)
            if (col[e] < k) Lk[(i64)perm[j] + N * (i64)col[e]] = val[e];
}

/* Power iteration for ||Theta - Lk Lk^T||_2 on ORIGINAL order coordinates x.
   v0: unit start vector.  Returns |v^T B v| after iters steps. */
double ko_pca_error_power(const double* x, i64 N, i32 d, const ko_kernel* K,
                          i32 k, const double* Lk, const double* v0, i32 iters) {
    double* v = (double*)malloc(sizeof(double) * (size_t)N);
    double* w = (double*)malloc(sizeof(double) * (size_t)N);
    double* c = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (i64 i = 0; i < N; ++i) v[i] = v0[i];
    double est = 0.0;
    for (i32 it = 0; it < iters; ++it) {
        ko_theta_dense_matvec(x, N, d, K, v, w);
        for (i32 a = 0; a < k; ++a) { double s = 0.0; for (i64 i = 0; i < N; ++i) s += Lk[i + N * a] * v[i]; c[a] = s; }
        for (i32 a = 0; a < k; ++a) for (i64 i = 0; i < N; ++i) w[i] -= Lk[i + N * a] * c[a];
        est = fabs(dotv(N, v, w));
        double nw = sqrt(dotv(N, w, w));
        if (nw == 0.0) break;
        for (i64 i = 0; i < N; ++i) v[i] = w[i] / nw;
    }
    free(v); free(w); free(c);
    return est;
}

/* ------------------------------------------------------------------------ */
/* Work counters of the left-looking factor:                                 */
/*   F = sum_{(j,i) in S, j>i} |R_j cap R_i| + sum_i |R_i|   (multiply-adds)  */
/*   M = sum_{(j,i) in S, j>i} (|R_j cap [0,i)| + |R_i|)     (merge steps)    */
/*   P = sum_{(j,i) in S, j>i} |R_j cap [0,i)|               (row prefixes)   */
/*   Rsum = sum_i |R_i|                                                       */
/* ------------------------------------------------------------------------ */

void ko_work_counters(i64 N, const i64* rowptr, const i32* col, i64* F, i64* M, i64* P, i64* Rsum) {
    i64 nnz = rowptr[N];
    i64* colptr = (i64*)malloc(sizeof(i64) * ((size_t)N + 1));
    i32* rowidx = (i32*)malloc(sizeof(i32) * (size_t)(nnz > 0 ? nnz : 1));
    i64* slot = (i64*)malloc(sizeof(i64) * (size_t)(nnz > 0 ? nnz : 1));
    ko_csr_to_csc(N, rowptr, col, colptr, rowidx, slot);
    i64 f = 0, mm = 0, pp = 0, rs = 0;
    for (i64 i = 0; i < N; ++i) {
        i64 a0 = rowptr[i], a1 = rowptr[i + 1] - 1;
        i64 ri = a1 - a0;
        rs += ri; f += ri;
        for (i64 q = colptr[i] + 1; q < colptr[i + 1]; ++q) {
            i64 j = rowidx[q];
            i64 b0 = rowptr[j], bij = slot[q];
            i64 u = a0, v = b0, inter = 0;
            while (u < a1 && v < bij) {
                if (col[u] == col[v]) { inter++; ++u; ++v; }
                else if (col[u] < col[v]) ++u;
                else ++v;
            }
            f += inter;
            pp += bij - b0;
            mm += (bij - b0) + ri;
        }
    }
    *F = f; *M = mm; *P = pp; *Rsum = rs;
    free(colptr); free(rowidx); free(slot);
}
