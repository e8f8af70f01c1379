// ICHOL(0) by column groups: the supernodal block factorisation of the
// stability appendix (a block Cholesky whose Schur-complement updates are kept
// on the supernode pairs of the pattern), for any pattern, in one persistent
// sync-free kernel.
//
// A *group* is a run of consecutive columns g0 .. g1-1 whose rows share one
// list of earlier columns (row a is row a-1 with a appended) and whose
// columns share one set of later rows (column a-1 below a is column a below
// a).  In the supernodal multicolour ordering every supernode is such a run
// (its rows and columns are unions of whole supernode ranges); in the maximin
// ordering nearly every group is a single column.  Long runs are cut into
// groups of at most MM columns.  With P the length of the shared prefix (the
// entries of row g0 before its diagonal), the group's block factorisation is
//
//   D     = Theta_AA - V^T V,       V = the P x m prefix values of A's rows
//   L_AA  = chol(D) with the zero-column rule of Section 4.4 (a nonpositive
//           pivot zeroes its column; later columns see it as zero)
//   L_jA  = (Theta_jA - L_j,prefix V) L_AA^{-T}   for every row j below A,
//
// which is Algorithm 2 on this pattern with the sums in another order (the
// appendix shows the block and the entry-wise algorithms agree).  The rows
// below A are the column g0 of the CSC past the group; each row j holds A's
// columns at consecutive positions, starting where the CSC slot of (j, g0)
// points.
//
// Work units ("tasks") are (group, chunk of rows below), one per CTA, listed
// with the groups in dependency order (level of the group's first column,
// then the schedule's order) and handed out by an atomic ticket.  A CTA that
// takes a task waits (bounded spin with backoff) until every group that owns
// a column of the prefix has published all its tasks, puts the prefix into
// shared memory (an open-addressing table column -> position, and the P x m
// values), forms D with compensated dot products spread over its warps,
// factors it on one warp in FP64, and then streams each row's prefix once
// for all m columns: groups of G lanes own a row, every entry is looked up
// once and feeds m compensated accumulators.  The row's m results then follow
// by a forward substitution with L_AA.  The chunk 0 task also writes L_AA and
// the pivots.  The task publishes by a release increment of done[group].
//
// Compared with the column tasks of factor.cu, a row's prefix is read once per
// group instead of once per column, so the operand stream shrinks by the mean
// group size.  Arithmetic: FP32 form -- values, products and the compensated
// (Dot2) sums in FP32, D, the small factorisation and the forward
// substitution in FP64 from the stored values; FP64 form -- FP64 throughout.
#include <algorithm>

#include "ichol.cuh"

namespace kc {

// One task per CTA of KC_BLOCK_THREADS threads; KC_BLOCK_MINB resident CTAs
// per SM that the register budget is cut for.
#ifndef KC_BLOCK_THREADS
#define KC_BLOCK_THREADS 128
#endif
#ifndef KC_BLOCK_MINB
#define KC_BLOCK_MINB 8
#endif
constexpr int BF_THREADS = KC_BLOCK_THREADS;
constexpr int BF_WARPS = BF_THREADS / 32;
constexpr int BF_MAXG = 8;       // columns per group at most
// (column, value) loads per lane in flight while streaming a row
#ifndef KC_BLOCK_BU
#define KC_BLOCK_BU 4
#endif
constexpr int BU = KC_BLOCK_BU;

template <typename T>
struct GroupArgs {
    int64_t N;
    int d;
    const double* __restrict__ x;
    const int64_t* __restrict__ rowptr;
    const int32_t* __restrict__ col;
    const int64_t* __restrict__ colptr;
    const int32_t* __restrict__ rowidx;
    const int64_t* __restrict__ slot;
    const int32_t* __restrict__ gstart;    // group g = columns [gstart[g], gstart[g+1])
    const int32_t* __restrict__ group_of;  // column -> group
    const int2* __restrict__ tasks;        // (group, chunk)
    int64_t ntasks;
    int rpt;
    T* val;
    double* diag;
    unsigned* done;  // per group: -(tasks) + finished tasks
    unsigned long long* ticket;
    int* status;
    unsigned long long* zero_piv;
    KernelParams kp;
    long long spin_limit;
    int hbits;  // prefix table: 2^hbits slots
    int pmax;   // longest shared prefix: rows of the value table
    int lanes;  // lanes per row
};

__device__ __forceinline__ int gslot(int k, int hbits) { return (int)(((unsigned)k * 2654435761u) >> (32 - hbits)); }

// position of column k in the staged prefix, or -1
__device__ __forceinline__ int prefix_find(const unsigned long long* tab, int hbits, int k) {
    const int mask = (1 << hbits) - 1;
    int h = gslot(k, hbits);
    for (;;) {
        const unsigned long long w = tab[h];
        const int key = (int)(unsigned)w;
        if (key == k) return (int)(w >> 32);
        if (key < 0) return -1;
        h = (h + 1) & mask;
    }
}

// (t, s), s <= t, of the lower-triangle index q = t (t + 1) / 2 + s
__device__ __forceinline__ void tri_ts(int q, int& t, int& s) {
    t = 0;
    while ((t + 1) * (t + 2) / 2 <= q) ++t;
    s = q - t * (t + 1) / 2;
}

// The rows q in [qb, qe) of the CSC below a group of m <= M4 <= MM columns g0 ..
// g0+m-1: each row's prefix streamed once by G lanes (BU loads per lane in
// flight, one table lookup per entry feeding m compensated accumulators),
// then the forward substitution with L_AA: each result (theta - sum -
// sum_w x_w L_uw) times the stored reciprocal of L_uu (0 for a dropped pivot);
// FP32 form in FP32 (the compensated sum's two parts subtracted in turn, as
// the column kernel finishes an entry), FP64 form in FP64.
template <typename T>
__device__ __forceinline__ T fsub_dot(T v, T a, T b);
template <>
__device__ __forceinline__ float fsub_dot(float v, float a, float b) { return fmaf(-a, b, v); }
template <>
__device__ __forceinline__ double fsub_dot(double v, double a, double b) { return fma(-a, b, v); }

template <typename T, int MM, bool GEN, int GC, int M4 = MM>
__device__ __forceinline__ void group_rows(const GroupArgs<T>& A, int64_t qb, int64_t qe, int g0, int m,
                                           const unsigned long long* tab, int hb, const T* V, const T* Laa,
                                           const double* Ld, const T* Linv) {
    const unsigned FULL = 0xffffffffu;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int G = GC > 0 ? GC : A.lanes, ngr = 32 / G, grp = lane / G, sub = lane % G;
    for (int64_t q0 = qb + (int64_t)(warp * ngr); q0 < qe; q0 += (int64_t)BF_WARPS * ngr) {
        const int64_t q = q0 + grp;
        const bool act = q < qe;
        int j = 0;
        int64_t e = 0, es = 0;
        if (act) {
            j = __ldg(&A.rowidx[q]);
            e = __ldg(&A.slot[q]);  // L_j,g0 lives at e, the prefix of row j is [es, e)
            es = A.rowptr[j];
        }
        T th = (T)0;  // lane sub: Theta_j,(g0+sub)
        if (act && sub < m)
            th = theta_off<T, GEN>(A.kp, A.d, A.x + (int64_t)j * A.d, A.x + (int64_t)(g0 + sub) * A.d);
        Acc<T> acc[M4];
        if (act) {
            for (int64_t f0 = es + sub; f0 < e; f0 += (int64_t)BU * G) {
                int k[BU];
                T w[BU];
#pragma unroll
                for (int v = 0; v < BU; ++v) {
                    const int64_t f = f0 + (int64_t)v * G;
                    k[v] = f < e ? __ldg(&A.col[f]) : -1;
                    w[v] = f < e ? ldcg(&A.val[f]) : (T)0;
                }
#pragma unroll
                for (int v = 0; v < BU; ++v) {
                    const int p = k[v] >= 0 ? prefix_find(tab, hb, k[v]) : -1;
                    if (p >= 0) {
                        const T* vp = V + (int64_t)p * MM;
#pragma unroll
                        for (int u = 0; u < M4; ++u)
                            if (u < m) acc[u].add(w[v], vp[u]);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < M4; ++u)
            if (u < m) acc[u].group_reduce(G);
        T x[M4];
#pragma unroll
        for (int u = 0; u < M4; ++u) {
            const T thu = __shfl_sync(FULL, th, grp * G + (u < m ? u : 0));
            if (u < m) {
                if constexpr (sizeof(T) == 4) {
                    float v = __fsub_rn(__fsub_rn(thu, acc[u].s), acc[u].c);
#pragma unroll
                    for (int w2 = 0; w2 < u; ++w2) v = fsub_dot(v, x[w2], Laa[u * MM + w2]);
                    x[u] = __fmul_rn(v, Linv[u]);
                } else {
                    double v = thu - acc[u].total();
#pragma unroll
                    for (int w2 = 0; w2 < u; ++w2) v = fsub_dot(v, x[w2], Laa[u * MM + w2]);
                    x[u] = v * Linv[u];  // (the GB300's FP64 divisions are slow)
                }
            }
        }
        if (act && sub == 0)
#pragma unroll
            for (int u = 0; u < M4; ++u)
                if (u < m) A.val[e + u] = x[u];
    }
}

// GC > 0: the lanes per row at compile time (the FP32 form's default 8).
template <typename T, int MM, bool GEN, int GC>
__global__ void __launch_bounds__(BF_THREADS, KC_BLOCK_MINB) ichol_group_k(GroupArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    // layout: D (FP64, lower triangle), the pivots' roots (FP64), L_AA (T),
    // control words, the prefix table (8-byte slots), the values V[p][t]
    double* D = (double*)smem;
    double* Ld = D + MM * (MM + 1) / 2;
    T* Laa = (T*)(Ld + MM);
    T* Linv = Laa + MM * MM;  // the reciprocals of the pivots' roots (0 for a dropped pivot)
    int* ctl = (int*)(Linv + MM);
    unsigned long long* tab = (unsigned long long*)(((uintptr_t)(ctl + 4) + 15) & ~(uintptr_t)15);
    T* V = (T*)(tab + (1 << A.hbits));
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    for (;;) {
        __syncthreads();  // the previous task's shared reads are done
        if (tid == 0) {
            const unsigned long long t = atomicAdd(A.ticket, 1ULL);
            ctl[0] = (int)min(t, (unsigned long long)A.ntasks);
            ctl[1] = ld_volatile_s32(A.status);
        }
        __syncthreads();
        const int64_t t = ctl[0];
        if (t >= A.ntasks || ctl[1] != 0) return;
        const int2 tk = A.tasks[t];
        const int g = tk.x, chunk = tk.y;
        const int g0 = A.gstart[g], m = A.gstart[g + 1] - g0;
        const int64_t a0 = A.rowptr[g0];
        const int P = (int)(A.rowptr[g0 + 1] - 1 - a0);

        // wait for the groups owning the prefix's columns (each group checked
        // where its run of columns starts)
        bool ok = true;
        for (int p = tid; p < P && ok; p += BF_THREADS) {
            const int gk = A.group_of[__ldg(&A.col[a0 + p])];
            if (p > 0 && A.group_of[__ldg(&A.col[a0 + p - 1])] == gk) continue;
            if ((int)ld_relaxed_u32(&A.done[gk]) < 0) ok = spin_done(&A.done[gk], A.status, A.spin_limit);
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
            return;
        }
        fence_acq_rel_gpu();  // acquire: the prefix values are visible from here on

        // stage the prefix: table column -> position (sized to this prefix, load
        // factor <= 3/4), values of the m rows
        int hb = 5;
        while (3 * (1 << hb) < 4 * P) ++hb;
        for (int h = tid; h < (1 << hb); h += BF_THREADS) tab[h] = ~0ull;
        int64_t rs[MM];
#pragma unroll
        for (int u = 0; u < MM; ++u) rs[u] = u < m ? A.rowptr[g0 + u] : 0;
        __syncthreads();
        {
            const int mask = (1 << hb) - 1;
            for (int p = tid; p < P; p += BF_THREADS) {
                const int k = __ldg(&A.col[a0 + p]);
                const unsigned long long w = ((unsigned long long)(unsigned)p << 32) | (unsigned)k;
                int h = gslot(k, hb);
                while (atomicCAS(&tab[h], ~0ull, w) != ~0ull) h = (h + 1) & mask;
#pragma unroll
                for (int u = 0; u < MM; ++u) V[(int64_t)p * MM + u] = u < m ? ldcg(&A.val[rs[u] + p]) : (T)0;
            }
        }
        __syncthreads();

        // D = Theta_AA - V^T V (lower triangle), the dots spread over the warps
        const KernelParams& kp = A.kp;
        for (int q = warp; q < m * (m + 1) / 2; q += BF_WARPS) {
            int tt, ss;
            tri_ts(q, tt, ss);
            Acc<T> acc;
            for (int p = lane; p < P; p += 32) acc.add(V[(int64_t)p * MM + tt], V[(int64_t)p * MM + ss]);
            acc.group_reduce(32);
            if (lane == 0) {
                const double th = tt == ss ? kp.sigma2 + kp.nugget
                                           : (double)theta_off<T, GEN>(kp, A.d, A.x + (int64_t)(g0 + tt) * A.d,
                                                                       A.x + (int64_t)(g0 + ss) * A.d);
                D[q] = th - acc.total();
            }
        }
        __syncthreads();

        // L_AA on warp 0, column by column in FP64 from the stored values; lane t
        // owns row t.  Every lane forms the pivot the same way (same bits).
        if (warp == 0) {
            for (int s = 0; s < m; ++s) {
                double p = D[s * (s + 1) / 2 + s];
                for (int u = 0; u < s; ++u) {
                    const double v = (double)Laa[s * MM + u];
                    p -= v * v;
                }
                const bool zero = !(p > 0.0);
                const double Lss = zero ? 0.0 : sqrt(p);
                const double rinv = zero ? 0.0 : 1.0 / Lss;  // one FP64 division per column
                if (lane > s && lane < m) {
                    double v = D[lane * (lane + 1) / 2 + s];
                    for (int u = 0; u < s; ++u) v -= (double)Laa[lane * MM + u] * (double)Laa[s * MM + u];
                    Laa[lane * MM + s] = (T)(v * rinv);
                }
                if (lane == 0) {
                    Laa[s * MM + s] = (T)Lss;
                    Ld[s] = Lss;
                    Linv[s] = (T)rinv;
                }
                __syncwarp();
            }
            if (chunk == 0 && lane < m) {
                const int64_t rb = A.rowptr[g0 + lane] + P;  // row g0+lane: columns g0 .. g0+lane
                for (int u = 0; u <= lane; ++u) A.val[rb + u] = Laa[lane * MM + u];
                A.diag[g0 + lane] = Ld[lane];
                if (Ld[lane] == 0.0) atomicAdd(A.zero_piv, 1ULL);
            }
        }
        __syncthreads();

        // the rows below the group: column g0 of the CSC past its first m rows,
        // FP32 form: one code path for every group size, accumulators past m predicated off (with a
        // second path for groups of at most 4 columns, instruction fetches missed the cache: 56.7
        // against 50.5 ms on the 2^20 supernodal pattern); FP64 keeps that second path (126.6 against
        // 138.4 ms)
        const int64_t qb = A.colptr[g0] + m + (int64_t)chunk * A.rpt;
        const int64_t qe = min(A.colptr[g0 + 1], qb + A.rpt);
        if constexpr (sizeof(T) == 8) {
            if (m <= 4) group_rows<T, MM, GEN, GC, 4>(A, qb, qe, g0, m, tab, hb, V, Laa, Ld, Linv);
            else group_rows<T, MM, GEN, GC>(A, qb, qe, g0, m, tab, hb, V, Laa, Ld, Linv);
        } else {
            group_rows<T, MM, GEN, GC>(A, qb, qe, g0, m, tab, hb, V, Laa, Ld, Linv);
        }
        __syncthreads();
        if (tid == 0) {
            fence_acq_rel_gpu();
            red_release_add_u32(&A.done[g], 1u);
        }
    }
}

// ------------------------------------------------------------ group plan

// same[a] = 1 when column a joins the group of column a-1: row a is row a-1
// with a appended, and column a-1 below a is column a below a.  A warp per
// column; the comparisons run over the lanes.  A comparison longer than
// GRP_CHUNK entries (the coarsest columns hold nearly every row) is only
// sized here: nchunk[a] chunks of GRP_CHUNK entries, which grp_same_long_k
// spreads over the grid (one warp walking a column of 10^6 rows took 14 ms).
constexpr int64_t GRP_CHUNK = 1024;
__global__ void grp_same_k(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const int64_t* __restrict__ colptr, const int32_t* __restrict__ rowidx, int64_t N,
                           int* __restrict__ same, int64_t* __restrict__ nchunk) {
    const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = lane_id();
    if (a >= N) return;
    int ok = a > 0;
    int64_t nc = 0;
    if (ok) {
        const int64_t r1 = rowptr[a - 1], n1 = rowptr[a] - r1, r2 = rowptr[a], n2 = rowptr[a + 1] - r2;
        const int64_t c1 = colptr[a - 1], m1 = colptr[a] - c1, c2 = colptr[a], m2 = colptr[a + 1] - c2;
        ok = n2 == n1 + 1 && m1 == m2 + 1 && m1 >= 2 && rowidx[c1 + 1] == (int32_t)a;
        const int64_t total = n1 + m2 - 1;  // row entries, then column entries below a
        if (ok && total > GRP_CHUNK) {
            nc = (total + GRP_CHUNK - 1) / GRP_CHUNK;  // same[a] = 1 until a chunk differs
        } else if (ok) {
            bool bad = false;
            for (int64_t p = lane; p < n1 && !bad; p += 32) bad = col[r2 + p] != col[r1 + p];
            for (int64_t q = lane; q + 1 < m2 && !bad; q += 32) bad = rowidx[c1 + 2 + q] != rowidx[c2 + 1 + q];
            ok = !__any_sync(0xffffffffu, bad);
        }
    }
    if (lane == 0) {
        same[a] = ok;
        nchunk[a] = nc;
    }
}

// The long comparisons of grp_same_k: chunk w of all of them (choff = the
// exclusive scan of nchunk, choff[N] chunks in all) goes to one warp, which
// finds its column by binary search in choff; a difference clears same[a]
// (every writer stores the same 0).
__global__ void grp_same_long_k(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const int64_t* __restrict__ colptr, const int32_t* __restrict__ rowidx, int64_t N,
                                const int64_t* __restrict__ choff, int* __restrict__ same) {
    const int lane = lane_id();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nch = choff[N];
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nch; w += nw) {
        int64_t lo = 0, hi = N;  // the last a with choff[a] <= w (its chunks hold w)
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (choff[mid] <= w) lo = mid;
            else hi = mid;
        }
        const int64_t a = lo;
        const int64_t r1 = rowptr[a - 1], n1 = rowptr[a] - r1, r2 = rowptr[a];
        const int64_t c1 = colptr[a - 1], c2 = colptr[a], m2 = colptr[a + 1] - c2;
        const int64_t t0 = (w - choff[a]) * GRP_CHUNK, t1 = min(n1 + m2 - 1, t0 + GRP_CHUNK);
        bool bad = false;
        for (int64_t t = t0 + lane; t < t1; t += 32)
            bad |= t < n1 ? col[r2 + t] != col[r1 + t] : rowidx[c1 + 2 + (t - n1)] != rowidx[c2 + 1 + (t - n1)];
        if (__any_sync(0xffffffffu, bad) && lane == 0) same[a] = 0;
    }
}

// sflag[a] = 1 where a run of columns begins (same[a] == 0)
__global__ void grp_runflag_k(const int* __restrict__ same, int64_t N, int64_t* __restrict__ sflag) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < N) sflag[a] = same[a] == 0;
}
// the exclusive scan made inclusive: incl[a] = runs starting at or before a
__global__ void grp_inclusive_k(const int64_t* __restrict__ sflag, int64_t N, int64_t* __restrict__ incl) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < N) incl[a] += sflag[a];
}
// run start of every column (the nearest column at or before it with same == 0)
__global__ void grp_runstart_k(const int* __restrict__ same, const int64_t* __restrict__ incl, int64_t N,
                               int32_t* __restrict__ runstart) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < N && !same[a]) runstart[incl[a] - 1] = (int32_t)a;
}
// start[a] = 1 where a group begins: a run's start, then every MM columns
__global__ void grp_start_k(const int64_t* __restrict__ incl, const int32_t* __restrict__ runstart, int64_t N, int MM,
                            int64_t* __restrict__ start) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    const int64_t q = a - runstart[incl[a] - 1];
    start[a] = (q % MM) == 0;
}
// gstart, group_of from the exclusive scan of start
__global__ void grp_ids_k(const int64_t* __restrict__ start, const int64_t* __restrict__ gex, int64_t N,
                          int32_t* __restrict__ gstart, int32_t* __restrict__ group_of) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N) return;
    const int64_t gid = gex[a] + start[a] - 1;
    group_of[a] = (int32_t)gid;
    if (start[a]) gstart[gid] = (int32_t)a;
}
// position-order flags of group starts, for compacting the schedule's order
__global__ void grp_orderflag_k(const int32_t* __restrict__ order, const int64_t* __restrict__ start, int64_t N,
                                int64_t* __restrict__ flag) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) flag[p] = start[order[p]];
}
// gorder[rank] = group of the rank-th group start in the schedule's order; its task count
__global__ void grp_tasks_count_k(const int32_t* __restrict__ order, const int64_t* __restrict__ flag,
                                  const int64_t* __restrict__ fex, const int32_t* __restrict__ group_of,
                                  const int32_t* __restrict__ gstart, const int64_t* __restrict__ colptr,
                                  const int64_t* __restrict__ rowptr, int64_t N, int rpt, int32_t* __restrict__ gorder,
                                  int64_t* __restrict__ cnt, unsigned* __restrict__ done, int* __restrict__ pmax) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N || !flag[p]) return;
    const int a = order[p];
    const int gi = group_of[a];
    const int m = gstart[gi + 1] - gstart[gi];
    const int64_t below = colptr[a + 1] - colptr[a] - m;
    const int64_t nt = below <= 0 ? 1 : (below + rpt - 1) / rpt;
    gorder[fex[p]] = gi;
    cnt[fex[p]] = nt;
    done[gi] = 0u - (unsigned)nt;
    atomicMax(pmax, (int)(rowptr[a + 1] - 1 - rowptr[a]));
}
__global__ void grp_tasks_fill_k(const int32_t* __restrict__ gorder, const int64_t* __restrict__ toff, int64_t ng,
                                 int2* __restrict__ tasks) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = lane_id();
    if (r >= ng) return;
    const int gi = gorder[r];
    for (int64_t t = toff[r] + lane; t < toff[r + 1]; t += 32) tasks[t] = make_int2(gi, (int)(t - toff[r]));
}

kc_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Arena& A, cudaStream_t s);

template <typename T, int MM, bool GEN>
static kc_status group_launch(const GroupArgs<T>& a, cudaStream_t s) {
    const size_t smem = sizeof(double) * (MM * (MM + 1) / 2 + MM) + sizeof(T) * (MM * MM + MM) + 16 + 16 +
                        sizeof(unsigned long long) * ((size_t)1 << a.hbits) + sizeof(T) * (size_t)a.pmax * MM;
    auto kfn = ichol_group_k<T, MM, GEN, 0>;
    if constexpr (sizeof(T) == 4)
        if (a.lanes == 8) kfn = ichol_group_k<T, MM, GEN, 8>;  // (the FP64 form measured no gain)
    KC_TRY(allow_dynamic_smem(kfn));
    int per_sm = 0;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, BF_THREADS, smem));
    if (per_sm < 1) return fail(KC_EINVAL, "grouped factor: the prefix table exceeds an SM's shared memory");
    ::kc::note_launch(), kfn<<<sm_count() * per_sm, BF_THREADS, smem, s>>>(a);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

kc_status factor_blocked_impl(const kc_pattern* P, const double* x, int d, const kc_kernel* kern, int prec, void* val,
                              double* diag, int64_t* zero_out, const kc_opts* o, cudaStream_t s) {
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
    KernelParams kp;
    KC_TRY(kernel_params(kern, &kp));
    const int64_t N = P->N;
    // rows per task: about one task per resident CTA and dependency level, (nnz - N) / (depth x
    // resident CTAs), as the nearest power of two in 64..512 (longer tasks spread the prologue over
    // more rows; shorter ones keep the SMs busy on narrow levels)
    int rpt = 64;
    if (o && o->rows_per_task > 0) {
        rpt = o->rows_per_task;
    } else {
        const double per = (double)(P->nnz - N) / ((double)std::max(P->depth, 1) * sm_count() * KC_BLOCK_MINB);
        while (rpt < 512 && per >= rpt * 1.4142135623730951) rpt *= 2;
    }
    const long long spin = (o && o->spin_limit_cycles > 0) ? o->spin_limit_cycles : 4000000000LL;
    // lanes per row: at least the group size (lane u of a row's lanes
    // evaluates Theta for column g0 + u)
    int lanes = BF_MAXG;
    if (o && o->lanes_per_row > 0) {
        lanes = o->lanes_per_row;
        if (lanes > 32 || (lanes & (lanes - 1))) return fail(KC_EINVAL, "lanes_per_row must be a power of two <= 32");
        lanes = std::max(lanes, BF_MAXG);
    }
    Arena A(s);
    KC_TRY(upload_coef(kp, A, s));
    // groups
    int* same;
    int64_t *sflag, *incl, *start, *gex, *oflag, *fex, *cnt, *toff;
    int32_t *runstart, *gstart, *group_of, *gorder;
    KC_TRY(A.get(&same, N));
    KC_TRY(A.get(&sflag, N));
    KC_TRY(A.get(&incl, N + 1));
    KC_TRY(A.get(&runstart, N));
    KC_TRY(A.get(&start, N));
    KC_TRY(A.get(&gex, N + 1));
    KC_TRY(A.get(&gstart, N + 1));
    KC_TRY(A.get(&group_of, N));
    int64_t *nchunk, *choff;
    KC_TRY(A.get(&nchunk, N));
    KC_TRY(A.get(&choff, N + 1));
    ::kc::note_launch(), grp_same_k<<<blocks_for(N * 32, 256), 256, 0, s>>>(P->rowptr, P->col, P->colptr, P->rowidx, N,
                                                                             same, nchunk);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i64(nchunk, choff, N, A, s));
    ::kc::note_launch(), grp_same_long_k<<<sm_count() * 8, 256, 0, s>>>(P->rowptr, P->col, P->colptr, P->rowidx, N,
                                                                         choff, same);
    KC_CUDA(cudaGetLastError());
    // incl[a] = number of runs starting at or before a (exclusive scan of the
    // run-start flags, plus the flag)
    ::kc::note_launch(), grp_runflag_k<<<blocks_for(N, 256), 256, 0, s>>>(same, N, sflag);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i64(sflag, incl, N, A, s));
    ::kc::note_launch(), grp_inclusive_k<<<blocks_for(N, 256), 256, 0, s>>>(sflag, N, incl);
    KC_CUDA(cudaGetLastError());
    ::kc::note_launch(), grp_runstart_k<<<blocks_for(N, 256), 256, 0, s>>>(same, incl, N, runstart);
    ::kc::note_launch(), grp_start_k<<<blocks_for(N, 256), 256, 0, s>>>(incl, runstart, N, BF_MAXG, start);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i64(start, gex, N, A, s));
    ::kc::note_launch(), grp_ids_k<<<blocks_for(N, 256), 256, 0, s>>>(start, gex, N, gstart, group_of);
    KC_CUDA(cudaGetLastError());
    int64_t ng = 0;
    {
        int64_t last_ex = 0, last_flag = 0;
        KC_CUDA(cudaMemcpyAsync(&last_ex, gex + N - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaMemcpyAsync(&last_flag, start + N - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        ng = last_ex + last_flag;
    }
    const int32_t nn = (int32_t)N;
    KC_CUDA(cudaMemcpyAsync(gstart + ng, &nn, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    // tasks: the groups in the schedule's order of their first columns
    unsigned* done;
    int* pmax;
    KC_TRY(A.get(&oflag, N));
    KC_TRY(A.get(&fex, N + 1));
    KC_TRY(A.get(&gorder, ng));
    KC_TRY(A.get(&cnt, ng));
    KC_TRY(A.get(&toff, ng + 1));
    KC_TRY(A.get(&done, ng));
    KC_TRY(A.get(&pmax, 1));
    KC_CUDA(cudaMemsetAsync(pmax, 0, sizeof(int), s));
    ::kc::note_launch(), grp_orderflag_k<<<blocks_for(N, 256), 256, 0, s>>>(P->order, start, N, oflag);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i64(oflag, fex, N, A, s));
    ::kc::note_launch(), grp_tasks_count_k<<<blocks_for(N, 256), 256, 0, s>>>(
        P->order, oflag, fex, group_of, gstart, P->colptr, P->rowptr, N, rpt, gorder, cnt, done, pmax);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i64(cnt, toff, ng, A, s));
    int64_t nt = 0;
    int hp = 0;
    KC_CUDA(cudaMemcpyAsync(&nt, toff + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaMemcpyAsync(&hp, pmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    int2* tasks;
    KC_TRY(A.get(&tasks, nt));
    ::kc::note_launch(), grp_tasks_fill_k<<<blocks_for(ng * 32, 256), 256, 0, s>>>(gorder, toff, ng, tasks);
    KC_CUDA(cudaGetLastError());
    unsigned long long *ticket, *zp;
    int* status;
    KC_TRY(A.get(&ticket, 1));
    KC_TRY(A.get(&zp, 1));
    KC_TRY(A.get(&status, 1));
    KC_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s));
    KC_CUDA(cudaMemsetAsync(zp, 0, sizeof(unsigned long long), s));
    KC_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    int hb = 5;
    while (3 * (1 << hb) < 4 * std::max(hp, 1)) ++hb;  // load factor <= 3/4
    const int pm = std::max(hp, 1);
    cudaEvent_t e0, e1;
    KC_CUDA(cudaEventCreate(&e0));
    KC_CUDA(cudaEventCreate(&e1));
    KC_CUDA(cudaEventRecord(e0, s));
    kc_status st;
    const bool gen = kp.nu_code > 2;
    if (prec == KC_FP64) {
        GroupArgs<double> a{N, d, x, P->rowptr, P->col, P->colptr, P->rowidx, P->slot, gstart, group_of, tasks, nt, rpt,
                            (double*)val, diag, done, ticket, status, zp, kp, spin, hb, pm, lanes};
        st = gen ? group_launch<double, BF_MAXG, true>(a, s) : group_launch<double, BF_MAXG, false>(a, s);
    } else {
        GroupArgs<float> a{N, d, x, P->rowptr, P->col, P->colptr, P->rowidx, P->slot, gstart, group_of, tasks, nt, rpt,
                           (float*)val, diag, done, ticket, status, zp, kp, spin, hb, pm, lanes};
        st = gen ? group_launch<float, BF_MAXG, true>(a, s) : group_launch<float, BF_MAXG, false>(a, s);
    }
    if (st != KC_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
    }
    KC_CUDA(cudaEventRecord(e1, s));
    int h_status = 0;
    unsigned long long h_zp = 0;
    KC_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaMemcpyAsync(&h_zp, zp, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) set_factor_kernel_ms(ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (zero_out) *zero_out = (int64_t)h_zp;
    if (h_status == DEV_TIMEOUT) return fail(KC_ETIMEOUT, "grouped factor: a dependency wait ran out");
    if (h_status != 0) return fail(KC_ECUDA, "grouped factor: device status " + std::to_string(h_status));
    return KC_OK;
}

}  // namespace kc
