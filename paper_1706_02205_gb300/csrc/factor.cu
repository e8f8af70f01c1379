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
// warp that takes a task waits (bounded spin with backoff, acquire loads)
// until every column k in R_i has published all its tasks, puts row i
// (index -> value) into an open-addressing hash table in shared memory,
// recomputes the pivot, and then merges the prefix of each row j of its chunk
// (entries k < i) against the table.  The rows of the chunk go in batches of
// 32: each lane first fetches one row's bookkeeping and evaluates its
// Theta_ji from the coordinates (entries are never stored), then lanes form
// groups of G (one 32-byte sector of values per group load); a group owns one
// row, each lane walks the row with stride G, loading U (col, val) pairs
// ahead (the staging depth) so that enough loads are in flight to cover HBM
// latency; in the FP32 form each lane also prefetches into L2 one sector of
// the row its group takes next and one of its own row's second round, which
// the merges would otherwise request only after the round before them.  The
// task publishes by a release increment of done[i].
//
// A second form, on request, stages the row prefixes of a batch in shared
// memory with bulk (TMA) copies into two buffers per warp completing on
// mbarriers, and merges from there; each lane merges the same entries in the
// same order as in the first form, so both give the same bits.  On the GB300
// the per-copy cost of the bulk engine for prefixes of a few hundred bytes
// makes it the slower form, which is why loads into registers are the
// default.
//
// Several independent point sets can be factored in one launch: their
// patterns are concatenated block-diagonally and every column names its set,
// whose Matern parameters the kernel then uses.
//
// FP32 form: values, products and the compensated (Dot2) sums stay in FP32;
// only the pivot and its square root are FP64 (the FP64 pipe of the GB300 is
// a small fraction of its FP32 rate).  FP64 form: everything in FP64.
//
// Forward progress: a task only waits on columns of lower level, whose tasks
// have smaller ticket numbers and were claimed by running warps, so the
// earliest unfinished task can always proceed.  Every wait is bounded: when it
// runs out the kernel records DEV_TIMEOUT in the status word and returns.
#include <algorithm>
#include <vector>

#include "grid.cuh"
#include "ichol.cuh"

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
    KernelParams kp;                 // kernel of a single set
    const double* __restrict__ aval;  // given entries (ENT = 2): the matrix on the pattern, CSR layout
    const int32_t* __restrict__ col_set;  // set of every column (NULL: one set)
    const KernelParams* __restrict__ kps; // kernels of the sets
    long long spin_limit;
    int hold_col;
    int hbits;  // hash table of 2^hbits slots per warp
    int lanes;  // lanes per row, 0 = from |R_i|
    int adaptive;  // chunk of at least |R_i|/4 rows
    int warp_smem;    // shared-memory bytes of one warp (table, then the bulk form's buffers and barriers)
    int stage_bytes;  // bulk form: bytes of each of the two stage buffers
};

// Rows of column k handled by one task.  Adaptive (the factor): at least a
// quarter of |R_k|, because every task re-stages row k, so a long row should
// not be staged again for every few rows below it.
__device__ __forceinline__ int rows_of_task(const int64_t* __restrict__ rowptr, int k, int rpt, int adaptive) {
    if (!adaptive) return rpt;
    const int nr = (int)(rowptr[k + 1] - rowptr[k] - 1);
    return max(rpt, nr >> 2);
}
__device__ __forceinline__ unsigned n_tasks_of(const int64_t* __restrict__ colptr, const int64_t* __restrict__ rowptr,
                                               int k, int rpt, int adaptive) {
    const int64_t m = colptr[k + 1] - colptr[k] - 1;  // rows below the diagonal
    const int r = rows_of_task(rowptr, k, rpt, adaptive);
    return m <= 0 ? 1u : (unsigned)((m + r - 1) / r);
}

__device__ __forceinline__ int hslot(int k, int hbits) { return (int)(((unsigned)k * 2654435761u) >> (32 - hbits)); }

// Open-addressing table (linear probing) of one row i in shared memory: key
// k in R_i -> L_ik.  FP32: one 8-byte slot per key (key in the low word, the
// value's bits in the high word), so a probe is a single shared load.  FP64:
// an array of values followed by an array of keys.  Empty slots have key -1.
template <typename T>
struct RowTable;
template <>
struct RowTable<float> {
    unsigned long long* s;
    int hbits;  // 2^hbits slots
    __device__ __forceinline__ RowTable(unsigned char* base, int hb) : s((unsigned long long*)base), hbits(hb) {}
    __device__ __forceinline__ void clear(int lane) {
        uint4* q = (uint4*)s;
        for (int h = lane; h < (1 << (hbits - 1)); h += 32) q[h] = make_uint4(~0u, ~0u, ~0u, ~0u);
    }
    __device__ __forceinline__ void insert(int k, float v) {
        const int mask = (1 << hbits) - 1;
        const unsigned long long w = ((unsigned long long)__float_as_uint(v) << 32) | (unsigned)k;
        int h = hslot(k, hbits);
        while (atomicCAS(&s[h], ~0ull, w) != ~0ull) h = (h + 1) & mask;
    }
    __device__ __forceinline__ bool find(int k, float& v) const {
        const int mask = (1 << hbits) - 1;
        int h = hslot(k, hbits);
        for (;;) {
            const unsigned long long w = s[h];
            const int key = (int)(unsigned)w;
            if (key == k) {
                v = __uint_as_float((unsigned)(w >> 32));
                return true;
            }
            if (key < 0) return false;
            h = (h + 1) & mask;
        }
    }
};
template <>
struct RowTable<double> {
    double* val;
    int* key;
    int hbits;
    __device__ __forceinline__ RowTable(unsigned char* base, int hb)
        : val((double*)base), key((int*)(val + (1 << hb))), hbits(hb) {}
    __device__ __forceinline__ void clear(int lane) {
        int4* q = (int4*)key;
        for (int h = lane; h < (1 << (hbits - 2)); h += 32) q[h] = make_int4(-1, -1, -1, -1);
    }
    __device__ __forceinline__ void insert(int k, double v) {
        const int mask = (1 << hbits) - 1;
        int h = hslot(k, hbits);
        while (atomicCAS(&key[h], -1, k) != -1) h = (h + 1) & mask;
        val[h] = v;
    }
    __device__ __forceinline__ bool find(int k, double& v) const {
        const int mask = (1 << hbits) - 1;
        int h = hslot(k, hbits);
        for (;;) {
            const int x = key[h];
            if (x == k) {
                v = val[h];
                return true;
            }
            if (x < 0) return false;
            h = (h + 1) & mask;
        }
    }
};

__device__ __forceinline__ int64_t bsearch_glob(const int32_t* __restrict__ a, int64_t lo, int64_t hi, int k) {
    int64_t end = hi;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(&a[mid]) < k) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && __ldg(&a[lo]) == k) ? lo : -1;
}

// Matern parameters of column i's set, read where they are used (not kept in
// registers through the merges).
template <typename T>
__device__ __forceinline__ const KernelParams& kparams(const FactorArgs<T>& A, int i) {
    return A.col_set ? A.kps[A.col_set[i]] : A.kp;
}

// Everything a task knows after its prologue.
template <typename T>
struct TaskCtx {
    int i, c, nr;
    int64_t a0, a1;  // R_i = col[a0..a1), L_ii at a1
    bool zero;       // dropped pivot: the whole column is zero
    bool staged;     // row i is in the table (else binary search in global memory)
    double Lii;
    T inv;
};

// Claim the next task and run its prologue: wait until every column k in
// R_i is complete, put row i into the table, form the pivot in FP64.
// Returns 0 (task ready), 1 (no tasks left), 2 (stop: a wait ran out or the
// kernel is stopping).
template <typename T, int ENT>
__device__ __forceinline__ int task_begin(const FactorArgs<T>& A, RowTable<T>& tab, int lane, TaskCtx<T>& X) {
    const unsigned FULL = 0xffffffffu;
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(A.ticket, 1ULL);
    t = __shfl_sync(FULL, t, 0);
    if ((int64_t)t >= A.ntasks) return 1;
    if (ld_volatile_s32(A.status) != 0) return 2;
    const int2 tk = A.tasks[t];
    X.i = tk.x;
    X.c = tk.y;
    X.a0 = A.rowptr[X.i];
    X.a1 = A.rowptr[X.i + 1] - 1;
    X.nr = (int)(X.a1 - X.a0);

    X.staged = 4 * X.nr <= 3 * (1 << A.hbits);  // load factor <= 3/4 (linear probing stays short)
    if (X.staged) tab.clear(lane);
    __syncwarp();
    // R_i in rounds of DEPS entries per lane: the column indices, the completion
    // counters of those columns (relaxed loads, all in flight together; a
    // bounded spin only on columns not yet complete), one acquire fence, then
    // the values into the table and the sum of squares (the accumulator of the
    // merges: FP32 form compensated, its two parts added in FP64 below).  Each
    // lane reads only the values of the columns it checked itself; the other
    // lanes' columns are ordered by the warp barrier at the end.
    constexpr int DEPS = 8;
    Acc<T> sq;
    for (int e0 = 0; e0 < X.nr; e0 += 32 * DEPS) {
        int kk[DEPS];
#pragma unroll
        for (int u = 0; u < DEPS; ++u) {
            const int e = e0 + lane + 32 * u;
            kk[u] = e < X.nr ? __ldg(&A.col[X.a0 + e]) : -1;
        }
        unsigned pend = 0;
#pragma unroll
        for (int u = 0; u < DEPS; ++u)
            if (kk[u] >= 0 && (int)ld_relaxed_u32(&A.done[kk[u]]) < 0) pend |= 1u << u;
        bool ok = true;
#pragma unroll
        for (int u = 0; u < DEPS; ++u)
            if (ok && ((pend >> u) & 1u)) ok = spin_done(&A.done[kk[u]], A.status, A.spin_limit);
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
            return 2;
        }
        fence_acq_rel_gpu();  // acquire: the columns' values are visible from here on
        T vv[DEPS];
#pragma unroll
        for (int u = 0; u < DEPS; ++u) vv[u] = kk[u] >= 0 ? ldcg(&A.val[X.a0 + e0 + lane + 32 * u]) : (T)0;
#pragma unroll
        for (int u = 0; u < DEPS; ++u)
            if (kk[u] >= 0) {
                if (X.staged) tab.insert(kk[u], vv[u]);
                sq.add(vv[u], vv[u]);
            }
    }
    sq.group_reduce(32);
    // Lane 0 forms the pivot and every lane takes its values: one pivot for the
    // whole task whichever lane writes a row (after a butterfly the partners'
    // compensations c + (c2 + e) and c2 + (c + e) may round apart), and the FP64
    // work runs on one lane.
    double Lii = 0.0;
    T inv = (T)0;
    int zero = 0;
    if (lane == 0) {
        double thii;
        if constexpr (ENT == 2) {
            thii = A.aval[X.a1];
        } else {
            const KernelParams& kp = kparams(A, X.i);
            thii = kp.sigma2 + kp.nugget;
        }
        const double p = thii - sq.total();
        zero = !(p > 0.0);
        Lii = zero ? 0.0 : sqrt(p);
        inv = zero ? (T)0 : Acc<T>::recip(Lii);
        if (X.c == 0) {
            A.val[X.a1] = (T)Lii;
            A.diag[X.i] = Lii;
            if (zero) atomicAdd(A.zero_piv, 1ULL);
        }
    }
    X.Lii = __shfl_sync(FULL, Lii, 0);
    X.inv = __shfl_sync(FULL, inv, 0);
    X.zero = __shfl_sync(FULL, zero, 0) != 0;
    __syncwarp();  // the table's inserts are visible to every lane
    return 0;
}

// Publish one finished task of column i.
template <typename T>
__device__ __forceinline__ void task_end(const FactorArgs<T>& A, int i, int lane) {
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0 && i != A.hold_col) red_release_add_u32(&A.done[i], 1u);
}

// Lanes per row: one 32-byte sector of values per group load (8 lanes in
// FP32, 4 in FP64), unless set.
template <typename T>
__device__ __forceinline__ int lanes_per_row(int lanes) {
    return lanes > 0 ? lanes : (int)(32 / sizeof(T));
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Merge of the prefix [es, be) of row j, read from global memory, against
// row i: U (col, val) pairs per lane in flight; the ragged end is masked.
// PF (long rows): each full round also prefetches into L2 the round after
// the next, which the loads would otherwise request one round late.
template <typename T, int U, int PF = 0>
__device__ __forceinline__ void merge_global(const FactorArgs<T>& A, const RowTable<T>& tab, const TaskCtx<T>& X,
                                             int64_t es, int64_t be, int sub, int G, Acc<T>& acc) {
    if (X.staged) {
        const int n = (int)(be - es);
        const int32_t* cp = A.col + es;
        const T* vp = A.val + es;
        int t = sub;
        for (; t + (U - 1) * G < n; t += U * G) {  // full rounds
            int k[U];
            T wv[U];
            if constexpr (PF) {
                constexpr int SEC = 32 / (int)sizeof(T);
                const int base2 = t - sub + 2 * U * G;
#pragma unroll
                for (int h = 0; h < U / SEC; ++h) {  // U*G entries = U/SEC sectors per lane
                    const int e2 = base2 + (h * G + sub) * SEC;
                    if (e2 < n) {
                        prefetch_l2(cp + e2);
                        prefetch_l2(vp + e2);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) k[u] = __ldg(cp + t + u * G);
#pragma unroll
            for (int u = 0; u < U; ++u) wv[u] = ldcg(vp + t + u * G);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                T hv;
                if (tab.find(k[u], hv)) acc.add(wv[u], hv);
            }
        }
        if (t < n) {  // the ragged end: one masked round
            int k[U];
            T wv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) k[u] = t + u * G < n ? __ldg(cp + t + u * G) : -1;
#pragma unroll
            for (int u = 0; u < U; ++u) wv[u] = t + u * G < n ? ldcg(vp + t + u * G) : (T)0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                T hv;
                if (k[u] >= 0 && tab.find(k[u], hv)) acc.add(wv[u], hv);
            }
        }
    } else {
        for (int64_t e = es + sub; e < be; e += G) {
            const int64_t pos = bsearch_glob(A.col, X.a0, X.a1, __ldg(&A.col[e]));
            if (pos >= 0) acc.add(ldcg(&A.val[e]), ldcg(&A.val[pos]));
        }
    }
}

// Row-j bookkeeping of the rows b0+lane of a batch: the slot of L_ji, the
// start of row j, and Theta_ji (loads and exponentials overlap across lanes).
template <typename T, int ENT>
__device__ __forceinline__ void batch_rows(const FactorArgs<T>& A, const TaskCtx<T>& X, int64_t b0, int nb, int lane,
                                           int64_t& my_e0, int64_t& my_b, T& my_th) {
    my_e0 = 0;
    my_b = 0;
    my_th = (T)0;
    if (lane < nb) {
        const int j = __ldg(&A.rowidx[b0 + lane]);
        my_b = __ldg(&A.slot[b0 + lane]);
        my_e0 = __ldg(&A.rowptr[j]);
        if constexpr (ENT == 2) {
            if (!X.zero) my_th = (T)__ldg(&A.aval[my_b]);
        } else {
            if (!X.zero)
                my_th = theta_off<T, ENT == 1>(kparams(A, X.i), A.d, A.x + (int64_t)j * A.d,
                                               A.x + (int64_t)X.i * A.d);
        }
    }
}

// ----------------------------------------------------------- register form
// Each lane keeps U (col, val) loads of its row prefix in flight in registers.
// Resident CTAs of 8 warps per SM that the register budget is cut for.
#ifndef KC_FACTOR_MIN_BLOCKS
#define KC_FACTOR_MIN_BLOCKS 4
#endif

// GC > 0: lanes per row fixed at compile time (the default for the FP32 form:
// the group loads' offsets become constants); 0: from A.lanes.  PF: the
// merges prefetch two rounds ahead (patterns with long rows).
template <typename T, int U, int ENT, int GC, int PF>
__global__ void __launch_bounds__(256, U >= 16 ? 3 : KC_FACTOR_MIN_BLOCKS) ichol_persistent_k(FactorArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    RowTable<T> tab(smem + (size_t)w * A.warp_smem, A.hbits);
    const unsigned FULL = 0xffffffffu;
    TaskCtx<T> X;
    for (;;) {
        if (task_begin<T, ENT>(A, tab, lane, X) != 0) return;
        const int G = GC > 0 ? GC : lanes_per_row<T>(A.lanes);
        const int ng = 32 / G, g = lane / G, sub = lane % G;
        const int rows = rows_of_task(A.rowptr, X.i, A.rpt, A.adaptive);
        const int64_t qs = A.colptr[X.i] + 1 + (int64_t)X.c * rows;
        const int64_t qe = min(A.colptr[X.i + 1], qs + rows);
        for (int64_t b0 = qs; b0 < qe; b0 += 32) {
            const int nb = (int)min((int64_t)32, qe - b0);
            int64_t my_e0, my_b;
            T my_th;
            batch_rows<T, ENT>(A, X, b0, nb, lane, my_e0, my_b, my_th);
            for (int r0 = 0; r0 < nb; r0 += ng) {
                const int r = r0 + g;
                const bool act = r < nb;
                const int src = act ? r : 0;
                const int64_t es = __shfl_sync(FULL, my_e0, src);
                const int64_t be = __shfl_sync(FULL, my_b, src);  // L_ji lives at be; the prefix is [es, be)
                const T th = __shfl_sync(FULL, my_th, src);
                if constexpr (GC > 0) {
                    // L2 prefetches that the merges below do not wait for: one sector per lane of the
                    // group's row in the next round of rows (its first U*G entries), and of this row past
                    // its first U*G entries (the second round, issued otherwise only after the first)
                    constexpr int SEC = 32 / (int)sizeof(T);
                    const int rn = r + ng;
                    const bool pn = rn < nb && !X.zero;
                    const int64_t esn = __shfl_sync(FULL, my_e0, pn ? rn : 0);
                    const int64_t ben = __shfl_sync(FULL, my_b, pn ? rn : 0);
                    const int64_t en = esn + sub * SEC, ec = es + U * G + sub * SEC;
                    if (pn && en < ben) {
                        prefetch_l2(A.col + en);
                        prefetch_l2(A.val + en);
                    }
                    if (act && !X.zero && ec < be) {
                        prefetch_l2(A.col + ec);
                        prefetch_l2(A.val + ec);
                    }
                }
                Acc<T> acc;
                if (act && !X.zero) merge_global<T, U, PF>(A, tab, X, es, be, sub, G, acc);
                acc.group_reduce(G);
                if (act && sub == 0) A.val[be] = X.zero ? (T)0 : acc.finish(th, X.Lii, X.inv);
            }
        }
        task_end(A, X.i, lane);
    }
}

// --------------------------------------------------------------- bulk form
// The prefixes of a stage of consecutive rows are copied from global memory
// into one of two shared-memory buffers of the warp by the bulk-copy (TMA)
// engine, completing on an mbarrier; the warp merges the previous stage from
// shared memory meanwhile.  The loads in flight then cost no registers, so a
// few warps per SM keep enough bytes in flight.  Each row's (col, val)
// extents are widened to 16-byte boundaries (a bulk copy's rule); a row that
// alone exceeds a buffer is merged from global memory instead.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// A stage: rows [s0, s1) of the current batch, in buffer `buf`; `direct`: one
// row merged from global memory; `bytes`: the buffer's barrier is armed.
struct Stage {
    int s0, s1, buf;
    bool direct, bytes;
};

// Issue the copies of the next stage starting at row c0 of the batch into
// buffer bi.  Each lane owns row lane of the batch: it sizes its widened
// extents, a warp scan places them, and the rows that fit are copied.
// my_off / my_meta receive the position of the lane's row in the buffer.
template <typename T>
__device__ __forceinline__ Stage stage_issue(const FactorArgs<T>& A, unsigned char* buf, uint64_t* bar, int bi,
                                             int c0, int nb, int lane, int64_t my_e0, int64_t my_b,
                                             uint32_t& my_off, uint32_t& my_meta) {
    const unsigned FULL = 0xffffffffu;
    uint32_t sz = 0, colB = 0, hc = 0, hv = 0;
    uintptr_t cl = 0, vl = 0;
    const bool mine = lane >= c0 && lane < nb;
    if (mine && my_b > my_e0) {
        const uintptr_t ca = (uintptr_t)(A.col + my_e0), ce = (uintptr_t)(A.col + my_b);
        const uintptr_t va = (uintptr_t)(A.val + my_e0), ve = (uintptr_t)(A.val + my_b);
        cl = ca & ~(uintptr_t)15;
        vl = va & ~(uintptr_t)15;
        colB = (uint32_t)(((ce + 15) & ~(uintptr_t)15) - cl);
        sz = colB + (uint32_t)(((ve + 15) & ~(uintptr_t)15) - vl);
        hc = (uint32_t)((ca - cl) >> 2);
        hv = (uint32_t)((va - vl) / sizeof(T));
    }
    uint32_t inc = sz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += n;
    }
    const bool fits = mine && inc <= (uint32_t)A.stage_bytes;
    const int cnt = __popc(__ballot_sync(FULL, fits));  // rows c0 .. c0+cnt-1: the scan is monotone
    Stage S;
    S.s0 = c0;
    S.buf = bi;
    if (cnt == 0) {
        S.s1 = c0 + 1;
        S.direct = true;
        S.bytes = false;
        return S;
    }
    S.s1 = c0 + cnt;
    S.direct = false;
    const uint32_t total = __shfl_sync(FULL, inc, c0 + cnt - 1);
    S.bytes = total > 0;
    if (fits) {
        my_off = inc - sz;
        my_meta = colB | (hc << 24) | (hv << 28);
    }
    if (S.bytes) {
        // the buffer's previous contents were read by this warp's generic loads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (lane == 0) mbar_expect(bar, total);
        __syncwarp();
        if (fits && sz > 0) {
            bulk_copy(buf + (inc - sz), (const void*)cl, colB, bar);
            bulk_copy(buf + (inc - sz) + colB, (const void*)vl, sz - colB, bar);
        }
    }
    return S;
}

// Merge of a prefix of n entries held in shared memory.
template <typename T, int U>
__device__ __forceinline__ void merge_smem(const RowTable<T>& tab, const int* cs, const T* vs, int n, int sub, int G,
                                           Acc<T>& acc) {
    for (int t = sub; t < n; t += U * G) {
        int k[U];
        T wv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = t + u * G;
            k[u] = q < n ? cs[q] : -1;
            wv[u] = q < n ? vs[q] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            T hv;
            if (k[u] >= 0 && tab.find(k[u], hv)) acc.add(wv[u], hv);
        }
    }
}

template <typename T, int U, int ENT>
__global__ void __launch_bounds__(128) ichol_bulk_k(FactorArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = lane_id();
    const int w = threadIdx.x >> 5;
    unsigned char* base = smem + (size_t)w * A.warp_smem;
    const int H = 1 << A.hbits;
    RowTable<T> tab(base, A.hbits);
    unsigned char* bufs = base + (size_t)H * (sizeof(int) + sizeof(T));
    uint64_t* bars = (uint64_t*)(bufs + 2 * (size_t)A.stage_bytes);
    const unsigned FULL = 0xffffffffu;
    if (lane == 0) {
        mbar_init(&bars[0]);
        mbar_init(&bars[1]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
    uint32_t phase = 0;  // bit b: parity of the next phase of barrier b
    TaskCtx<T> X;
    for (;;) {
        if (task_begin<T, ENT>(A, tab, lane, X) != 0) return;
        // values of finished columns were written by other SMs through the generic
        // proxy and acquired above; the bulk copies read them through the async proxy
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const int G = lanes_per_row<T>(A.lanes);
        const int ng = 32 / G, g = lane / G, sub = lane % G;
        const int rows = rows_of_task(A.rowptr, X.i, A.rpt, A.adaptive);
        const int64_t qs = A.colptr[X.i] + 1 + (int64_t)X.c * rows;
        const int64_t qe = min(A.colptr[X.i + 1], qs + rows);
        const bool bulk = X.staged && !X.zero;
        for (int64_t b0 = qs; b0 < qe; b0 += 32) {
            const int nb = (int)min((int64_t)32, qe - b0);
            int64_t my_e0, my_b;
            T my_th;
            batch_rows<T, ENT>(A, X, b0, nb, lane, my_e0, my_b, my_th);
            uint32_t off0 = 0, meta0 = 0, off1 = 0, meta1 = 0;  // the lane's row in buffer 0 / 1
            Stage cur;
            if (bulk) cur = stage_issue(A, bufs, &bars[0], 0, 0, nb, lane, my_e0, my_b, off0, meta0);
            else cur = Stage{0, nb, 0, true, false};
            while (cur.s0 < nb) {
                Stage nxt{nb, nb, 0, true, false};
                if (bulk && cur.s1 < nb) {
                    if (cur.buf == 0)
                        nxt = stage_issue(A, bufs + A.stage_bytes, &bars[1], 1, cur.s1, nb, lane, my_e0, my_b, off1,
                                          meta1);
                    else
                        nxt = stage_issue(A, bufs, &bars[0], 0, cur.s1, nb, lane, my_e0, my_b, off0, meta0);
                }
                if (cur.bytes) {
                    const bool ok = mbar_wait(&bars[cur.buf], (phase >> cur.buf) & 1u, A.spin_limit);
                    phase ^= 1u << cur.buf;
                    if (!__all_sync(FULL, ok)) {
                        // give the copies still in flight a bounded chance to land, then stop
                        if (nxt.bytes) mbar_wait(&bars[nxt.buf], (phase >> nxt.buf) & 1u, A.spin_limit);
                        if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
                        return;
                    }
                }
                const unsigned char* sb = bufs + (size_t)cur.buf * A.stage_bytes;
                const uint32_t my_off = cur.buf ? off1 : off0, my_meta = cur.buf ? meta1 : meta0;
                for (int r0 = cur.s0; r0 < cur.s1; r0 += ng) {
                    const int r = r0 + g;
                    const bool act = r < cur.s1;
                    const int src = act ? r : cur.s0;
                    const int64_t es = __shfl_sync(FULL, my_e0, src);
                    const int64_t be = __shfl_sync(FULL, my_b, src);
                    const T th = __shfl_sync(FULL, my_th, src);
                    const uint32_t ro = __shfl_sync(FULL, my_off, src);
                    const uint32_t rm = __shfl_sync(FULL, my_meta, src);
                    Acc<T> acc;
                    if (act && !X.zero) {
                        if (cur.direct) {
                            merge_global<T, U>(A, tab, X, es, be, sub, G, acc);
                        } else {
                            const uint32_t colB = rm & 0xffffffu;
                            const int* cs = (const int*)(sb + ro) + (rm >> 24 & 15u);
                            const T* vs = (const T*)(sb + ro + colB) + (rm >> 28);
                            merge_smem<T, U>(tab, cs, vs, (int)(be - es), sub, G, acc);
                        }
                    }
                    acc.group_reduce(G);
                    if (act && sub == 0) A.val[be] = X.zero ? (T)0 : acc.finish(th, X.Lii, X.inv);
                }
                __syncwarp();
                cur = nxt;
            }
        }
        task_end(A, X.i, lane);
    }
}

// done[k] = -(tasks of column k), as an unsigned word
__global__ void done_init_k(const int64_t* __restrict__ colptr, const int64_t* __restrict__ rowptr, int64_t N, int rpt,
                            int adaptive, unsigned* __restrict__ done) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) done[k] = 0u - n_tasks_of(colptr, rowptr, (int)k, rpt, adaptive);
}

// tasks of column order[p]: n_tasks_of(order[p])
__global__ void task_count_k(const int32_t* __restrict__ order, const int64_t* __restrict__ colptr,
                             const int64_t* __restrict__ rowptr, int64_t N, int rpt, int adaptive,
                             int64_t* __restrict__ cnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) cnt[p] = n_tasks_of(colptr, rowptr, order[p], rpt, adaptive);
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

// Build the task list of a pattern (its columns in the schedule's order:
// by level, within a level in space-filling-curve order when the schedule was
// given the points, so that consecutive tasks merge rows of neighbouring
// points, which share most of their entries); returns the count on the host.
kc_status build_tasks(const kc_pattern* P, int rpt, Arena& A, cudaStream_t s, int2** tasks_out, int64_t* ntasks_out,
                      int* max_row_out, bool adaptive) {
    int64_t N = P->N;
    int64_t* cnt;
    int64_t* toff;
    int* mr;
    KC_TRY(A.get(&cnt, N));
    KC_TRY(A.get(&toff, N + 1));
    KC_TRY(A.get(&mr, 1));
    const int32_t* order = P->order;
    ::kc::note_launch(), task_count_k<<<blocks_for(N, 256), 256, 0, s>>>(order, P->colptr, P->rowptr, N, rpt,
                                                                            adaptive ? 1 : 0, cnt);
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
    ::kc::note_launch(), task_fill_k<<<blocks_for(N * 32, 256), 256, 0, s>>>(order, toff, N, tasks);
    KC_CUDA(cudaGetLastError());
    *tasks_out = tasks;
    *ntasks_out = nt;
    *max_row_out = hmr;
    return KC_OK;
}

// ---------------------------------------------------------------- launch core
// Everything one persistent launch needs.  kc_factor fills it with
// stream-ordered scratch; a kc_factor_plan keeps it across launches.
struct FactorCore {
    kc_pattern P;
    int prec = KC_FP32_FORM;
    int d = 2;
    const double* x = nullptr;
    int2* tasks = nullptr;
    int64_t ntasks = 0;
    int maxr = 0;
    unsigned* done = nullptr;
    unsigned long long* ticket = nullptr;
    unsigned long long* zp = nullptr;
    int* status = nullptr;
    KernelParams kp{};
    const int32_t* col_set = nullptr;
    KernelParams* kps = nullptr;
    bool general = false;  // some set's kernel is not a closed-form Matern
    const double* aval = nullptr;  // given entries (kc_factor_given)
    int rpt = 128, lanes = 0, unroll = 8, warps = 8, hbits = 7, ctas = 0, adaptive = 0;
    int stage_req = 0;    // requested stage-buffer bytes: 0 automatic, < 0 register form
    int stage_bytes = 0;  // chosen (0: register form)
    int bulk_warps = 4;
    bool warps_auto = true;  // register form: CTA size from the occupancy of the row tables
    long long spin = 4000000000LL;
    int hold = -1;
};

template <typename T, int U, int ENT>
static kc_status launch_core(const FactorCore& F, T* val, double* diag, cudaStream_t s) {
    FactorArgs<T> a;
    a.N = F.P.N;
    a.d = F.d;
    a.x = F.x;
    a.rowptr = F.P.rowptr;
    a.col = F.P.col;
    a.colptr = F.P.colptr;
    a.rowidx = F.P.rowidx;
    a.slot = F.P.slot;
    a.tasks = F.tasks;
    a.ntasks = F.ntasks;
    a.rpt = F.rpt;
    a.val = val;
    a.diag = diag;
    a.done = F.done;
    a.ticket = F.ticket;
    a.status = F.status;
    a.zero_piv = F.zp;
    a.kp = F.kp;
    a.aval = F.aval;
    a.col_set = F.col_set;
    a.kps = F.kps;
    a.spin_limit = F.spin;
    a.hold_col = F.hold;
    a.hbits = F.hbits;
    a.lanes = F.lanes;
    a.adaptive = F.adaptive;
    a.stage_bytes = F.stage_bytes;
    const size_t table = (size_t)(1 << F.hbits) * (sizeof(int) + sizeof(T));
    const bool bulk = ENT == 0 && F.stage_bytes > 0;  // the other entry sources: register form
    // bulk form: table, two stage buffers, two mbarriers per warp (128-byte aligned)
    a.warp_smem = (int)(bulk ? (table + 2 * (size_t)F.stage_bytes + 16 + 127) / 128 * 128 : table);
    int warps = bulk ? F.bulk_warps : F.warps;
    if (bulk) {
        int dev = 0, optin = 0;
        KC_CUDA(cudaGetDevice(&dev));
        KC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        warps = std::min(warps, optin / a.warp_smem);
        if (warps < 1) return fail(KC_EINVAL, "factor: stage_bytes too large for one warp's shared memory");
    }
    // FP32 form with 8 lanes per row (the default, or chosen by a plan's tuner): the lanes at compile time
    const bool g8 = sizeof(T) == 4 && (F.lanes == 0 || F.lanes == 8);
    auto kfn = ichol_persistent_k<T, U, ENT, 0, 0>;
    if constexpr (sizeof(T) == 4)
        if (g8) kfn = ichol_persistent_k<T, U, ENT, 8, 0>;
    if constexpr (ENT == 0)
        if (F.P.nnz >= 400 * F.P.N) {  // long rows (the 3-D workloads): prefetch two rounds ahead
            if constexpr (sizeof(T) == 4) kfn = g8 ? ichol_persistent_k<T, U, 0, 8, 1> : ichol_persistent_k<T, U, 0, 0, 1>;
            else kfn = ichol_persistent_k<T, U, 0, 0, 1>;
        }
    if constexpr (ENT == 0)
        if (bulk) kfn = ichol_bulk_k<T, U, 0>;
    int per_sm = 0;
    KC_TRY(allow_dynamic_smem(kfn));
    if (!bulk && F.warps_auto) {
        // CTA size with the most resident warps: a large row table (long rows)
        // fits one 8-warp CTA per SM where several smaller CTAs fit more warps.
        // A smaller CTA must win by over 20%: filling the shared memory to the
        // last CTA leaves the L1 cache (which the column index loads use) too small.
        int best = 0;
        for (int w = 8; w >= 1; w >>= 1) {
            const size_t sm_w = (size_t)w * a.warp_smem;
            int n = 0;
            KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kfn, w * 32, sm_w));
            if (n * w * 5 > best * 6) {
                best = n * w;
                warps = w;
            }
        }
    }
    const size_t smem = (size_t)warps * a.warp_smem;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, warps * 32, smem));
    if (F.ctas > 0 && F.ctas < per_sm) per_sm = F.ctas;
    if (F.ctas < 0) per_sm = std::max(1, per_sm + F.ctas);  // leave -ctas CTA slots per SM to other streams
    if (per_sm < 1) return fail(KC_EINVAL, "factor: shared memory of one CTA exceeds the SM (stage_bytes too large?)");
    ::kc::note_launch(), done_init_k<<<blocks_for(F.P.N, 256), 256, 0, s>>>(F.P.colptr, F.P.rowptr, F.P.N, F.rpt,
                                                                           F.adaptive, F.done);
    KC_CUDA(cudaMemsetAsync(F.ticket, 0, sizeof(unsigned long long), s));
    KC_CUDA(cudaMemsetAsync(F.zp, 0, sizeof(unsigned long long), s));
    KC_CUDA(cudaMemsetAsync(F.status, 0, sizeof(int), s));
    ::kc::note_launch(), kfn<<<sm_count() * per_sm, warps * 32, smem, s>>>(a);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// The closed-form Matern kernels take the unroll asked for; the other entry
// sources one instantiation per precision (register form, 8 loads in flight
// per lane in the FP32 form, 4 in FP64).
static kc_status launch_any(const FactorCore& F, void* val, double* diag, cudaStream_t s) {
    if (F.aval)
        return F.prec == KC_FP64 ? launch_core<double, 4, 2>(F, (double*)val, diag, s)
                                 : launch_core<float, 8, 2>(F, (float*)val, diag, s);
    if (F.general)
        return F.prec == KC_FP64 ? launch_core<double, 4, 1>(F, (double*)val, diag, s)
                                 : launch_core<float, 8, 1>(F, (float*)val, diag, s);
    if (F.prec == KC_FP64)
        return F.unroll >= 8 ? launch_core<double, 8, 0>(F, (double*)val, diag, s)
                             : launch_core<double, 4, 0>(F, (double*)val, diag, s);
    if (F.unroll >= 16) return launch_core<float, 16, 0>(F, (float*)val, diag, s);
    return F.unroll >= 8 ? launch_core<float, 8, 0>(F, (float*)val, diag, s)
                         : launch_core<float, 4, 0>(F, (float*)val, diag, s);
}

static kc_status read_status(const FactorCore& F, int64_t* zero_out, cudaStream_t s) {
    int h_status = 0;
    unsigned long long h_zp = 0;
    KC_CUDA(cudaMemcpyAsync(&h_status, F.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaMemcpyAsync(&h_zp, F.zp, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (zero_out) *zero_out = (int64_t)h_zp;
    if (h_status == DEV_TIMEOUT) return fail(KC_ETIMEOUT, "factor: a dependency wait ran out");
    if (h_status != 0) return fail(KC_ECUDA, "factor: device status " + std::to_string(h_status));
    return KC_OK;
}

static kc_status apply_opts(FactorCore& F, const kc_opts* o) {
    F.rpt = (o && o->rows_per_task > 0) ? o->rows_per_task : 0;  // 0: from the level width (auto_rows)
    F.warps = (o && o->warps_per_cta > 0) ? o->warps_per_cta : 8;
    F.warps_auto = !(o && o->warps_per_cta > 0);
    if (F.warps > 8) return fail(KC_EINVAL, "warps_per_cta must be <= 8");
    F.spin = (o && o->spin_limit_cycles > 0) ? o->spin_limit_cycles : 4000000000LL;
    F.ctas = o ? o->ctas_per_sm : 0;
    F.hold = (o && o->test_hold_column > 0) ? o->test_hold_column - 1 : -1;
    F.lanes = 0;
    if (o && o->lanes_per_row > 0) {
        int L = o->lanes_per_row;
        if (L > 32 || (L & (L - 1))) return fail(KC_EINVAL, "lanes_per_row must be a power of two <= 32");
        F.lanes = L;
    }
    F.unroll = (o && o->unroll > 0) ? o->unroll : 0;  // 0: from the mean row length (pick_hash)
    F.stage_req = o ? o->stage_bytes : 0;
    if (F.stage_req > 65536) return fail(KC_EINVAL, "stage_bytes must be <= 65536");
    F.adaptive = (o && o->adaptive_chunks) ? 1 : 0;
    if (F.unroll != 0 && F.unroll != 4 && F.unroll != 8 && F.unroll != 16)
        return fail(KC_EINVAL, "unroll must be 4, 8 or 16");
    return KC_OK;
}

static void pick_hash(FactorCore& F) {
    // hash table: 4/3 of the longest row at least (load factor <= 3/4), a power
    // of two in 128..2048 slots; a longer row falls back to binary search in
    // global memory
    int hb = 7;
    while (hb < 11 && 3 * (1 << hb) < 4 * F.maxr) ++hb;
    F.hbits = hb;
    // staging depth: 16 loads per lane in flight for long rows (FP32 form),
    // else 8; the FP64 form takes at most 8
    if (F.unroll == 0) F.unroll = F.prec == KC_FP64 ? 4 : (F.P.nnz >= 400 * F.P.N ? 16 : 8);
    // bulk form (on request): stage buffers of the requested size; a row
    // prefix longer than a buffer is merged from global memory
    F.stage_bytes = F.stage_req <= 0 ? 0 : std::max(64, (F.stage_req + 15) / 16 * 16);
    F.bulk_warps = F.warps < 4 ? F.warps : 4;
}

// Rows per task, unless set: about one task per resident warp per level,
// (nnz - N) / (depth * warps), as a power of two in 16..128.  Smaller tasks
// keep narrow levels busy; larger ones stage each pivot row fewer times.
static void auto_rows(FactorCore& F) {
    if (F.rpt > 0) return;
    const double warps = (double)sm_count() * 32.0;
    const double per = (double)(F.P.nnz - F.P.N) / ((double)std::max(1, F.P.depth) * warps);
    int r = 16;
    while (r < 128 && per > r * 1.41421356) r <<= 1;
    F.rpt = r;
}

// One factorisation: entries from the covariance function kern at the
// points x, or (kern NULL) the given matrix aval on the pattern.
static kc_status factor_run(const kc_pattern* P, const double* x, int d, const kc_kernel* kern, const double* aval,
                            int prec, void* val, double* diag, int64_t* zero_out, const kc_opts* o, cudaStream_t s) {
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
    FactorCore F;
    if (kern) {
        KC_TRY(kernel_params(kern, &F.kp));
        F.general = F.kp.nu_code > 2;
    } else {
        F.aval = aval;
    }
    KC_TRY(apply_opts(F, o));
    F.P = *P;
    F.prec = prec;
    F.d = d;
    F.x = x;
    auto_rows(F);
    Arena A(s);
    KC_TRY(upload_coef(F.kp, A, s));
    KC_TRY(build_tasks(P, F.rpt, A, s, &F.tasks, &F.ntasks, &F.maxr, F.adaptive != 0));
    pick_hash(F);
    KC_TRY(A.get(&F.done, P->N));
    KC_TRY(A.get(&F.ticket, 1));
    KC_TRY(A.get(&F.zp, 1));
    KC_TRY(A.get(&F.status, 1));
    cudaEvent_t e0, e1;
    KC_CUDA(cudaEventCreate(&e0));
    KC_CUDA(cudaEventCreate(&e1));
    KC_CUDA(cudaEventRecord(e0, s));
    kc_status st = launch_any(F, val, diag, s);
    if (st != KC_OK) return st;
    KC_CUDA(cudaEventRecord(e1, s));
    st = read_status(F, zero_out, s);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) set_factor_kernel_ms(ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

kc_status factor_impl(const kc_pattern* P, const double* x, int d, const kc_kernel* kern, int prec, void* val,
                      double* diag, int64_t* zero_out, const kc_opts* o, cudaStream_t s) {
    return factor_run(P, x, d, kern, nullptr, prec, val, diag, zero_out, o, s);
}

kc_status factor_given_impl(const kc_pattern* P, const double* aval, int prec, void* val, double* diag,
                            int64_t* zero_out, const kc_opts* o, cudaStream_t s) {
    return factor_run(P, nullptr, 0, nullptr, aval, prec, val, diag, zero_out, o, s);
}

}  // namespace kc

// ------------------------------------------------------------------ plans
// A plan keeps the task list and the counters of one pattern so that the
// factorisation is a single capturable launch (no allocation, no host sync).
struct kc_factor_plan {
    kc::FactorCore F;
    std::vector<void*> owned;
};

namespace kc {

static kc_status plan_alloc(kc_factor_plan* pl, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(plan)");
    pl->owned.push_back(*p);
    return KC_OK;
}

kc_status plan_create_impl(const kc_pattern* P, const double* x, int d, const kc_kernel* kerns, int nsets,
                           const int32_t* col_set, int prec, const kc_opts* o, kc_factor_plan** out, cudaStream_t s) {
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
    if (nsets < 1 || (nsets > 1 && !col_set)) return fail(KC_EINVAL, "nsets >= 1; col_set required when nsets > 1");
    kc_factor_plan* pl = new kc_factor_plan();
    FactorCore& F = pl->F;
    auto bail = [&](kc_status st) {
        for (void* p : pl->owned) cudaFree(p);
        delete pl;
        return st;
    };
    kc_status st = kernel_params(&kerns[0], &F.kp);
    if (st == KC_OK) st = apply_opts(F, o);
    if (st != KC_OK) return bail(st);
    F.general = F.kp.nu_code > 2;
    F.P = *P;
    F.prec = prec;
    F.d = d;
    F.x = x;
    F.col_set = nsets > 1 ? col_set : nullptr;
    auto_rows(F);
    {
        Arena A(s);
        int2* t;
        st = build_tasks(P, F.rpt, A, s, &t, &F.ntasks, &F.maxr, F.adaptive != 0);
        if (st != KC_OK) return bail(st);
        if ((st = plan_alloc(pl, (void**)&F.tasks, sizeof(int2) * F.ntasks)) != KC_OK) return bail(st);
        if (cudaMemcpyAsync(F.tasks, t, sizeof(int2) * F.ntasks, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return bail(fail(KC_ECUDA, "plan: task copy"));
    }
    pick_hash(F);
    if ((st = plan_alloc(pl, (void**)&F.done, sizeof(unsigned) * P->N)) != KC_OK) return bail(st);
    if ((st = plan_alloc(pl, (void**)&F.ticket, 64)) != KC_OK) return bail(st);
    if ((st = plan_alloc(pl, (void**)&F.zp, 64)) != KC_OK) return bail(st);
    if ((st = plan_alloc(pl, (void**)&F.status, 64)) != KC_OK) return bail(st);
    if (F.kp.nu_code == 3) {
        double* tab;
        if ((st = plan_alloc(pl, (void**)&tab, sizeof(double) * KC_COEF_LEN)) != KC_OK) return bail(st);
        if ((st = upload_coef(F.kp, tab, s)) != KC_OK) return bail(st);
    }
    if (nsets > 1) {
        std::vector<KernelParams> h(nsets);
        for (int k = 0; k < nsets; ++k) {
            if ((st = kernel_params(&kerns[k], &h[k])) != KC_OK) return bail(st);
            if (h[k].nu_code > 2) F.general = true;
            if (h[k].nu_code == 3) {
                double* tab;
                if ((st = plan_alloc(pl, (void**)&tab, sizeof(double) * KC_COEF_LEN)) != KC_OK) return bail(st);
                if ((st = upload_coef(h[k], tab, s)) != KC_OK) return bail(st);
            }
        }
        if ((st = plan_alloc(pl, (void**)&F.kps, sizeof(KernelParams) * nsets)) != KC_OK) return bail(st);
        if (cudaMemcpy(F.kps, h.data(), sizeof(KernelParams) * nsets, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(KC_ECUDA, "plan: kernel parameter copy"));
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(KC_ECUDA, "plan: synchronize"));
    *out = pl;
    return KC_OK;
}

kc_status plan_launch_impl(kc_factor_plan* pl, void* val, double* diag, cudaStream_t s) {
    return launch_any(pl->F, val, diag, s);
}

kc_status plan_finish_impl(kc_factor_plan* pl, int64_t* zero_out, cudaStream_t s) {
    return read_status(pl->F, zero_out, s);
}

// Pick lanes per row (the warp share of one row) and the staging depth by
// timing every combination once on the plan's own problem.
kc_status plan_tune_impl(kc_factor_plan* pl, void* val, double* diag, int32_t* lanes_out, int32_t* unroll_out,
                         double* best_ms_out, cudaStream_t s) {
    FactorCore& F = pl->F;
    const int lanes_c[] = {2, 4, 8, 16};
    const int unroll_c[] = {8, 16};
    cudaEvent_t e0, e1;
    KC_CUDA(cudaEventCreate(&e0));
    KC_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    int bl = F.lanes, bu = F.unroll;
    KC_TRY(launch_any(F, val, diag, s));  // warm-up
    KC_TRY(read_status(F, nullptr, s));
    for (int L : lanes_c)
        for (int U : unroll_c) {
            F.lanes = L;
            F.unroll = U;
            KC_CUDA(cudaEventRecord(e0, s));
            KC_TRY(launch_any(F, val, diag, s));
            KC_CUDA(cudaEventRecord(e1, s));
            KC_TRY(read_status(F, nullptr, s));
            float ms = 0.f;
            KC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                bl = L;
                bu = U;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    F.lanes = bl;
    F.unroll = bu;
    if (lanes_out) *lanes_out = bl;
    if (unroll_out) *unroll_out = bu;
    if (best_ms_out) *best_ms_out = best;
    return KC_OK;
}

void plan_destroy_impl(kc_factor_plan* pl) {
    if (!pl) return;
    for (void* p : pl->owned) cudaFree(p);
    delete pl;
}

}  // namespace kc
