// a7: L L^T x = b with the sparse factor (task (2) of Section 1), as two
// sync-free level-scheduled triangular solves in one persistent launch each.
//
// Forward  L y = b:   y_j = (b_j - sum_{k in R_j} L_jk y_k) / L_jj, one warp per
//                     row, rows in (level, index) order; row j waits for the
//                     ready flags of its R_j.
// Backward L^T x = y: x_i = (y_i - sum_{j in C_i} L_ji x_j) / L_ii, over the
//                     CSC columns in reverse level order; wide columns are cut
//                     into chunks of rows, each chunk stores its partial sums
//                     in a slot of its own; the last chunk to finish of every
//                     group of 32 adds its group's slots, and the last group
//                     of a column to finish adds the group sums and finishes
//                     x_i.  Every sum runs in a fixed order across the lanes
//                     of a warp, so every result repeats bit for bit.
//
// Vectors are point-major inside with a power-of-two stride NR >= nrhs
// (v[k * NR + r]), so one point's right-hand sides are one aligned run that a
// lane gathers with 16-byte loads.  A lane owns entries of the row (or rows of
// the column): the readiness checks go out as relaxed loads all at once (a
// bounded spin only on points not yet solved, then one acquire fence), the
// values and the gathers follow in a few rounds, and the warp reduces its NR
// partial sums with a reduce-scatter.  A dropped pivot (L_ii = 0) uses
// sqrt(Theta_ii).
//
// Arithmetic.  FP64 form: vectors, products and sums in FP64.  FP32 form (L in
// FP32): the GB300's FP64 pipe is a small fraction of its FP32 rate, so the
// vectors are kept as pairs of floats (hi, lo) with hi + lo the FP64 value to
// about 2^-48, every product L_jk (hi + lo) is formed with TwoProduct (fmaf)
// plus the small L_jk lo term, and the sums are compensated (TwoSum, the
// scheme of Ogita, Rump and Oishi's Dot2); each row's result is formed in
// FP64 and split back into a pair.  The solution is about 2^-45 accurate
// relative to the sums' magnitudes, where FP64 gives 2^-53.
#include <type_traits>

#include "pairs.cuh"
#include "solver.cuh"

namespace kc {

// Right-hand sides a lane of the FP32-form kernels keeps (an entry's NR are
// split over NR / KC_SOLVE_NRL lanes), and the resident 256-thread CTAs per
// SM their register budget is cut for.
#ifndef KC_SOLVE_NRL
#define KC_SOLVE_NRL 8
#endif
#ifndef KC_SOLVE_MINB
#define KC_SOLVE_MINB 3
#endif

// Longest back-off (ns) between two polls of a readiness flag.
#ifndef KC_SOLVE_BACKOFF_MAX
#define KC_SOLVE_BACKOFF_MAX 512
#endif

template <typename T>
struct SolveArgs {
    int64_t N;
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
    double* y;        // point-major output of the forward solve / input of backward (FP64 form)
    double* x;        // point-major output of the backward solve
    float2* yf;       // FP32 form: y as (hi, lo) pairs
    float2* xf;       // FP32 form: x as (hi, lo) pairs (gathered by later columns; x above gets FP64)
    double* acc;      // partial sums of the chunks of wide columns: NR per task, at the task's index
    unsigned* cnt;    // finished chunk groups per column (backward)
    unsigned* gcnt;   // finished chunks per group of 32, at the group's first task
    int* ready;       // per point flag
    unsigned long long* ticket;
    int* status;
    long long spin_limit;
};

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// bounded wait (backoff) on a point not yet solved; false when the budget ran
// out or the kernel is stopping
__device__ __forceinline__ bool spin_flag(const int* f, const int* status, long long limit) {
    const long long t0 = clock64();
    unsigned ns = 32;
    while (ld_relaxed_s32(f) == 0) {
        if (clock64() - t0 > limit || ld_volatile_s32(status) != 0) return false;
        __nanosleep(ns);  // back off so waiting warps do not flood L2 with polls
        if (ns < KC_SOLVE_BACKOFF_MAX) ns <<= 1;
    }
    return true;
}

// Loads of a point's vector values, which other SMs write during the launch.
// When one point's values fill whole 128-byte lines by themselves (LINE =
// bytes per point = 128, i.e. 16 right-hand sides), no SM can read a line of
// point k before k's ready flag is set, after its values were written, so the
// line may be cached in L1 (KC_SOLVE_GATHER_L1); coarse points are gathered by
// nearly every row.  Otherwise lines are shared by neighbouring points and the
// loads go to L2.
#ifndef KC_SOLVE_GATHER_L1
#define KC_SOLVE_GATHER_L1 1
#endif
template <int LINE, typename V>
__device__ __forceinline__ V ld_vec(const V* p) {
    if constexpr (KC_SOLVE_GATHER_L1 && LINE == 128) return __ldca(p);
    else return __ldcg(p);
}

// The NR values of point k (16-byte loads).
template <int NR>
__device__ __forceinline__ void gather(const double* v, int k, double* out) {
    if constexpr (NR == 1) {
        out[0] = __ldcg(v + k);
    } else {
        const double2* p = (const double2*)(v + (int64_t)k * NR);
#pragma unroll
        for (int q = 0; q < NR / 2; ++q) {
            const double2 w = ld_vec<NR * 8>(p + q);
            out[2 * q] = w.x;
            out[2 * q + 1] = w.y;
        }
    }
}

// Warp reduce-scatter of NR partial sums per lane: each level halves the
// values a lane keeps (offsets 16, 8, ...), plain sums finish the rest.  The
// lane ends with the full sum of right-hand side rhs_of_lane<NR>(lane).
template <int NR>
__device__ __forceinline__ double reduce_scatter(double (&v)[NR], int lane) {
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int h = NR / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < h; ++q) {
            const double send = up ? v[q] : v[q + h];
            const double keep = up ? v[q + h] : v[q];
            v[q] = keep + __shfl_xor_sync(FULL, send, o);
        }
    }
    constexpr int L = NR == 1 ? 0 : NR == 2 ? 1 : NR == 4 ? 2 : NR == 8 ? 3 : 4;
#pragma unroll
    for (int o = 16 >> L; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(FULL, v[0], o);
    return v[0];
}
template <int NR>
__device__ __forceinline__ int rhs_of_lane(int lane) {
    int r = 0;
#pragma unroll
    for (int h = NR / 2, o = 16; h >= 1; h >>= 1, o >>= 1)
        if (lane & o) r += h;
    return r;
}
// one writer per right-hand side: the lanes sharing r differ in the low bits
template <int NR>
__device__ __forceinline__ bool rhs_writer(int lane) {
    return (lane & (32 / NR - 1)) == 0;
}

// Entries in flight per lane while gathering: at most 32 doubles.
template <int NR>
struct Depth {
    static constexpr int E = NR >= 4 ? 32 / NR : 8;
};

// Readiness of the points kk[0..D) (negative: none): relaxed loads together,
// bounded spins on the rest, one acquire fence.  False: a wait ran out.
template <int D>
__device__ __forceinline__ bool points_ready(const int* ready, const int (&kk)[D], const int* status, long long lim) {
    unsigned pend = 0;
#pragma unroll
    for (int u = 0; u < D; ++u)
        if (kk[u] >= 0 && ld_relaxed_s32(&ready[kk[u]]) == 0) pend |= 1u << u;
    bool ok = true;
#pragma unroll
    for (int u = 0; u < D; ++u)
        if (ok && ((pend >> u) & 1u)) ok = spin_flag(&ready[kk[u]], status, lim);
    ok = __all_sync(0xffffffffu, ok);
    fence_acq_rel_gpu();  // acquire: the points' values are visible from here on
    return ok;
}

// acc[r] += w[u] * v[k[u] * NR + r] for the D entries, E gathers at a time
template <int NR, int D>
__device__ __forceinline__ void gather_fma(const double* v, const int (&k)[D], const double (&w)[D],
                                           double (&acc)[NR]) {
    constexpr int E = Depth<NR>::E < D ? Depth<NR>::E : D;
#pragma unroll
    for (int u0 = 0; u0 < D; u0 += E) {
        double g[E][NR];
#pragma unroll
        for (int q = 0; q < E; ++q) {
            if (k[u0 + q] >= 0) gather<NR>(v, k[u0 + q], g[q]);
            else
#pragma unroll
                for (int r = 0; r < NR; ++r) g[q][r] = 0.0;
        }
#pragma unroll
        for (int q = 0; q < E; ++q)
            if (k[u0 + q] >= 0)  // the FP64 pipe is scarce: no products for empty slots
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] = fma(w[u0 + q], g[q][r], acc[r]);
    }
}

// Publish a solved point: the warp's writes of its values, then its ready
// flag with release semantics (KC_SOLVE_PUB_FENCE: with a fence of every lane
// before the warp barrier as well).
#ifndef KC_SOLVE_PUB_FENCE
#define KC_SOLVE_PUB_FENCE 1
#endif
__device__ __forceinline__ void publish_ready(int* f, int lane) {
#if KC_SOLVE_PUB_FENCE
    fence_acq_rel_gpu();
#endif
    __syncwarp();
    if (lane == 0) st_release_s32(f, 1);
}

// Sum over cnt slots of NR doubles (slot p0, p0 + stride, ...) in a fixed
// order: lane l takes right-hand side l % NR and every (32 / NR)-th slot from
// l / NR on; the lanes of one right-hand side then add their sums by a fixed
// butterfly.  Every lane returns the total of right-hand side lane % NR.
template <int NR>
__device__ __forceinline__ double combine_slots(const double* part, int64_t p0, int64_t stride, int cnt, int lane) {
    constexpr int LP = 32 / NR;
    const int r = lane % NR;
    double s = 0.0;
    for (int k = lane / NR; k < cnt; k += LP) s += __ldcg(&part[(p0 + (int64_t)k * stride) * NR + r]);
#pragma unroll
    for (int o = 16; o >= NR; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// A chunk c of column i (task index ti, nch > 1 chunks) with its partial sums
// already in its slot: counts it in its group of 32 chunks; the group's last
// chunk adds the group's slots and leaves the sum in the group's first slot;
// the column's last group adds the group sums.  Returns true (and the total
// of right-hand side lane % NR in `total`) when this warp finishes column i.
template <int NR>
__device__ __forceinline__ bool combine_chunks(double* part, unsigned* gcnt, unsigned* cnt, int i, int64_t ti, int c,
                                               unsigned nch, int lane, double& total) {
    const unsigned FULL = 0xffffffffu;
    const int64_t base = ti - c;
    const int g = c >> 5, ng = (int)((nch + 31) >> 5);
    const int gsz = (int)min(32u, nch - 32u * (unsigned)g);
    unsigned prev = 0;
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0) prev = atomicAdd(&gcnt[base + 32 * g], 1u);
    prev = __shfl_sync(FULL, prev, 0);
    if ((int)prev != gsz - 1) return false;
    fence_acq_rel_gpu();  // acquire: the group's slots are visible
    double gs = combine_slots<NR>(part, base + 32 * g, 1, gsz, lane);
    if (ng == 1) {
        total = gs;
        return true;
    }
    if (lane < NR) part[(base + 32 * g) * NR + lane] = gs;
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0) prev = atomicAdd(&cnt[i], 1u);
    prev = __shfl_sync(FULL, prev, 0);
    if ((int)prev != ng - 1) return false;
    fence_acq_rel_gpu();
    total = combine_slots<NR>(part, base, 32, ng, lane);
    return true;
}

template <typename T, int NR>
__global__ void __launch_bounds__(256) fwd_solve_k(SolveArgs<T> A) {
    constexpr int D = 8;  // entries of R_j per lane per round
    const int lane = lane_id();
    const unsigned FULL = 0xffffffffu;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(A.ticket, 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= A.N) return;
        if (ld_volatile_s32(A.status) != 0) return;
        const int j = A.order[t];
        const int64_t a = A.rowptr[j];
        const int n = (int)(A.rowptr[j + 1] - 1 - a);
        double acc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = 0.0;
        for (int e0 = 0; e0 < n; e0 += 32 * D) {
            int kk[D];
#pragma unroll
            for (int u = 0; u < D; ++u) {
                const int e = e0 + lane + 32 * u;
                kk[u] = e < n ? __ldg(&A.col[a + e]) : -1;
            }
            double w[D];  // static data: loaded before the wait
#pragma unroll
            for (int u = 0; u < D; ++u) w[u] = kk[u] >= 0 ? (double)__ldg(&A.val[a + e0 + lane + 32 * u]) : 0.0;
            if (!points_ready<D>(A.ready, kk, A.status, A.spin_limit)) {
                if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
                return;
            }
            gather_fma<NR, D>(A.y, kk, w, acc);
        }
        const double s = reduce_scatter<NR>(acc, lane);
        if (rhs_writer<NR>(lane)) {
            const int r = rhs_of_lane<NR>(lane);
            double dj = A.diag[j];
            if (!(dj > 0.0)) dj = A.diag_fallback;
            A.y[(int64_t)j * NR + r] = (A.b[(int64_t)j * NR + r] - s) / dj;
        }
        publish_ready(&A.ready[j], lane);
    }
}

template <typename T, int NR>
__global__ void __launch_bounds__(256) bwd_solve_k(SolveArgs<T> A) {
    constexpr int D = 4;  // rows of the chunk per lane per round
    const int lane = lane_id();
    const unsigned FULL = 0xffffffffu;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(A.ticket, 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= A.ntasks) return;
        if (ld_volatile_s32(A.status) != 0) return;
        const int64_t ti = A.ntasks - 1 - (int64_t)t;
        const int2 tk = A.tasks[ti];
        const int i = tk.x, c = tk.y;
        const int64_t c0 = A.colptr[i], c1 = A.colptr[i + 1];
        const int64_t m = c1 - c0 - 1;
        const unsigned nch = m <= 0 ? 1u : (unsigned)((m + A.rpt - 1) / A.rpt);
        const int64_t qs = c0 + 1 + (int64_t)c * A.rpt;
        const int nq = (int)(min(c1, qs + A.rpt) - qs);
        double acc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = 0.0;
        for (int q0 = 0; q0 < nq; q0 += 32 * D) {
            int jj[D];
            int64_t pp[D];
#pragma unroll
            for (int u = 0; u < D; ++u) {
                const int q = q0 + lane + 32 * u;
                jj[u] = q < nq ? __ldg(&A.rowidx[qs + q]) : -1;
                pp[u] = q < nq ? __ldg(&A.slot[qs + q]) : 0;
            }
            double w[D];  // static data: loaded before the wait
#pragma unroll
            for (int u = 0; u < D; ++u) w[u] = jj[u] >= 0 ? (double)__ldg(&A.val[pp[u]]) : 0.0;
            if (!points_ready<D>(A.ready, jj, A.status, A.spin_limit)) {
                if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
                return;
            }
            gather_fma<NR, D>(A.x, jj, w, acc);
        }
        double s = reduce_scatter<NR>(acc, lane);
        bool wr = rhs_writer<NR>(lane);
        int r = rhs_of_lane<NR>(lane);
        bool finish = true;
        if (nch > 1) {
            if (wr) A.acc[ti * NR + r] = s;
            finish = combine_chunks<NR>(A.acc, A.gcnt, A.cnt, i, ti, c, nch, lane, s);
            wr = lane < NR;  // the combined sums: right-hand side lane % NR
            r = lane % NR;
        }
        if (finish) {
            if (wr) {
                double di = A.diag[i];
                if (!(di > 0.0)) di = A.diag_fallback;
                A.x[(int64_t)i * NR + r] = (A.y[(int64_t)i * NR + r] - s) / di;
            }
            publish_ready(&A.ready[i], lane);
        }
    }
}

// ------------------------------------------------ FP32 form: float pairs
// Lane layout of the pair kernels: an entry's NR right-hand sides are split
// over P lanes of NRL each (NR = 16: two lanes of 8; else one lane), so a lane
// keeps NRL compensated sums and gathers NRL pairs per entry: half the
// registers of one lane per entry at NR = 16, hence twice the resident warps.
template <int NR>
struct PairLayout {
    static constexpr int NRL = NR > KC_SOLVE_NRL ? KC_SOLVE_NRL : NR;  // right-hand sides per lane
    static constexpr int P = NR / NRL;           // lanes per entry (1 or 2)
    static constexpr int SLOTS = 32 / P;         // entries per warp and round
    static constexpr int L = NRL == 1 ? 0 : NRL == 2 ? 1 : NRL == 4 ? 2 : 3;  // halving levels
};

// Reduce-scatter of the NRL (s, c) pairs over the lanes holding the same block
// of right-hand sides (offsets 16, 8, ... down to P); returns the FP64 sum of
// right-hand side pair_rhs<NR>(lane).
template <int NR>
__device__ __forceinline__ double reduce_scatter_pair(float (&s)[PairLayout<NR>::NRL],
                                                      float (&c)[PairLayout<NR>::NRL], int lane) {
    using PL = PairLayout<NR>;
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int h = PL::NRL / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < h; ++q) {
            const float ss = up ? s[q] : s[q + h], sc = up ? c[q] : c[q + h];
            const float ks = up ? s[q + h] : s[q], kc = up ? c[q + h] : c[q];
            const float rs = __shfl_xor_sync(FULL, ss, o), rc = __shfl_xor_sync(FULL, sc, o);
            s[q] = ks;
            c[q] = kc;
            pair_merge(s[q], c[q], rs, rc);
        }
    }
#pragma unroll
    for (int o = 16 >> PL::L; o >= PL::P; o >>= 1) {
        const float rs = __shfl_xor_sync(FULL, s[0], o), rc = __shfl_xor_sync(FULL, c[0], o);
        pair_merge(s[0], c[0], rs, rc);
    }
    return (double)s[0] + (double)c[0];
}
template <int NR>
__device__ __forceinline__ int pair_rhs(int lane) {
    using PL = PairLayout<NR>;
    int r = (lane & (PL::P - 1)) * PL::NRL;
#pragma unroll
    for (int h = PL::NRL / 2, o = 16; h >= 1; h >>= 1, o >>= 1)
        if (lane & o) r += h;
    return r;
}
// one writer per right-hand side: the lanes sharing one differ only in the
// bits between the block bits and the halving bits
template <int NR>
__device__ __forceinline__ bool pair_writer(int lane) {
    using PL = PairLayout<NR>;
    return (lane & ((32 >> PL::L) - 1) & ~(PL::P - 1)) == 0;
}

// (s, c)[r] += w[u] * v[k[u]][block + r], E gathers at a time, nothing for empty slots
template <int NR, int D>
__device__ __forceinline__ void gather_pair_add(const float2* v, const int (&k)[D], const float (&w)[D], int block,
                                                float (&s)[PairLayout<NR>::NRL], float (&c)[PairLayout<NR>::NRL]) {
    constexpr int NRL = PairLayout<NR>::NRL;
    constexpr int E0 = NRL >= 2 ? 16 / NRL : 8;  // at most 16 pairs in flight per lane
    constexpr int E = E0 < D ? E0 : D;
#pragma unroll
    for (int u0 = 0; u0 < D; u0 += E) {
        float hi[E][NRL], lo[E][NRL];
#pragma unroll
        for (int q = 0; q < E; ++q)
            if (k[u0 + q] >= 0) {
                const float2* p = v + (int64_t)k[u0 + q] * NR + block;
                if constexpr (NRL == 1) {
                    const float2 x = __ldcg(p);
                    hi[q][0] = x.x;
                    lo[q][0] = x.y;
                } else {
#pragma unroll
                    for (int m = 0; m < NRL / 2; ++m) {
                        const float4 x = ld_vec<NR * 8>((const float4*)p + m);
                        hi[q][2 * m] = x.x;
                        lo[q][2 * m] = x.y;
                        hi[q][2 * m + 1] = x.z;
                        lo[q][2 * m + 1] = x.w;
                    }
                }
            }
#pragma unroll
        for (int q = 0; q < E; ++q)
            if (k[u0 + q] >= 0)
#pragma unroll
                for (int r = 0; r < NRL; ++r) pair_add(s[r], c[r], w[u0 + q], hi[q][r], lo[q][r]);
    }
}

template <int NR>
__global__ void __launch_bounds__(256, KC_SOLVE_MINB) fwd_solve_pair_k(SolveArgs<float> A) {
    using PL = PairLayout<NR>;
    constexpr int D = PL::NRL >= 8 ? 6 : 8;  // entries per lane and round (within 80 registers)
    const int lane = lane_id();
    const int el = lane / PL::P, block = (lane & (PL::P - 1)) * PL::NRL;
    const unsigned FULL = 0xffffffffu;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(A.ticket, 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= A.N) return;
        if (ld_volatile_s32(A.status) != 0) return;
        const int j = A.order[t];
        const int64_t a = A.rowptr[j];
        const int n = (int)(A.rowptr[j + 1] - 1 - a);
        float s[PL::NRL], c[PL::NRL];
#pragma unroll
        for (int r = 0; r < PL::NRL; ++r) s[r] = c[r] = 0.f;
        for (int e0 = 0; e0 < n; e0 += PL::SLOTS * D) {
            int kk[D];
            float w[D];  // static data: loaded before the wait
#pragma unroll
            for (int u = 0; u < D; ++u) {
                const int e = e0 + el + PL::SLOTS * u;
                kk[u] = e < n ? __ldg(&A.col[a + e]) : -1;
                w[u] = e < n ? __ldg(&A.val[a + e]) : 0.f;
            }
            if (!points_ready<D>(A.ready, kk, A.status, A.spin_limit)) {
                if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
                return;
            }
            gather_pair_add<NR, D>(A.yf, kk, w, block, s, c);
        }
        const double sum = reduce_scatter_pair<NR>(s, c, lane);
        if (pair_writer<NR>(lane)) {
            const int r = pair_rhs<NR>(lane);
            double dj = A.diag[j];
            if (!(dj > 0.0)) dj = A.diag_fallback;
            A.yf[(int64_t)j * NR + r] = pair_of((A.b[(int64_t)j * NR + r] - sum) / dj);
        }
        publish_ready(&A.ready[j], lane);
    }
}

template <int NR>
__global__ void __launch_bounds__(256, KC_SOLVE_MINB) bwd_solve_pair_k(SolveArgs<float> A) {
    using PL = PairLayout<NR>;
    constexpr int D = 4;
    const int lane = lane_id();
    const int el = lane / PL::P, block = (lane & (PL::P - 1)) * PL::NRL;
    const unsigned FULL = 0xffffffffu;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(A.ticket, 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= A.ntasks) return;
        if (ld_volatile_s32(A.status) != 0) return;
        const int64_t ti = A.ntasks - 1 - (int64_t)t;
        const int2 tk = A.tasks[ti];
        const int i = tk.x, ch = tk.y;
        const int64_t c0 = A.colptr[i], c1 = A.colptr[i + 1];
        const int64_t m = c1 - c0 - 1;
        const unsigned nch = m <= 0 ? 1u : (unsigned)((m + A.rpt - 1) / A.rpt);
        const int64_t qs = c0 + 1 + (int64_t)ch * A.rpt;
        const int nq = (int)(min(c1, qs + A.rpt) - qs);
        float s[PL::NRL], c[PL::NRL];
#pragma unroll
        for (int r = 0; r < PL::NRL; ++r) s[r] = c[r] = 0.f;
        for (int q0 = 0; q0 < nq; q0 += PL::SLOTS * D) {
            int jj[D];
            float w[D];  // static data: loaded before the wait
#pragma unroll
            for (int u = 0; u < D; ++u) {
                const int q = q0 + el + PL::SLOTS * u;
                jj[u] = q < nq ? __ldg(&A.rowidx[qs + q]) : -1;
                w[u] = q < nq ? __ldg(&A.val[__ldg(&A.slot[qs + q])]) : 0.f;
            }
            if (!points_ready<D>(A.ready, jj, A.status, A.spin_limit)) {
                if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
                return;
            }
            gather_pair_add<NR, D>(A.xf, jj, w, block, s, c);
        }
        double sum = reduce_scatter_pair<NR>(s, c, lane);
        bool wr = pair_writer<NR>(lane);
        int r = pair_rhs<NR>(lane);
        bool finish = true;
        if (nch > 1) {
            if (wr) A.acc[ti * NR + r] = sum;
            finish = combine_chunks<NR>(A.acc, A.gcnt, A.cnt, i, ti, ch, nch, lane, sum);
            wr = lane < NR;  // the combined sums: right-hand side lane % NR
            r = lane % NR;
        }
        if (finish) {
            if (wr) {
                double di = A.diag[i];
                if (!(di > 0.0)) di = A.diag_fallback;
                const double xi = (value_of(A.yf[(int64_t)i * NR + r]) - sum) / di;
                A.xf[(int64_t)i * NR + r] = pair_of(xi);
                A.x[(int64_t)i * NR + r] = xi;
            }
            publish_ready(&A.ready[i], lane);
        }
    }
}

// out[k * stride + r] = b[r * N + perm[k]] for r < nrhs, 0 for nrhs <= r < stride
__global__ void to_point_major_k(const double* __restrict__ b, const int32_t* __restrict__ perm, int64_t N, int nrhs,
                                 int stride, double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * stride) {
        int64_t k = t / stride;
        int r = (int)(t % stride);
        out[t] = r < nrhs ? b[(int64_t)r * N + perm[k]] : 0.0;
    }
}
__global__ void from_point_major_k(const double* __restrict__ xp, const int32_t* __restrict__ perm, int64_t N,
                                   int nrhs, int stride, double* __restrict__ x) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * nrhs) {
        int64_t k = t / nrhs;
        int r = (int)(t % nrhs);
        x[(int64_t)r * N + perm[k]] = xp[k * stride + r];
    }
}

// Rows of a column per backward-solve task (wider columns are cut into chunks
// whose sums the column's last chunk adds in chunk order).
#ifndef KC_SOLVE_ROWS
#define KC_SOLVE_ROWS 128
#endif

kc_status solver_init(Solver& S, const kc_pattern* P, int nrhs_cap, const kc_opts* o, Arena& A, cudaStream_t s) {
    S.P = P;
    S.rpt = (o && o->rows_per_task > 0) ? o->rows_per_task : KC_SOLVE_ROWS;
    if (o && o->spin_limit_cycles > 0) S.spin = o->spin_limit_cycles;
    KC_TRY(build_tasks(P, S.rpt, A, s, &S.tasks, &S.ntasks, &S.maxr));
    S.nrhs_cap = nrhs_cap;
    KC_TRY(A.get(&S.ready, P->N));
    KC_TRY(A.get(&S.cnt, P->N));
    KC_TRY(A.get(&S.acc, S.ntasks * nrhs_cap));
    KC_TRY(A.get(&S.gcnt, S.ntasks));
    KC_TRY(A.get(&S.ticket, 2));
    KC_TRY(A.get(&S.status, 1));
    KC_TRY(A.get(&S.y, P->N * nrhs_cap));
    KC_TRY(A.get(&S.xf, P->N * nrhs_cap));
    return KC_OK;
}

// z = (L L^T)^{-1} rhs, point-major, positions order.  Does not synchronise;
// the status word is checked by solver_check.
template <typename T, int NR>
static kc_status solve_launch(Solver& S, SolveArgs<T> a, int nrhs, cudaStream_t s) {
    const kc_pattern* P = S.P;
    const int grid = sm_count() * 8;
    KC_CUDA(cudaMemsetAsync(S.ready, 0, sizeof(int) * P->N, s));
    KC_CUDA(cudaMemsetAsync(S.ticket, 0, 2 * sizeof(unsigned long long), s));
    KC_CUDA(cudaMemsetAsync(S.status, 0, sizeof(int), s));
    a.ticket = S.ticket;
    if constexpr (std::is_same<T, float>::value) ::kc::note_launch(), fwd_solve_pair_k<NR><<<grid, 256, 0, s>>>(a);
    else ::kc::note_launch(), fwd_solve_k<T, NR><<<grid, 256, 0, s>>>(a);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaMemsetAsync(S.ready, 0, sizeof(int) * P->N, s));
    KC_CUDA(cudaMemsetAsync(S.cnt, 0, sizeof(unsigned) * P->N, s));
    KC_CUDA(cudaMemsetAsync(S.gcnt, 0, sizeof(unsigned) * S.ntasks, s));
    a.ticket = S.ticket + 1;
    if constexpr (std::is_same<T, float>::value) ::kc::note_launch(), bwd_solve_pair_k<NR><<<grid, 256, 0, s>>>(a);
    else ::kc::note_launch(), bwd_solve_k<T, NR><<<grid, 256, 0, s>>>(a);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

template <typename T>
static SolveArgs<T> solve_args(Solver& S, const T* val, const double* diag, double diag_fallback, const double* rhs,
                               double* z);

// z = (L L^T)^{-1} rhs, point-major with stride nrhs (a power of two <= 16),
// positions order.  Does not synchronise; the status word is checked by
// solver_check.
template <typename T>
kc_status solver_apply(Solver& S, const T* val, const double* diag, double diag_fallback, const double* rhs,
                       double* z, int nrhs, cudaStream_t s) {
    if (nrhs < 1 || nrhs > 16 || (nrhs & (nrhs - 1)) || nrhs > S.nrhs_cap)
        return fail(KC_EINVAL, "internal: solver stride must be a power of two <= 16");
    SolveArgs<T> a = solve_args<T>(S, val, diag, diag_fallback, rhs, z);
    switch (nrhs) {
        case 1: return solve_launch<T, 1>(S, a, nrhs, s);
        case 2: return solve_launch<T, 2>(S, a, nrhs, s);
        case 4: return solve_launch<T, 4>(S, a, nrhs, s);
        case 8: return solve_launch<T, 8>(S, a, nrhs, s);
        default: return solve_launch<T, 16>(S, a, nrhs, s);
    }
}

template <typename T>
static SolveArgs<T> solve_args(Solver& S, const T* val, const double* diag, double diag_fallback, const double* rhs,
                               double* z) {
    const kc_pattern* P = S.P;
    SolveArgs<T> a;
    a.N = P->N;
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
    a.yf = (float2*)S.y;  // same bytes as the FP64 vector
    a.xf = S.xf;
    a.acc = S.acc;
    a.cnt = S.cnt;
    a.gcnt = S.gcnt;
    a.ready = S.ready;
    a.status = S.status;
    a.spin_limit = S.spin;
    return a;
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

// The permutations between original-order right-hand sides b[r*N + i] and
// point-major vectors in position order v[k*stride + r] (perm[k] = i), by
// tiles of 32 points in original order: the rows of b are read and written
// coalesced, and each point's stride values form one line (128 bytes at
// stride 16) written or read whole; the inverse permutation is formed first.
constexpr int PM_WARPS = 8;
// pos starts at -1; an index outside 0..N-1 is ignored, and a point without a
// position is skipped by the tiled kernels (no access outside the arrays for
// a perm that is not a permutation)
__global__ void pm_inverse_perm_k(const int32_t* __restrict__ perm, int64_t N, int32_t* __restrict__ pos) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) {
        const int32_t i = perm[k];
        if (i >= 0 && i < N) pos[i] = (int32_t)k;
    }
}
__global__ void __launch_bounds__(PM_WARPS * 32) to_point_major_tiled_k(const double* __restrict__ b,
                                                                       const int32_t* __restrict__ pos, int64_t N,
                                                                       int nrhs, int stride, double* __restrict__ out) {
    __shared__ double tile[PM_WARPS][32][17];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int64_t i0 = ((int64_t)blockIdx.x * PM_WARPS + w) * 32;
    if (i0 >= N) return;
    const bool in = i0 + lane < N;
    for (int r = 0; r < stride; ++r) tile[w][lane][r] = (in && r < nrhs) ? b[(int64_t)r * N + i0 + lane] : 0.0;
    __syncwarp();
    for (int e = lane; e < 32 * stride; e += 32) {
        const int p = e / stride, r = e - p * stride;
        const int32_t k = i0 + p < N ? pos[i0 + p] : -1;
        if (k >= 0) out[(int64_t)k * stride + r] = tile[w][p][r];
    }
}
__global__ void __launch_bounds__(PM_WARPS * 32) from_point_major_tiled_k(const double* __restrict__ xp,
                                                                         const int32_t* __restrict__ pos, int64_t N,
                                                                         int nrhs, int stride, double* __restrict__ x) {
    __shared__ double tile[PM_WARPS][32][17];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int64_t i0 = ((int64_t)blockIdx.x * PM_WARPS + w) * 32;
    if (i0 >= N) return;
    for (int e = lane; e < 32 * stride; e += 32) {
        const int p = e / stride, r = e - p * stride;
        const int32_t k = i0 + p < N ? pos[i0 + p] : -1;
        tile[w][p][r] = k >= 0 ? xp[(int64_t)k * stride + r] : 0.0;
    }
    __syncwarp();
    if (i0 + lane < N)
        for (int r = 0; r < nrhs; ++r) x[(int64_t)r * N + i0 + lane] = tile[w][lane][r];
}

static kc_status inverse_perm(const int32_t* perm, int64_t N, int32_t** pos, cudaStream_t s) {
    KC_TRY(scratch_alloc((void**)pos, sizeof(int32_t) * (size_t)(N > 0 ? N : 1), s));
    KC_CUDA(cudaMemsetAsync(*pos, 0xFF, sizeof(int32_t) * (size_t)(N > 0 ? N : 1), s));
    ::kc::note_launch(), pm_inverse_perm_k<<<blocks_for(N, 256), 256, 0, s>>>(perm, N, *pos);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

kc_status to_point_major(const double* b, const int32_t* perm, int64_t N, int nrhs, double* out, cudaStream_t s,
                         int stride) {
    if (stride < nrhs) stride = nrhs;
    if (stride > 16) {
        ::kc::note_launch(), to_point_major_k<<<blocks_for(N * stride, 256), 256, 0, s>>>(b, perm, N, nrhs, stride, out);
        KC_CUDA(cudaGetLastError());
        return KC_OK;
    }
    int32_t* pos = nullptr;
    KC_TRY(inverse_perm(perm, N, &pos, s));
    ::kc::note_launch(), to_point_major_tiled_k<<<blocks_for(N, PM_WARPS * 32), PM_WARPS * 32, 0, s>>>(b, pos, N, nrhs,
                                                                                                   stride, out);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(pos, s);
    if (e != cudaSuccess) return cuda_fail(e, "to_point_major_tiled_k");
    return KC_OK;
}
kc_status from_point_major(const double* xp, const int32_t* perm, int64_t N, int nrhs, double* x, cudaStream_t s,
                           int stride) {
    if (stride < nrhs) stride = nrhs;
    if (stride > 16) {
        ::kc::note_launch(), from_point_major_k<<<blocks_for(N * nrhs, 256), 256, 0, s>>>(xp, perm, N, nrhs, stride, x);
        KC_CUDA(cudaGetLastError());
        return KC_OK;
    }
    int32_t* pos = nullptr;
    KC_TRY(inverse_perm(perm, N, &pos, s));
    ::kc::note_launch(), from_point_major_tiled_k<<<blocks_for(N, PM_WARPS * 32), PM_WARPS * 32, 0, s>>>(xp, pos, N, nrhs,
                                                                                                     stride, x);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(pos, s);
    if (e != cudaSuccess) return cuda_fail(e, "from_point_major_tiled_k");
    return KC_OK;
}

kc_status solve_impl(const kc_pattern* P, int prec, const void* val, const double* diag, const kc_kernel* kern,
                     const int32_t* perm, const double* b, int nrhs, double* x, const kc_opts* o, cudaStream_t s) {
    KernelParams kp;
    KC_TRY(kernel_params(kern, &kp));
    if (nrhs < 1 || nrhs > 16) return fail(KC_EINVAL, "nrhs must be in 1..16");
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
    int ns = 1;
    while (ns < nrhs) ns <<= 1;  // padded stride: aligned gathers; the extra columns stay zero
    Arena A(s);
    Solver S;
    KC_TRY(solver_init(S, P, ns, o, A, s));
    double *bp, *zp;
    KC_TRY(A.get(&bp, P->N * ns));
    KC_TRY(A.get(&zp, P->N * ns));
    KC_TRY(to_point_major(b, perm, P->N, nrhs, bp, s, ns));
    double fb = sqrt(kp.sigma2 + kp.nugget);
    if (prec == KC_FP64) KC_TRY(solver_apply<double>(S, (const double*)val, diag, fb, bp, zp, ns, s));
    else KC_TRY(solver_apply<float>(S, (const float*)val, diag, fb, bp, zp, ns, s));
    KC_TRY(from_point_major(zp, perm, P->N, nrhs, x, s, ns));
    return solver_check(S, s);
}

}  // namespace kc
