// Supernodal multicolour ordering and sparsity pattern (the paper's
// Construction in its stability section), on the device.
//
// Readings (the same as the oracle's): h = 1/2; l[1], the largest finite
// length scale, normalises the hierarchy, so maximin position m is on level
// k(m) = the smallest k >= 1 with l[m] >= l[1] 2^-k (position 0 on level 1),
// and the hierarchical pseudometric d(a, b) = dist / (l[1] 2^-min(k(a), k(b)))
// makes "d <= rho" read dist <= R_k, R_k = (rho l[1]) 2^-k with k the
// smaller level.  Supernodes of a level are chosen greedily in maximin order
// (a point is one unless an earlier supernode of its level is within d <=
// rho); every point joins the nearest supernode of its level (squared
// distance, ties to the smaller index); supernodes A, B are a pattern pair
// when some members a, b have d(a, b) <= rho; colours are greedy per level in
// maximin order of the supernodes; the order sorts by (level, colour,
// supernode, maximin position); S holds (q, p), p <= q, whenever the
// supernodes of q and p are a pair.
//
// Every pair these rules test lies in the max-rule pattern S_rho of the same
// rho (for a before b, d(a, b) <= rho means dist <= R_k(a) <= rho l[a]), so
// the construction filters that pattern's rows (later neighbours follow by
// symmetry).  The two greedy passes run as rounds that reproduce the
// sequential result exactly: a point decides once every earlier neighbour
// has (lexicographically first independent set; Jones-Plassmann colouring in
// index order).  Rounds are host-driven launches, so no kernel waits.
#include <algorithm>

#include "common.cuh"

namespace kc {

constexpr int SN_THREADS = 256;
constexpr int SN_WARPS = SN_THREADS / 32;
constexpr int SN_MAX_COLORS = 64;
constexpr int SN_MAX_ROUNDS = 1 << 20;
enum : int8_t { SN_UNDEC = 0, SN_IN = 1, SN_OUT = 2 };

__device__ __forceinline__ double sn_R(double rl1, int k) { return ldexp(rl1, -k); }

__global__ void sn_level_k(const double* __restrict__ l, int64_t N, int32_t* __restrict__ lev) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    int k = 1;
    if (m > 0) {
        const double l1 = l[1], lm = l[m];
        while (k < 1100 && !(lm >= ldexp(l1, -k))) ++k;
    }
    lev[m] = k;
}

// conflicts of m: same level, dist <= R_k.  The earlier ones come from row m
// of the pattern; the later ones by symmetry (m is a later conflict of each
// of its earlier ones), so no CSC column is scanned (the first maximin
// columns hold nearly every point).  mode 0 counts both kinds (cnt_e[m], and
// cnt_l[i] += 1 for each earlier conflict i); mode 1 fills list[off[m] ..]
// with the earlier conflicts first, then, from the other side, the later
// ones (their order within the list is immaterial).
__global__ void sn_conflicts_k(const double* __restrict__ x, int d, const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, const int32_t* __restrict__ lev, int64_t N,
                               double rl1, int mode, int32_t* __restrict__ cnt_e, int32_t* __restrict__ cnt_l,
                               const int64_t* __restrict__ off, int32_t* __restrict__ fill_l,
                               int32_t* __restrict__ list) {
    const int64_t m = (int64_t)blockIdx.x * SN_WARPS + (threadIdx.x >> 5);
    if (m >= N) return;
    const int lane = lane_id();
    const int k = lev[m];
    const double R = sn_R(rl1, k);
    const double* xm = x + m * d;
    int64_t w = mode ? off[m] : 0;
    int ne = 0;
    const int64_t a0 = rowptr[m], a1 = rowptr[m + 1] - 1;  // row m without its diagonal
    for (int64_t e0 = a0; e0 < a1; e0 += 32) {
        const int64_t e = e0 + lane;
        bool hit = false;
        int32_t i = -1;
        if (e < a1) {
            i = col[e];
            hit = lev[i] == k && sqrt(dist2_exact(xm, x + (int64_t)i * d, d)) <= R;
        }
        const unsigned b = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            if (mode) {
                list[w + __popc(b & ((1u << lane) - 1))] = i;
                list[off[i] + cnt_e[i] + atomicAdd(&fill_l[i], 1)] = (int32_t)m;
            } else {
                atomicAdd(&cnt_l[i], 1);
            }
        }
        w += __popc(b);
        ne += __popc(b);
    }
    if (!mode && lane == 0) cnt_e[m] = ne;
}

__global__ void sn_sum_k(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int64_t N,
                         int32_t* __restrict__ c) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) c[t] = a[t] + b[t];
}

// one round of the greedy independent set: m joins when every earlier
// conflict is decided and none joined; leaves as soon as one joined
__global__ void sn_mis_round_k(const int64_t* __restrict__ off, const int32_t* __restrict__ cnt_e,
                               const int32_t* __restrict__ list, int64_t N, int8_t* state,
                               unsigned long long* __restrict__ undecided) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    volatile int8_t* st = state;
    if (st[m] != SN_UNDEC) return;
    bool blocked = false;
    const int64_t e0 = off[m], e1 = e0 + cnt_e[m];
    for (int64_t e = e0; e < e1; ++e) {
        const int8_t t = st[list[e]];
        if (t == SN_IN) {
            st[m] = SN_OUT;
            return;
        }
        if (t == SN_UNDEC) blocked = true;
    }
    if (blocked) atomicAdd(undecided, 1ULL);
    else st[m] = SN_IN;
}

// nearest supernode of m's level among m's conflicts (and m itself)
__global__ void sn_assign_k(const double* __restrict__ x, int d, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ cnt, const int32_t* __restrict__ list,
                            const int8_t* __restrict__ state, int64_t N, int32_t* __restrict__ node) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    if (state[m] == SN_IN) {
        node[m] = (int32_t)m;
        return;
    }
    double best = 1.0 / 0.0;
    int32_t bs = -1;
    const double* xm = x + m * d;
    for (int64_t e = off[m]; e < off[m] + cnt[m]; ++e) {
        const int32_t s = list[e];
        if (state[s] != SN_IN) continue;
        const double e2 = dist2_exact(xm, x + (int64_t)s * d, d);
        if (e2 < best || (e2 == best && s < bs)) {
            best = e2;
            bs = s;
        }
    }
    node[m] = bs;
}

// supernode pairs: for each pattern entry (b, a), a < b, with dist <= R_k(a),
// the unordered pair of their supernodes; plus (A, A) for every supernode.
// mode 0 counts per row, mode 1 fills at off[b].
__global__ void sn_pairs_k(const double* __restrict__ x, int d, const int64_t* __restrict__ rowptr,
                           const int32_t* __restrict__ col, const int32_t* __restrict__ lev,
                           const int32_t* __restrict__ node, int64_t N, double rl1, int B, int mode,
                           int32_t* __restrict__ cnt, const int64_t* __restrict__ off, uint64_t* __restrict__ keys) {
    const int64_t b = (int64_t)blockIdx.x * SN_WARPS + (threadIdx.x >> 5);
    if (b >= N) return;
    const int lane = lane_id();
    const double* xb = x + b * d;
    const uint32_t nb = (uint32_t)node[b];
    int64_t w = mode ? off[b] : 0;
    int n = 0;
    const int64_t a0 = rowptr[b], a1 = rowptr[b + 1] - 1;
    for (int64_t e0 = a0; e0 < a1; e0 += 32) {
        const int64_t e = e0 + lane;
        bool hit = false;
        uint64_t key = 0;
        if (e < a1) {
            const int32_t a = col[e];
            hit = sqrt(dist2_exact(xb, x + (int64_t)a * d, d)) <= sn_R(rl1, lev[a]);
            const uint32_t na = (uint32_t)node[a];
            key = na < nb ? ((uint64_t)na << B | nb) : ((uint64_t)nb << B | na);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (mode && hit) keys[w + __popc(bal & ((1u << lane) - 1))] = key;
        w += __popc(bal);
        n += __popc(bal);
    }
    if (lane == 0) {
        const bool self = node[b] == (int32_t)b;  // the supernode's own block
        if (mode && self) keys[w] = (uint64_t)nb << B | nb;
        if (!mode) cnt[b] = n + (self ? 1 : 0);
    }
}

__global__ void sn_unique_mark_k(const uint64_t* __restrict__ k, int64_t n, int32_t* __restrict__ first) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) first[t] = (t == 0 || k[t] != k[t - 1]) ? 1 : 0;
}
__global__ void sn_unique_fill_k(const uint64_t* __restrict__ k, const int32_t* __restrict__ first,
                                 const int64_t* __restrict__ pos, int64_t n, uint64_t* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && first[t]) out[pos[t]] = k[t];
}

// per supernode: earlier same-level neighbours (for the colours); mode 0
// counts into cnt[hi], mode 1 fills
__global__ void sn_color_adj_k(const uint64_t* __restrict__ pairs, int64_t np, const int32_t* __restrict__ lev,
                               int B, int mode, int32_t* __restrict__ cnt, const int64_t* __restrict__ off,
                               int32_t* __restrict__ fill, int32_t* __restrict__ list) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const uint32_t lo = (uint32_t)(pairs[t] >> B), hi = (uint32_t)(pairs[t] & ((1ULL << B) - 1));
    if (lo == hi || lev[lo] != lev[hi]) return;
    if (!mode) atomicAdd(&cnt[hi], 1);
    else list[off[hi] + atomicAdd(&fill[hi], 1)] = (int32_t)lo;
}

// one Jones-Plassmann round in index order: a supernode takes the smallest
// colour its earlier neighbours lack once all of them have one
__global__ void sn_color_round_k(const int64_t* __restrict__ off, const int32_t* __restrict__ cnt,
                                 const int32_t* __restrict__ list, const int8_t* __restrict__ state, int64_t N,
                                 int32_t* color, unsigned long long* __restrict__ pending, int* __restrict__ err) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= N || state[a] != SN_IN) return;
    volatile int32_t* c = color;
    if (c[a] >= 0) return;
    unsigned long long used = 0;
    for (int64_t e = off[a]; e < off[a] + cnt[a]; ++e) {
        const int32_t cb = c[list[e]];
        if (cb < 0) {
            atomicAdd(pending, 1ULL);
            return;
        }
        used |= 1ULL << cb;
    }
    if (used == ~0ULL) {
        atomicExch(err, 1);
        c[a] = SN_MAX_COLORS - 1;
        return;
    }
    c[a] = __ffsll(~used) - 1;
}

// order key (level, colour, supernode) with the maximin position as value
__global__ void sn_order_keys_k(const int32_t* __restrict__ lev, const int32_t* __restrict__ node,
                                const int32_t* __restrict__ color, int64_t N, uint64_t* __restrict__ key,
                                int64_t* __restrict__ val) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    const int32_t s = node[m];
    key[m] = (uint64_t)lev[m] << 37 | (uint64_t)color[s] << 31 | (uint64_t)(uint32_t)s;
    val[m] = m;
}

// new position q: maximin position, the per-position outputs, the points,
// and the range [start, end) of each supernode
__global__ void sn_scatter_k(const int64_t* __restrict__ mval, const int32_t* __restrict__ lev,
                             const int32_t* __restrict__ node, const int32_t* __restrict__ color,
                             const double* __restrict__ x, int d, int64_t N, int32_t* __restrict__ newm,
                             int32_t* __restrict__ lev_out, int32_t* __restrict__ node_out,
                             int32_t* __restrict__ color_out, double* __restrict__ x_new, int32_t* __restrict__ start,
                             int32_t* __restrict__ end) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N) return;
    const int32_t m = (int32_t)mval[q];
    const int32_t s = node[m];
    if (newm) newm[q] = m;
    if (lev_out) lev_out[q] = lev[m];
    if (node_out) node_out[q] = s;
    if (color_out) color_out[q] = color[s];
    if (x_new)
        for (int t = 0; t < d; ++t) x_new[q * d + t] = x[(int64_t)m * d + t];
    if (q == 0 || node[(int32_t)mval[q - 1]] != s) start[s] = (int32_t)q;
    if (q == N - 1 || node[(int32_t)mval[q + 1]] != s) end[s] = (int32_t)(q + 1);
}

// supernode neighbour lists (both directions, the supernode itself
// included), sorted by the start of the neighbour's range: every pair gives
// the entries (lo; start[hi]) -> hi and (hi; start[lo]) -> lo (the second a
// sentinel that sorts last when lo == hi), one radix sort orders them by
// supernode then start, and cnt[A] counts A's entries.
__global__ void sn_nb_keys_k(const uint64_t* __restrict__ pairs, int64_t np, const int32_t* __restrict__ start,
                             int B, int32_t* __restrict__ cnt, uint64_t* __restrict__ key,
                             int64_t* __restrict__ val) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const uint32_t lo = (uint32_t)(pairs[t] >> B), hi = (uint32_t)(pairs[t] & ((1ULL << B) - 1));
    atomicAdd(&cnt[lo], 1);
    key[2 * t] = (uint64_t)lo << B | (uint32_t)start[hi];
    val[2 * t] = hi;
    if (lo != hi) {
        atomicAdd(&cnt[hi], 1);
        key[2 * t + 1] = (uint64_t)hi << B | (uint32_t)start[lo];
        val[2 * t + 1] = lo;
    } else {
        key[2 * t + 1] = ~0ULL;
        val[2 * t + 1] = -1;
    }
}

__global__ void sn_nb_take_k(const int64_t* __restrict__ val, int64_t n, int32_t* __restrict__ list) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) list[t] = (int32_t)val[t];
}

// row q of S: the ranges of q's supernode's neighbours that start at or
// before q, cut at q.  mode 0 counts, mode 1 fills (one warp per row).
__global__ void sn_rows_k(const int32_t* __restrict__ newm, const int32_t* __restrict__ node,
                          const int64_t* __restrict__ off, const int32_t* __restrict__ cnt,
                          const int32_t* __restrict__ list, const int32_t* __restrict__ start,
                          const int32_t* __restrict__ end, int64_t N, int mode, int64_t* __restrict__ rowcnt,
                          const int64_t* __restrict__ rowptr, int32_t* __restrict__ col) {
    const int64_t q = (int64_t)blockIdx.x * SN_WARPS + (threadIdx.x >> 5);
    if (q >= N) return;
    const int lane = lane_id();
    const int32_t a = node[newm[q]];
    const int64_t b0 = off[a], b1 = b0 + cnt[a];
    int64_t w = mode ? rowptr[q] : 0;
    for (int64_t e = b0; e < b1; ++e) {
        const int32_t b = list[e];
        const int64_t s0 = start[b];
        if (s0 > q) break;  // sorted by start
        const int64_t len = min((int64_t)end[b], q + 1) - s0;
        if (mode)
            for (int64_t t = lane; t < len; t += 32) col[w + t] = (int32_t)(s0 + t);
        w += len;
    }
    if (!mode && lane == 0) rowcnt[q] = w;
}

// ------------------------------------------------------------------ driver
struct SnState {
    int32_t* lev = nullptr;      // per maximin position
    int8_t* state = nullptr;     // supernode or not
    int32_t* node = nullptr;     // per maximin position
    uint64_t* pairs = nullptr;   // unique supernode pairs (lo << B | hi), sorted
    int64_t npairs = 0;
    int B = 1;                   // bits of an index: N - 1 < 2^B
};

static kc_status sync_read(const void* dev, void* host, size_t bytes, cudaStream_t s) {
    KC_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    return KC_OK;
}

// the unique supernode pairs of the pattern
static kc_status sn_pairs(const double* x, int d, const kc_pattern* P, double rl1, SnState& S, Arena& A,
                          cudaStream_t s) {
    const int64_t N = P->N;
    int32_t* cnt;
    int64_t* off;
    KC_TRY(A.get(&cnt, N));
    KC_TRY(A.get(&off, N + 1));
    note_launch(), sn_pairs_k<<<blocks_for(N, SN_WARPS), SN_THREADS, 0, s>>>(x, d, P->rowptr, P->col, S.lev, S.node,
                                                                            N, rl1, S.B, 0, cnt, nullptr, nullptr);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i32_to_i64(cnt, off, N, A, s));
    int64_t total = 0;
    KC_TRY(sync_read(off + N, &total, sizeof(total), s));
    uint64_t *k0, *k1;
    int64_t *v0, *v1;
    KC_TRY(A.get(&k0, total));
    KC_TRY(A.get(&k1, total));
    KC_TRY(A.get(&v0, total));
    KC_TRY(A.get(&v1, total));
    note_launch(), sn_pairs_k<<<blocks_for(N, SN_WARPS), SN_THREADS, 0, s>>>(x, d, P->rowptr, P->col, S.lev, S.node,
                                                                            N, rl1, S.B, 1, cnt, off, k0);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaMemsetAsync(v0, 0, sizeof(int64_t) * total, s));
    KC_TRY(radix_sort_u64_i64(k0, v0, k1, v1, total, 2 * S.B, A, s));
    int32_t* first;
    int64_t* pos;
    KC_TRY(A.get(&first, total));
    KC_TRY(A.get(&pos, total + 1));
    note_launch(), sn_unique_mark_k<<<blocks_for(total, 256), 256, 0, s>>>(k1, total, first);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i32_to_i64(first, pos, total, A, s));
    KC_TRY(sync_read(pos + total, &S.npairs, sizeof(int64_t), s));
    KC_TRY(A.get(&S.pairs, S.npairs));
    note_launch(), sn_unique_fill_k<<<blocks_for(total, 256), 256, 0, s>>>(k1, first, pos, total, S.pairs);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// levels, supernodes and the assignment (per maximin position)
static kc_status sn_nodes(const double* x, int d, const double* l, const kc_pattern* P, double rl1, SnState& S,
                          Arena& A, cudaStream_t s) {
    const int64_t N = P->N;
    KC_TRY(A.get(&S.lev, N));
    KC_TRY(A.get(&S.state, N));
    KC_TRY(A.get(&S.node, N));
    note_launch(), sn_level_k<<<blocks_for(N, 256), 256, 0, s>>>(l, N, S.lev);
    KC_CUDA(cudaGetLastError());
    int32_t *cnt_e, *cnt_l, *fill_l, *cnt, *list;
    int64_t* off;
    KC_TRY(A.get(&cnt_e, N));
    KC_TRY(A.get(&cnt_l, N));
    KC_TRY(A.get(&fill_l, N));
    KC_TRY(A.get(&cnt, N));
    KC_TRY(A.get(&off, N + 1));
    KC_CUDA(cudaMemsetAsync(cnt_l, 0, sizeof(int32_t) * N, s));
    KC_CUDA(cudaMemsetAsync(fill_l, 0, sizeof(int32_t) * N, s));
    note_launch(), sn_conflicts_k<<<blocks_for(N, SN_WARPS), SN_THREADS, 0, s>>>(
        x, d, P->rowptr, P->col, S.lev, N, rl1, 0, cnt_e, cnt_l, nullptr, nullptr, nullptr);
    KC_CUDA(cudaGetLastError());
    note_launch(), sn_sum_k<<<blocks_for(N, 256), 256, 0, s>>>(cnt_e, cnt_l, N, cnt);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i32_to_i64(cnt, off, N, A, s));
    int64_t total = 0;
    KC_TRY(sync_read(off + N, &total, sizeof(total), s));
    KC_TRY(A.get(&list, total));
    note_launch(), sn_conflicts_k<<<blocks_for(N, SN_WARPS), SN_THREADS, 0, s>>>(
        x, d, P->rowptr, P->col, S.lev, N, rl1, 1, cnt_e, cnt_l, off, fill_l, list);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaMemsetAsync(S.state, 0, N, s));
    unsigned long long* und;
    KC_TRY(A.get(&und, 1));
    int rounds = 0;
    for (;;) {
        KC_CUDA(cudaMemsetAsync(und, 0, sizeof(unsigned long long), s));
        note_launch(), sn_mis_round_k<<<blocks_for(N, 256), 256, 0, s>>>(off, cnt_e, list, N, S.state, und);
        KC_CUDA(cudaGetLastError());
        unsigned long long h = 0;
        KC_TRY(sync_read(und, &h, sizeof(h), s));
        if (h == 0) break;
        if (++rounds > SN_MAX_ROUNDS) return fail(KC_ECUDA, "supernodal: independent-set rounds did not finish");
    }
    note_launch(), sn_assign_k<<<blocks_for(N, 256), 256, 0, s>>>(x, d, off, cnt, list, S.state, N, S.node);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// colours of the supernodes (per maximin position of the supernode)
static kc_status sn_colors(const SnState& S, int64_t N, int32_t* color, Arena& A, cudaStream_t s) {
    int32_t *cnt, *fill, *list;
    int64_t* off;
    KC_TRY(A.get(&cnt, N));
    KC_TRY(A.get(&fill, N));
    KC_TRY(A.get(&off, N + 1));
    KC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * N, s));
    KC_CUDA(cudaMemsetAsync(fill, 0, sizeof(int32_t) * N, s));
    note_launch(), sn_color_adj_k<<<blocks_for(S.npairs, 256), 256, 0, s>>>(S.pairs, S.npairs, S.lev, S.B, 0, cnt,
                                                                           nullptr, nullptr, nullptr);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i32_to_i64(cnt, off, N, A, s));
    int64_t total = 0;
    KC_TRY(sync_read(off + N, &total, sizeof(total), s));
    KC_TRY(A.get(&list, total));
    note_launch(), sn_color_adj_k<<<blocks_for(S.npairs, 256), 256, 0, s>>>(S.pairs, S.npairs, S.lev, S.B, 1, cnt,
                                                                           off, fill, list);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaMemsetAsync(color, 0xff, sizeof(int32_t) * N, s));  // -1: uncoloured
    unsigned long long* pend;
    int* err;
    KC_TRY(A.get(&pend, 1));
    KC_TRY(A.get(&err, 1));
    KC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    int rounds = 0;
    for (;;) {
        KC_CUDA(cudaMemsetAsync(pend, 0, sizeof(unsigned long long), s));
        note_launch(), sn_color_round_k<<<blocks_for(N, 256), 256, 0, s>>>(off, cnt, list, S.state, N, color, pend,
                                                                          err);
        KC_CUDA(cudaGetLastError());
        unsigned long long h = 0;
        KC_TRY(sync_read(pend, &h, sizeof(h), s));
        if (h == 0) break;
        if (++rounds > SN_MAX_ROUNDS) return fail(KC_ECUDA, "supernodal: colouring rounds did not finish");
    }
    int herr = 0;
    KC_TRY(sync_read(err, &herr, sizeof(int), s));
    if (herr) return fail(KC_EINVAL, "supernodal: a level needs more than 64 colours (rho too large)");
    return KC_OK;
}

// the order: maximin position of every new position (mval, int64) and the
// supernode ranges
static kc_status sn_order(const SnState& S, const int32_t* color, int64_t N, int64_t** mval, Arena& A,
                          cudaStream_t s) {
    uint64_t *k0, *k1;
    int64_t *v0, *v1;
    KC_TRY(A.get(&k0, N));
    KC_TRY(A.get(&k1, N));
    KC_TRY(A.get(&v0, N));
    KC_TRY(A.get(&v1, N));
    note_launch(), sn_order_keys_k<<<blocks_for(N, 256), 256, 0, s>>>(S.lev, S.node, color, N, k0, v0);
    KC_CUDA(cudaGetLastError());
    KC_TRY(radix_sort_u64_i64(k0, v0, k1, v1, N, 48, A, s));
    *mval = v1;
    return KC_OK;
}

// neighbour lists sorted by range start, the row counts and rowptr, and the
// rows themselves when col has room for them
static kc_status sn_rows(const SnState& S, const int32_t* newm, const int32_t* start, const int32_t* end, int64_t N,
                         int64_t* rowptr, int64_t* nnz_out, int32_t* col, int64_t col_cap, Arena& A, cudaStream_t s) {
    int32_t *cnt, *list;
    int64_t* off;
    KC_TRY(A.get(&cnt, N));
    KC_TRY(A.get(&off, N + 1));
    KC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * N, s));
    const int64_t ne = 2 * S.npairs;
    uint64_t *k0, *k1;
    int64_t *v0, *v1;
    KC_TRY(A.get(&k0, ne));
    KC_TRY(A.get(&k1, ne));
    KC_TRY(A.get(&v0, ne));
    KC_TRY(A.get(&v1, ne));
    note_launch(), sn_nb_keys_k<<<blocks_for(S.npairs, 256), 256, 0, s>>>(S.pairs, S.npairs, start, S.B, cnt, k0,
                                                                          v0);
    KC_CUDA(cudaGetLastError());
    KC_TRY(radix_sort_u64_i64(k0, v0, k1, v1, ne, 2 * S.B + 1, A, s));  // + the sentinel bit
    KC_TRY(exclusive_scan_i32_to_i64(cnt, off, N, A, s));
    KC_TRY(A.get(&list, ne));
    note_launch(), sn_nb_take_k<<<blocks_for(ne, 256), 256, 0, s>>>(v1, ne, list);
    KC_CUDA(cudaGetLastError());
    if (nnz_out) {
        int64_t* rowcnt;
        KC_TRY(A.get(&rowcnt, N));
        note_launch(), sn_rows_k<<<blocks_for(N, SN_WARPS), SN_THREADS, 0, s>>>(newm, S.node, off, cnt, list, start,
                                                                               end, N, 0, rowcnt, nullptr, nullptr);
        KC_CUDA(cudaGetLastError());
        KC_TRY(exclusive_scan_i64(rowcnt, rowptr, N, A, s));
        KC_TRY(sync_read(rowptr + N, nnz_out, sizeof(int64_t), s));
        if (!col || *nnz_out > col_cap) return KC_OK;
    }
    note_launch(), sn_rows_k<<<blocks_for(N, SN_WARPS), SN_THREADS, 0, s>>>(newm, S.node, off, cnt, list, start,
                                                                           end, N, 1, nullptr, rowptr, col);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaStreamSynchronize(s));
    return KC_OK;
}

// nnz_out given: rowptr and nnz are computed, and col is filled when it holds
// col_cap >= nnz entries; nnz_out NULL: col is filled from the given rowptr
kc_status supernodal_impl(const double* x_ord, const double* l, int d, double rho, const kc_pattern* P,
                          int32_t* newm, int32_t* level, int32_t* node_out, int32_t* color_out, double* x_new,
                          int64_t* rowptr, int64_t* nnz_out, int32_t* col, int64_t col_cap, cudaStream_t s) {
    const int64_t N = P->N;
    double l1 = 1.0;
    if (N > 1) KC_CUDA(cudaMemcpy(&l1, l + 1, sizeof(double), cudaMemcpyDeviceToHost));
    const double rl1 = rho * l1;
    Arena A(s);
    SnState S;
    while (S.B < 31 && ((int64_t)1 << S.B) < N) ++S.B;
    KC_TRY(sn_nodes(x_ord, d, l, P, rl1, S, A, s));
    KC_TRY(sn_pairs(x_ord, d, P, rl1, S, A, s));
    int32_t* color;
    KC_TRY(A.get(&color, N));
    KC_TRY(sn_colors(S, N, color, A, s));
    int64_t* mval;
    KC_TRY(sn_order(S, color, N, &mval, A, s));
    int32_t *start, *end, *nm = newm;
    KC_TRY(A.get(&start, N));
    KC_TRY(A.get(&end, N));
    if (!nm) KC_TRY(A.get(&nm, N));
    note_launch(), sn_scatter_k<<<blocks_for(N, 256), 256, 0, s>>>(mval, S.lev, S.node, color, x_ord, d, N, nm, level,
                                                                  node_out, color_out, x_new, start, end);
    KC_CUDA(cudaGetLastError());
    return sn_rows(S, nm, start, end, N, rowptr, nnz_out, col, col_cap, A, s);
}

}  // namespace kc
