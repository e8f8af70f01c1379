// a4: the dependency schedule of the factorisation.
//
// Column i of the left-looking ICHOL(0) (Algorithm 2) needs every column k in
// row i of L (k in R_i) to be complete, so the columns form a DAG whose
// levels are level(i) = 1 + max_{k in R_i} level(k).  This file builds, on the
// device: the CSC view of L (rows of each column ascending, with the CSR slot
// of every entry), the levels (a sync-free kernel over rows in index order),
// and the columns sorted by level with a stable radix sort; within a level by
// index, or, given the points, by the Morton code of each column's point, so
// that the factor's consecutive tasks and the solves' consecutive rows touch
// neighbouring points, whose rows share most of their entries (L2 reuse).
#include "grid.cuh"

namespace kc {

// Sort items of the CSR entries: key = column, value = (row << pb) | position
// with pb bits for positions, so the sorted items carry their rows (no gather
// after the sort).
__global__ void col_keys_k(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t N, int pb,
                           uint32_t* __restrict__ key, int64_t* __restrict__ val) {
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = lane_id();
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < N; j += nw) {
        const int64_t a = rowptr[j], b = rowptr[j + 1];
        for (int64_t e = a + lane; e < b; e += 32) {
            key[e] = (uint32_t)col[e];
            val[e] = (j << pb) | e;
        }
    }
}

// After the stable sort by column: slot[q] = CSR position, rowidx[q] = its row,
// colptr[c] = first q of column c (every column holds its diagonal).
__global__ void csc_finish_k(const uint32_t* __restrict__ skey, const int64_t* __restrict__ sval, int64_t nnz,
                             int64_t N, int pb, int64_t* __restrict__ colptr, int32_t* __restrict__ rowidx,
                             int64_t* __restrict__ slot) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nnz) {
        const int64_t v = sval[q];
        slot[q] = v & (((int64_t)1 << pb) - 1);
        rowidx[q] = (int32_t)(v >> pb);
        uint32_t c = skey[q];
        if (q == 0 || skey[q - 1] != c) colptr[c] = q;
    }
    if (q == 0) colptr[N] = nnz;
}

// level[j] = 1 + max level over row j; rows claimed in index order, so a row
// waits only on rows with smaller index that were claimed before it.
__device__ __forceinline__ int ld_relaxed_level(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// level[j] = 1 + max level over row j; rows claimed in index order, so a row
// waits only on rows with smaller index that were claimed before it.  Each
// lane reads up to 8 of the row's levels with relaxed loads all in flight
// together and spins (bounded, with back-off) only on those not yet set.
// Only the level values are read, so no acquire ordering is needed.
__global__ void levels_k(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t N,
                         int* __restrict__ level, unsigned long long* __restrict__ ticket, int* __restrict__ depth,
                         int* __restrict__ status, long long spin_limit) {
    constexpr int D = 8;
    int lane = lane_id();
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1ULL);
        t = __shfl_sync(0xffffffffu, t, 0);
        if ((int64_t)t >= N) return;
        if (ld_volatile_s32(status) != 0) return;
        const int64_t j = (int64_t)t;
        const int64_t a = rowptr[j];
        const int n = (int)(rowptr[j + 1] - 1 - a);
        int m = 0;
        bool ok = true;
        for (int e0 = 0; e0 < n; e0 += 32 * D) {
            int kk[D], v[D];
#pragma unroll
            for (int u = 0; u < D; ++u) {
                const int e = e0 + lane + 32 * u;
                kk[u] = e < n ? __ldg(&col[a + e]) : -1;
            }
#pragma unroll
            for (int u = 0; u < D; ++u) v[u] = kk[u] >= 0 ? ld_relaxed_level(&level[kk[u]]) : 0;
#pragma unroll
            for (int u = 0; u < D; ++u) {
                if (kk[u] >= 0 && v[u] == 0 && ok) {
                    const long long t0 = clock64();
                    unsigned ns = 32;
                    while ((v[u] = ld_relaxed_level(&level[kk[u]])) == 0) {
                        if (clock64() - t0 > spin_limit || ld_volatile_s32(status) != 0) {
                            ok = false;
                            break;
                        }
                        __nanosleep(ns);
                        if (ns < 512) ns <<= 1;
                    }
                }
                m = max(m, v[u]);
            }
            if (!__all_sync(0xffffffffu, ok)) break;
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicCAS(status, 0, DEV_TIMEOUT);
            return;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            st_release_s32(&level[j], m + 1);
            atomicMax(depth, m + 1);
        }
    }
}
__global__ void level_keys_k(const int* __restrict__ level, int64_t N, uint32_t* __restrict__ key,
                             int64_t* __restrict__ val) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) {
        key[j] = (uint32_t)level[j];
        val[j] = j;
    }
}

__global__ void level_morton_keys_k(const int* __restrict__ level, const double* __restrict__ x, int d, Box3 box,
                                    int64_t N, uint64_t* __restrict__ key, int64_t* __restrict__ val) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) {
        key[j] = ((uint64_t)(uint32_t)level[j] << 32) | morton_of(x + j * d, d, box);
        val[j] = j;
    }
}
__global__ void order_out_k(const int64_t* __restrict__ sval, int64_t N, int32_t* __restrict__ order) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) order[p] = (int32_t)sval[p];
}

#ifndef KC_LEVELS_BLOCKS_PER_SM
#define KC_LEVELS_BLOCKS_PER_SM 2
#endif

// A second stream for work that runs beside the caller's stream `home`:
// fork() makes it wait for the work enqueued on home so far, join() makes
// home wait for it.  Going out of scope joins (if not joined yet) and
// releases the stream and events, so that scratch freed on home afterwards
// (an Arena declared before this object) is never freed under the second
// stream's work, whichever way the function returns.
struct AuxStream {
    cudaStream_t home = nullptr, s = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    bool joined = true;
    kc_status fork(cudaStream_t from) {
        home = from;
        KC_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        KC_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        KC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        KC_CUDA(cudaEventRecord(ev[0], from));
        KC_CUDA(cudaStreamWaitEvent(s, ev[0], 0));
        joined = false;
        return KC_OK;
    }
    kc_status join() {
        if (joined) return KC_OK;
        joined = true;
        KC_CUDA(cudaEventRecord(ev[1], s));
        KC_CUDA(cudaStreamWaitEvent(home, ev[1], 0));
        return KC_OK;
    }
    ~AuxStream() {
        if (!joined && s) {
            cudaEventRecord(ev[1], s);
            cudaStreamWaitEvent(home, ev[1], 0);
        }
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (s) cudaStreamDestroy(s);
    }
};

static int bits_for(int64_t v) {
    int b = 1;
    while (b < 63 && ((int64_t)1 << b) <= v) ++b;
    return b;
}

kc_status schedule_impl(int64_t N, const int64_t* rowptr, const int32_t* col, int64_t nnz, const double* x, int d,
                        int64_t* colptr, int32_t* rowidx, int64_t* slot, int32_t* level, int32_t* order,
                        int32_t* depth_out, cudaStream_t s) {
    Arena A(s);
    // The levels (a dependency chain, latency-bound) run on a second stream next to the CSC sort
    // (bound by its ranking): both read only the CSR rows.  The level kernel takes a quarter of the
    // SMs' thread slots so that the sort's blocks find room.
    unsigned long long* ticket;
    int* dev_depth;
    int* status;
    KC_TRY(A.get(&ticket, 1));
    KC_TRY(A.get(&dev_depth, 1));
    KC_TRY(A.get(&status, 1));
    KC_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s));
    KC_CUDA(cudaMemsetAsync(dev_depth, 0, sizeof(int), s));
    KC_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    KC_CUDA(cudaMemsetAsync(level, 0, sizeof(int) * N, s));
    AuxStream aux;
    KC_TRY(aux.fork(s));
    const int sms = sm_count();
    ::kc::note_launch(), levels_k<<<sms * KC_LEVELS_BLOCKS_PER_SM, 256, 0, aux.s>>>(rowptr, col, N, level, ticket,
                                                                               dev_depth, status, 4000000000LL);
    KC_CUDA(cudaGetLastError());

    // CSC by a stable sort of the CSR entries by column
    const int pb = bits_for(nnz);
    if (pb + bits_for(N) > 63) {
        return fail(KC_EINVAL, "schedule: N and nnz too large for packed sort values");
    }
    uint32_t *k0, *k1;
    int64_t *v0, *v1;
    KC_TRY(A.get(&k0, nnz));
    KC_TRY(A.get(&k1, nnz));
    KC_TRY(A.get(&v0, nnz));
    KC_TRY(A.get(&v1, nnz));
    ::kc::note_launch(), col_keys_k<<<sms * 8, 256, 0, s>>>(rowptr, col, N, pb, k0, v0);
    KC_CUDA(cudaGetLastError());
    KC_TRY(radix_sort_u32_i64(k0, v0, k1, v1, nnz, bits_for(N), A, s));
    ::kc::note_launch(), csc_finish_k<<<blocks_for(nnz, 256), 256, 0, s>>>(k1, v1, nnz, N, pb, colptr, rowidx, slot);
    KC_CUDA(cudaGetLastError());

    KC_TRY(aux.join());  // the levels are complete on s from here on
    int h_depth = 0, h_status = 0;
    KC_CUDA(cudaMemcpyAsync(&h_depth, dev_depth, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (h_status != 0) return fail(KC_ETIMEOUT, "level computation: a dependency wait ran out");

    if (x) {
        // columns sorted by (level, Morton code of the point)
        double lo[3], hi[3];
        KC_TRY(bbox(x, N, d, lo, hi, A, s));
        Box3 box;
        for (int t = 0; t < 3; ++t) {
            box.lo[t] = t < d ? lo[t] : 0.0;
            const double e = t < d ? hi[t] - lo[t] : 0.0;
            box.inv[t] = e > 0 ? 1.0 / e : 0.0;
        }
        uint64_t *m0, *m1;
        KC_TRY(A.get(&m0, N));
        KC_TRY(A.get(&m1, N));
        ::kc::note_launch(), level_morton_keys_k<<<blocks_for(N, 256), 256, 0, s>>>(level, x, d, box, N, m0, v0);
        KC_CUDA(cudaGetLastError());
        KC_TRY(radix_sort_u64_i64(m0, v0, m1, v1, N, 32 + bits_for(h_depth), A, s));
    } else {
        // columns sorted by (level, index)
        ::kc::note_launch(), level_keys_k<<<blocks_for(N, 256), 256, 0, s>>>(level, N, k0, v0);
        KC_CUDA(cudaGetLastError());
        KC_TRY(radix_sort_u32_i64(k0, v0, k1, v1, N, bits_for(h_depth), A, s));
    }
    ::kc::note_launch(), order_out_k<<<blocks_for(N, 256), 256, 0, s>>>(v1, N, order);
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaStreamSynchronize(s));
    if (depth_out) *depth_out = h_depth;
    return KC_OK;
}

}  // namespace kc
