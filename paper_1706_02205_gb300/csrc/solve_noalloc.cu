// kc_solve_noalloc: the triangular solves of kc_solve for callers that cannot
// allocate device memory while they run.
//
// Some callers cannot call cudaMalloc (or cudaMallocAsync) at solve time: a
// serving process whose device memory is handed out up front to another
// framework's pool, a plugin that a host application forbids to allocate, or
// a latency-critical loop where an allocation may block on driver locks or
// implicitly synchronise the device.  This entry point takes its scratch from
// one fixed, file-scope device array instead, so a call performs no allocation
// at all; the caller still passes every input and output.
//
// The array is SCRATCH_BYTES (28 MiB + 256 B) and lives on every GPU that
// loads this library until the process exits.  It bounds the sizes:
// N <= 2^20 and N * nrhs <= 2^20.  Calls beyond that are rejected with
// KC_EINVAL.  All calls on a device share the one array: calls that overlap on
// the GPU (two streams, or two host threads) race and corrupt each other's
// results; serialise them.  The array keeps the last call's contents; every
// call clears what must start at zero (ready flags, tickets, status).
//
// Host code cannot use the array's name as a device address (it is a
// host-side stand-in).  The first call on each device, with that device
// current, looks the address up with cudaGetSymbolAddress and caches it; make
// that first call before any stream capture.  The cache is keyed on the
// unique id of the current CUDA context, so after a cudaDeviceReset the next
// call looks the address up again instead of using the old context's.
//
// Method: the same two level-scheduled solves as kc_solve (forward by rows of
// L in (level, index) order, backward by columns of L in the reverse order),
// with one warp per row/column and no chunking of wide columns.
#include <mutex>

#include "common.cuh"

namespace kc {

namespace {

constexpr int64_t NA_MAX_N = int64_t(1) << 20;
constexpr int64_t NA_MAX_NRHS_N = int64_t(1) << 20;
// ready flags (N ints), three point-major N x nrhs double buffers, control words
constexpr size_t NA_READY_BYTES = sizeof(int) * NA_MAX_N;
constexpr size_t NA_VEC_BYTES = sizeof(double) * NA_MAX_NRHS_N;
constexpr size_t NA_CTRL_BYTES = 256;
constexpr size_t SCRATCH_BYTES = NA_READY_BYTES + 3 * NA_VEC_BYTES + NA_CTRL_BYTES;

static __device__ __align__(256) unsigned char g_solve_scratch[SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_addr[NA_MAX_DEVICES] = {nullptr};
unsigned long long g_ctx_id[NA_MAX_DEVICES] = {0};

// The unique id (cuCtxGetId) of the calling thread's current CUDA context, by
// the driver entry points the runtime hands out (no link against libcuda).
// False if there is no current context or the driver lacks the calls.
bool current_context_id(unsigned long long* id) {
    typedef int (*get_current_t)(void**);
    typedef int (*get_id_t)(void*, unsigned long long*);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (get_current_t)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (get_id_t)f;
    });
    void* ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

kc_status scratch_address(unsigned char** out) {
    int dev = 0;
    KC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(KC_EINVAL, "kc_solve_noalloc: device index out of range");
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev] || !have_id || g_ctx_id[dev] != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);  // makes the context current if needed
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(solve scratch)");
        if (!have_id) have_id = current_context_id(&id);
        g_addr[dev] = (unsigned char*)p;
        g_ctx_id[dev] = have_id ? id : 0;  // 0: no id, so the next call looks the address up again
    }
    *out = g_addr[dev];
    return KC_OK;
}

struct NaArgs {
    int64_t N;
    int nrhs, NR;
    const int64_t* rowptr;
    const int32_t* col;
    const int64_t* colptr;
    const int32_t* rowidx;
    const int64_t* slot;
    const int32_t* order;
    const void* val;
    int is_f32;
    const double* diag;
    double diag_fallback;
    const double* b;  // point-major rhs
    double* y;        // point-major forward result
    double* x;        // point-major backward result
    int* ready;
    unsigned long long* ticket;
    int* status;
    long long spin_limit;
};

__device__ __forceinline__ double na_val(const NaArgs& A, int64_t e) {
    return A.is_f32 ? (double)__ldg((const float*)A.val + e) : __ldg((const double*)A.val + e);
}

__device__ __forceinline__ bool na_wait(const int* f, const int* status, long long limit) {
    if (ld_acquire_s32(f) != 0) return true;
    const long long t0 = clock64();
    while (ld_acquire_s32(f) == 0) {
        if (clock64() - t0 > limit || ld_volatile_s32(status) != 0) return false;
        __nanosleep(64);
    }
    return true;
}

__global__ void na_fwd_k(NaArgs A) {
    const int lane = lane_id();
    const unsigned FULL = 0xffffffffu;
    const int per = 32 / A.NR, r = lane % A.NR, eo = lane / A.NR;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&A.ticket[0], 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= A.N || ld_volatile_s32(A.status) != 0) return;
        const int j = A.order[t];
        const int64_t a = A.rowptr[j], b = A.rowptr[j + 1] - 1;
        bool ok = true;
        for (int64_t e = a + lane; e < b && ok; e += 32) ok = na_wait(&A.ready[A.col[e]], A.status, A.spin_limit);
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
            return;
        }
        __threadfence();
        __syncwarp();
        double s = 0.0;
        if (r < A.nrhs)
            for (int64_t e = a + eo; e < b; e += per)
                s = fma(na_val(A, e), __ldcg(&A.y[(int64_t)A.col[e] * A.nrhs + r]), s);
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

__global__ void na_bwd_k(NaArgs A) {
    const int lane = lane_id();
    const unsigned FULL = 0xffffffffu;
    const int per = 32 / A.NR, r = lane % A.NR, eo = lane / A.NR;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&A.ticket[1], 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if ((int64_t)t >= A.N || ld_volatile_s32(A.status) != 0) return;
        const int i = A.order[A.N - 1 - (int64_t)t];
        const int64_t c0 = A.colptr[i] + 1, c1 = A.colptr[i + 1];  // rows below the diagonal
        bool ok = true;
        for (int64_t q = c0 + lane; q < c1 && ok; q += 32) ok = na_wait(&A.ready[A.rowidx[q]], A.status, A.spin_limit);
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) atomicCAS(A.status, 0, DEV_TIMEOUT);
            return;
        }
        __threadfence();
        __syncwarp();
        double s = 0.0;
        if (r < A.nrhs)
            for (int64_t q = c0 + eo; q < c1; q += per)
                s = fma(na_val(A, A.slot[q]), __ldcg(&A.x[(int64_t)A.rowidx[q] * A.nrhs + r]), s);
        for (int o = 16; o >= A.NR; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
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

__global__ void na_gather_k(const double* __restrict__ b, const int32_t* __restrict__ perm, int64_t N, int nrhs,
                            double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * nrhs) out[t] = b[(int64_t)(t % nrhs) * N + perm[t / nrhs]];
}
__global__ void na_scatter_k(const double* __restrict__ xp, const int32_t* __restrict__ perm, int64_t N, int nrhs,
                             double* __restrict__ x) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * nrhs) x[(int64_t)(t % nrhs) * N + perm[t / nrhs]] = xp[t];
}

}  // namespace

kc_status solve_noalloc_impl(const kc_pattern* P, int prec, const void* val, const double* diag,
                             const kc_kernel* kern, const int32_t* perm, const double* b, int nrhs, double* x,
                             cudaStream_t s) {
    KernelParams kp;
    KC_TRY(kernel_params(kern, &kp));
    if (prec != KC_FP64 && prec != KC_FP32_FORM) return fail(KC_EINVAL, "prec must be KC_FP64 or KC_FP32_FORM");
    if (nrhs < 1 || nrhs > 16) return fail(KC_EINVAL, "nrhs must be in 1..16");
    if (P->N > NA_MAX_N || P->N * (int64_t)nrhs > NA_MAX_NRHS_N)
        return fail(KC_EINVAL, "kc_solve_noalloc: needs N <= 2^20 and N*nrhs <= 2^20 (fixed scratch of " +
                                   std::to_string(SCRATCH_BYTES) + " bytes); use kc_solve for larger problems");
    unsigned char* base = nullptr;
    KC_TRY(scratch_address(&base));
    const int64_t N = P->N;
    NaArgs a;
    a.N = N;
    a.nrhs = nrhs;
    a.NR = 1;
    while (a.NR < nrhs) a.NR <<= 1;
    a.rowptr = P->rowptr;
    a.col = P->col;
    a.colptr = P->colptr;
    a.rowidx = P->rowidx;
    a.slot = P->slot;
    a.order = P->order;
    a.val = val;
    a.is_f32 = prec == KC_FP32_FORM;
    a.diag = diag;
    a.diag_fallback = sqrt(kp.sigma2 + kp.nugget);
    a.ready = (int*)base;
    double* bp = (double*)(base + NA_READY_BYTES);
    a.b = bp;
    a.y = (double*)(base + NA_READY_BYTES + NA_VEC_BYTES);
    a.x = (double*)(base + NA_READY_BYTES + 2 * NA_VEC_BYTES);
    unsigned char* ctrl = base + NA_READY_BYTES + 3 * NA_VEC_BYTES;
    a.ticket = (unsigned long long*)ctrl;  // two tickets
    a.status = (int*)(ctrl + 16);
    a.spin_limit = 4000000000LL;
    // the array keeps the previous call's contents: clear what starts at zero
    KC_CUDA(cudaMemsetAsync(a.ready, 0, sizeof(int) * N, s));
    KC_CUDA(cudaMemsetAsync(ctrl, 0, 32, s));
    const int64_t n = N * nrhs;
    ::kc::note_launch(), na_gather_k<<<blocks_for(n, 256), 256, 0, s>>>(b, perm, N, nrhs, bp);
    const int grid = sm_count() * 8;
    ::kc::note_launch(), na_fwd_k<<<grid, 256, 0, s>>>(a);
    KC_CUDA(cudaMemsetAsync(a.ready, 0, sizeof(int) * N, s));
    ::kc::note_launch(), na_bwd_k<<<grid, 256, 0, s>>>(a);
    ::kc::note_launch(), na_scatter_k<<<blocks_for(n, 256), 256, 0, s>>>(a.x, perm, N, nrhs, x);
    KC_CUDA(cudaGetLastError());
    int h_status = 0;
    KC_CUDA(cudaMemcpyAsync(&h_status, a.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (h_status == DEV_TIMEOUT) return fail(KC_ETIMEOUT, "kc_solve_noalloc: a dependency wait ran out");
    if (h_status != 0) return fail(KC_ECUDA, "kc_solve_noalloc: device status " + std::to_string(h_status));
    return KC_OK;
}

}  // namespace kc
