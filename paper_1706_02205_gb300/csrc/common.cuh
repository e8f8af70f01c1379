// Shared device helpers of libkchol (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/kchol.h"

namespace kc {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
const char* last_error_cstr();
kc_status fail(kc_status st, const std::string& msg);
kc_status cuda_fail(cudaError_t e, const char* what);

#define KC_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t _e = (call);                                             \
        if (_e != cudaSuccess) return ::kc::cuda_fail(_e, #call);            \
    } while (0)

#define KC_TRY(expr)                                                         \
    do {                                                                     \
        kc_status _s = (expr);                                               \
        if (_s != KC_OK) return _s;                                          \
    } while (0)

// Device status word values written by kernels (0 = fine).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD_INPUT = 2 };

// ------------------------------------------------------- stream scratch
// The scratch comes from a private stream-ordered memory pool per device
// (scratch_pool), never from the device's default pool, so other users of
// cudaMallocAsync in the process are not affected.  The pool keeps up to
// SCRATCH_KEEP_BYTES of freed memory mapped for the next call (with a release
// threshold of 0 every call would map its scratch -- GBs for a 2^20-point
// schedule -- afresh); kc_scratch_trim returns it to the driver.
constexpr uint64_t SCRATCH_KEEP_BYTES = 16ull << 30;
kc_status scratch_pool(cudaMemPool_t* out);
kc_status scratch_alloc(void** p, size_t bytes, cudaStream_t s);
kc_status scratch_trim(int64_t keep_bytes);

// Stream-ordered scratch: every buffer is freed (cudaFreeAsync) when the
// arena goes out of scope, after the work enqueued before that point.
struct Arena {
    cudaStream_t s;
    static constexpr int CAP = 128;
    void* ptrs[CAP];
    int n = 0;
    explicit Arena(cudaStream_t st) : s(st) {}
    ~Arena() {
        for (int i = n - 1; i >= 0; --i) cudaFreeAsync(ptrs[i], s);
    }
    template <typename T>
    kc_status get(T** out, size_t count) {
        if (n == CAP) return fail(KC_ENOMEM, "scratch arena full");
        void* p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        KC_TRY(scratch_alloc(&p, bytes, s));
        ptrs[n++] = p;
        *out = (T*)p;
        return KC_OK;
    }
};

int sm_count();

// Every kernel launch of the library goes through note_launch() (a process-wide
// counter, read by kc_launch_count) so callers can see how much device work ran.
void note_launch();
int64_t launch_count();
// Device time of the last persistent factor kernel (CUDA events on its stream).
void set_factor_kernel_ms(double ms);
double factor_kernel_ms();

// ------------------------------------------------------ device helpers
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_s32(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_s32(const int* p) { return *(volatile const int*)p; }
// Acquire-release fence at GPU scope: after relaxed loads of ready flags it
// orders the loads that follow (acquire); before a flag is released it orders
// this thread's earlier writes (release).  Lighter than __threadfence()
// (sequentially consistent).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// relaxed load at GPU scope: an acquire fence after it completes the synchronisation
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Loads that bypass L1 (values written by other SMs during the same launch).
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

// Squared distance summed in coordinate order, every operation rounded on its
// own (no FMA contraction), so the bits equal a plain CPU evaluation.
__device__ __forceinline__ double dist2_exact(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        double u = __dsub_rn(a[t], b[t]);
        s = __dadd_rn(s, __dmul_rn(u, u));
    }
    return s;
}

// Matern covariance, closed forms for nu in {1/2, 3/2, 5/2}; nu_code = 0,1,2.
// scale = sqrt(2 nu)/ell.
__device__ __forceinline__ double matern_f64(double r, int nu_code, double scale, double sigma2) {
    double t = r * scale;
    double e = exp(-t);
    if (nu_code == 0) return sigma2 * e;
    if (nu_code == 1) return sigma2 * (1.0 + t) * e;
    return sigma2 * (1.0 + t + t * t * (1.0 / 3.0)) * e;
}
// roundings pinned with the _rn intrinsics (never contracted), so that every
// inlined copy gives the same bits
__device__ __forceinline__ float matern_f32(float r, int nu_code, float scale, float sigma2) {
    const float t = __fmul_rn(r, scale);
    const float e = expf(-t);
    if (nu_code == 0) return __fmul_rn(sigma2, e);
    if (nu_code == 1) return __fmul_rn(__fmul_rn(sigma2, __fadd_rn(1.0f, t)), e);
    const float poly = fmaf(__fmul_rn(t, 1.0f / 3.0f), t, __fadd_rn(1.0f, t));
    return __fmul_rn(__fmul_rn(sigma2, poly), e);
}

// Let a kernel take as much dynamic shared memory as the device allows
// beside its static shared memory.  Every caller sets the same value, so
// host threads launching the kernel concurrently (each with its own size)
// never lower the limit under one another.
template <typename F>
inline kc_status allow_dynamic_smem(F* func) {
    int dev = 0, optin = 0;
    KC_CUDA(cudaGetDevice(&dev));
    KC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    KC_CUDA(cudaFuncGetAttributes(&fa, func));
    KC_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
    return KC_OK;
}

// Covariance function of one point set (Section 4.4), as the kernels use it.
//   nu_code 0, 1, 2: Matern with nu = 1/2, 3/2, 5/2 (closed forms);
//   nu_code 3: Matern with another nu = n + mu, |mu| <= 1/2 (Bessel K_nu);
//   nu_code 4: the Cauchy class.
struct KernelParams {
    int nu_code;
    int n;          // code 3: integer part of nu + 1/2
    double scale;   // codes 0-3: sqrt(2 nu) / ell; code 4: 1 / ell
    double sigma2;
    double nugget;
    double nu, mu;               // code 3
    double gam1, gam2, gp, gm;   // code 3: (1/G(1-mu) -+ 1/G(1+mu)) / (2 mu | 2), G(1+mu), G(1-mu)
    double fact;                 // code 3: mu pi / sin(mu pi)
    double lognorm;              // code 3: log(2^{1-nu} / Gamma(nu))
    double alpha, expo;          // code 4: alpha, -beta / alpha
    int iser;                    // code 3: the I-series of coef applies for t <= 2 (nu not near an integer)
    int cheb;                    // code 3: the Chebyshev pieces of coef apply for t > 2 (nu <= 8)
    const double* coef;          // code 3: device table of KC_COEF_LEN doubles (matern_coef_table), or NULL
};
kc_status kernel_params(const kc_kernel* k, KernelParams* out);

// Per-kernel table of a Matern of general nu (code 3), KC_COEF_LEN doubles:
//   [0, KC_ISER)             a_k, [KC_ISER, 2 KC_ISER) b_k: for t <= 2,
//     G / sigma2 = sum_k a_k s^k - t^{2 nu} sum_k b_k s^k, s = t^2 / 4
//     (the power series of I_{-nu} and I_nu in K_nu = pi (I_{-nu} - I_nu) / (2 sin(nu pi)));
//   then KC_CHEB_P pieces of KC_CHEB_N Chebyshev coefficients: piece p fits
//     e^t sqrt(t) K_nu(t) on [2^{p+1}, 2^{p+2}].
constexpr int KC_ISER = 24;
constexpr int KC_CHEB_N = 24;
constexpr int KC_CHEB_P = 9;
constexpr int KC_COEF_LEN = 2 * KC_ISER + KC_CHEB_P * KC_CHEB_N;
void matern_coef_table(const KernelParams& kp, double* tab);
// Fill a device table (dst, KC_COEF_LEN doubles) for kp and point kp.coef at
// it; a no-op for kernels without one.
kc_status upload_coef(KernelParams& kp, double* dst, cudaStream_t s);
// Same with the table taken from the arena.
kc_status upload_coef(KernelParams& kp, Arena& A, cudaStream_t s);

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------- primitives
// Exclusive scan of n int64 values: out[0..n] with out[n] = total.
// `out` may alias `in` only if out has n+1 slots starting at in.
kc_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Arena& A, cudaStream_t s);
kc_status exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, Arena& A, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of key.
// Keys/values are sorted from (k_in, v_in) into (k_out, v_out); the inputs are
// used as ping-pong buffers and are clobbered.
kc_status radix_sort_u64_i64(uint64_t* k_in, int64_t* v_in, uint64_t* k_out, int64_t* v_out, int64_t n,
                             int bits, Arena& A, cudaStream_t s);
kc_status radix_sort_u32_i64(uint32_t* k_in, int64_t* v_in, uint32_t* k_out, int64_t* v_out, int64_t n,
                             int bits, Arena& A, cudaStream_t s);

inline unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace kc
