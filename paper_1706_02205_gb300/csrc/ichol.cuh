// Arithmetic shared by the ICHOL(0) kernels (the column-task kernel of
// factor.cu and the column-group kernel of factor_block.cu): the
// accumulators of the two precisions, Theta_ji from the coordinates, and the
// bounded wait on a dependency's completion counter.
#pragma once
#include "covariance.cuh"

namespace kc {

// Accumulators.  FP32: compensated dot product Dot2 of Ogita, Rump and Oishi
// (TwoProduct by fma, TwoSum of the running sum, errors summed apart); FP64:
// plain fma.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void group_reduce(int G) {
        for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    // (theta - sum) / L_ii, a correctly rounded division as Algorithm 2
    // states it (a stored reciprocal moves ill-conditioned columns by more
    // than the FP64 bar)
    __device__ __forceinline__ double finish(double th, double Lii, double) const { return (th - s) / Lii; }
    __device__ __forceinline__ double total() const { return s; }
    __device__ __forceinline__ static double recip(double) { return 0.0; }  // finish divides
};
template <>
struct Acc<float> {
    // every operation rounded on its own (the _rn intrinsics are never
    // contracted into an FMA): the error-free transformations rely on it, and
    // every inlined copy then rounds the same way
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float ep = fmaf(a, b, -p);
        const float ns = __fadd_rn(s, p);
        const float z = __fsub_rn(ns, s);
        const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(ns, z)), __fsub_rn(p, z));
        s = ns;
        c = __fadd_rn(c, __fadd_rn(ep, es));
    }
    __device__ __forceinline__ void group_reduce(int G) {
        for (int o = G >> 1; o > 0; o >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
            const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
            const float t = __fadd_rn(s, s2);
            const float z = __fsub_rn(t, s);
            const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
            s = t;
            c = __fadd_rn(c, __fadd_rn(c2, e));
        }
    }
    __device__ __forceinline__ float finish(float th, double, float inv) const {
        return __fmul_rn(__fsub_rn(__fsub_rn(th, s), c), inv);
    }
    // both parts in FP64: the compensated sum to about FP64 accuracy
    __device__ __forceinline__ double total() const { return (double)s + (double)c; }
    __device__ __forceinline__ static float recip(double Lii) { return __frcp_rn((float)Lii); }
};

// Where the entries come from (a template parameter of the kernels, so that
// each instantiation holds only its own entry code):
//   ENT = 0: the closed-form Matern kernels (nu = 1/2, 3/2, 5/2);
//   ENT = 1: every covariance function (the calls behind the other families
//            would cost the closed-form kernels registers);
//   ENT = 2: a given matrix on the pattern (aval, Section 6).
// Theta_ji off the diagonal from the coordinates (ENT 0 and 1, GEN = ENT == 1).
template <typename T, bool GEN>
__device__ __forceinline__ T theta_off(const KernelParams& kp, int d, const double* xj, const double* xi) {
    if constexpr (sizeof(T) == 8) {
        double s = 0.0;
        for (int t = 0; t < d; ++t) {
            double u = xj[t] - xi[t];
            s = fma(u, u, s);
        }
        if constexpr (GEN) return cov_f64(kp, sqrt(s));
        else return matern_f64(sqrt(s), kp.nu_code, kp.scale, kp.sigma2);
    } else {
        float s = 0.f;
        for (int t = 0; t < d; ++t) {
            float u = (float)(xj[t] - xi[t]);
            s = fmaf(u, u, s);
        }
        if constexpr (GEN) return cov_f32(kp, sqrtf(s));
        else return matern_f32(sqrtf(s), kp.nu_code, (float)kp.scale, (float)kp.sigma2);
    }
}

// done[k] starts at minus the number of tasks of column k and every finished
// task adds one, so column k is complete exactly when done[k] >= 0: one load
// per dependency.  The loads are relaxed so that a lane's checks all go out
// at once; an acquire fence after them orders the value loads that follow.
// spin_done: bounded wait (backoff) on a column not yet complete; false when
// the budget ran out or the kernel is stopping.
__device__ __forceinline__ bool spin_done(const unsigned* f, const int* status, long long limit) {
    const long long t0 = clock64();
    unsigned ns = 32;
    while ((int)ld_relaxed_u32(f) < 0) {
        if (clock64() - t0 > limit || ld_volatile_s32(status) != 0) return false;
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
    }
    return true;
}

}  // namespace kc
