// Covariance functions of Section 4.4 evaluated on the device: the Matern
// class (Eq. (Matern)) for any nu > 0 and the Cauchy class of Gneiting.
// The closed forms of nu = 1/2, 3/2, 5/2 live in common.cuh (matern_f64,
// matern_f32) and are the only code on the path of those kernels; the other
// families sit behind calls so that they add no registers to the hot loops.
#pragma once
#include "common.cuh"

namespace kc {

// Matern with general nu at t = sqrt(2 nu) r / ell > 0:
//   sigma2 2^{1-nu} / Gamma(nu) t^nu K_nu(t).
// K_mu and K_{mu+1} for |mu| <= 1/2 come from Temme's series (t <= 2;
// N. M. Temme, J. Comput. Phys. 19 (1975) 324) or from Steed's evaluation
// of the continued fraction for K_{mu+1}/K_mu together with the series that
// normalises it (t > 2; I. J. Thompson and A. R. Barnett, J. Comput. Phys. 64
// (1987) 490); K_nu then follows by the upward recurrence
// K_{m+1}(t) = K_{m-1}(t) + (2m/t) K_m(t), which is stable for K.
// Every iteration count is bounded.
static __device__ __noinline__ double matern_general_f64(double t, int n, double nu, double mu, double gam1, double gam2,
                                                  double gp, double gm, double fact, double lognorm,
                                                  double sigma2) {
    if (!(t > 0.0)) return sigma2;
    double k0, k1;
    if (t <= 2.0) {
        // K_mu = sum_k c_k f_k and K_{mu+1} = (2/t) sum_k c_k (p_k - k f_k), c_k = (t^2/4)^k / k!
        const double lx = log(0.5 * t);
        const double sg = -mu * lx;  // mu log(2/t)
        const double shs = fabs(sg) < 1e-3 ? 1.0 + sg * sg * (1.0 / 6.0) : sinh(sg) / sg;
        double f = fact * (cosh(sg) * gam1 - shs * lx * gam2);
        const double e = exp(sg);  // (t/2)^{-mu}
        double p = 0.5 * e * gp, q = 0.5 / e * gm;
        const double y = 0.25 * t * t;
        double c = 1.0, s0 = f, s1 = p;
        for (int k = 1; k < 200; ++k) {
            const double dk = (double)k;
            f = (dk * f + p + q) / (dk * dk - mu * mu);
            c *= y / dk;
            p /= dk - mu;
            q /= dk + mu;
            const double tf = c * f;
            s0 += tf;
            s1 += c * (p - dk * f);
            if (fabs(tf) < 1e-17 * fabs(s0)) break;
        }
        k0 = s0;
        k1 = s1 * (2.0 / t);
    } else {
        // Steed: the continued fraction as a sum of its convergent differences
        // (h), and alongside it the sum s with K_mu = sqrt(pi/(2t)) e^{-t} / s
        const double a1 = 0.25 - mu * mu;
        double b = 2.0 * (1.0 + t), d = 1.0 / b, dh = d, h = d;
        double qa = 0.0, qb = 1.0, qs = a1, c = a1, a = -a1;
        double s = 1.0 + qs * dh;
        for (int i = 1; i < 1000; ++i) {
            a -= 2.0 * i;
            c = -a * c / (i + 1.0);
            const double qn = (qa - b * qb) / a;
            qa = qb;
            qb = qn;
            qs += c * qn;
            b += 2.0;
            d = 1.0 / (b + a * d);
            dh = (b * d - 1.0) * dh;
            h += dh;
            const double ds = qs * dh;
            s += ds;
            if (fabs(ds) < 1e-17 * fabs(s)) break;
        }
        k0 = sqrt(3.14159265358979323846 / (2.0 * t)) * exp(-t) / s;
        k1 = k0 * (mu + t + 0.5 - a1 * h) / t;
    }
    for (int m = 1; m < n; ++m) {
        const double kn = k0 + (2.0 * (mu + m) / t) * k1;
        k0 = k1;
        k1 = kn;
    }
    const double kv = n == 0 ? k0 : k1;
    if (kv == 0.0) return 0.0;
    return sigma2 * exp(lognorm + nu * log(t)) * kv;
}

// Cauchy class: sigma2 (1 + u^alpha)^{-beta/alpha}, u = r / ell
static __device__ __noinline__ double cauchy_f64(double u, double alpha, double expo, double sigma2) {
    return sigma2 * exp(expo * log1p(pow(u, alpha)));
}
static __device__ __noinline__ float cauchy_f32(float u, float alpha, float expo, float sigma2) {
    return __fmul_rn(sigma2, expf(__fmul_rn(expo, log1pf(powf(u, alpha)))));
}

// The covariance function at distance r (no nugget), as the FP64 path
// evaluates it.
__device__ __forceinline__ double cov_f64(const KernelParams& kp, double r) {
    if (kp.nu_code <= 2) return matern_f64(r, kp.nu_code, kp.scale, kp.sigma2);
    if (kp.nu_code == 3)
        return matern_general_f64(r * kp.scale, kp.n, kp.nu, kp.mu, kp.gam1, kp.gam2, kp.gp, kp.gm, kp.fact,
                                  kp.lognorm, kp.sigma2);
    return cauchy_f64(r * kp.scale, kp.alpha, kp.expo, kp.sigma2);
}

// As the FP32 form evaluates it: closed forms and the Cauchy class in float;
// a Matern of other nu in double, rounded.
__device__ __forceinline__ float cov_f32(const KernelParams& kp, float r) {
    if (kp.nu_code <= 2) return matern_f32(r, kp.nu_code, (float)kp.scale, (float)kp.sigma2);
    if (kp.nu_code == 3)
        return (float)matern_general_f64((double)r * kp.scale, kp.n, kp.nu, kp.mu, kp.gam1, kp.gam2, kp.gp, kp.gm,
                                         kp.fact, kp.lognorm, kp.sigma2);
    return cauchy_f32(__fmul_rn(r, (float)kp.scale), (float)kp.alpha, (float)kp.expo, (float)kp.sigma2);
}

}  // namespace kc
