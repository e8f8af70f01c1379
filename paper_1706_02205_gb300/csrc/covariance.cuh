// Covariance functions of Section 4.4 evaluated on the device: the Matern
// class (Eq. (Matern)) for any nu > 0 and the Cauchy class of Gneiting.
// The closed forms of nu = 1/2, 3/2, 5/2 live in common.cuh (matern_f64,
// matern_f32) and are the only code on the path of those kernels; the other
// families sit behind calls so that they add no registers to the hot loops.
#pragma once
#include "common.cuh"

namespace kc {

// Steed's evaluation (I. J. Thompson and A. R. Barnett, J. Comput. Phys. 64
// (1987) 490) of the continued fraction for K_{mu+1}/K_mu, summed as the
// differences of its convergents (h), together with the series s that
// normalises it: K_mu(t) = sqrt(pi / (2t)) e^{-t} / s.  For t > 2 and
// |mu| <= 1/2; returns both values scaled by e^t sqrt(t), which keeps them in
// range for any t.  The iteration count is bounded.
__host__ __device__ inline void steed_scaled(double t, double mu, double& g0, double& g1) {
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
    g0 = 1.2533141373155002512 / s;  // sqrt(pi / 2)
    g1 = g0 * (mu + t + 0.5 - a1 * h) / t;
}

// K_{mu+n} from K_mu, K_{mu+1} by the upward recurrence
// K_{m+1}(t) = K_{m-1}(t) + (2m/t) K_m(t), stable for K (any common scale).
__host__ __device__ inline double k_upward(double t, double mu, int n, double k0, double k1) {
    if (n == 0) return k0;
    for (int m = 1; m < n; ++m) {
        const double kn = k0 + (2.0 * (mu + m) / t) * k1;
        k0 = k1;
        k1 = kn;
    }
    return k1;
}

// Matern with general nu at t = sqrt(2 nu) r / ell (Eq. (Matern)):
//   G = sigma2 2^{1-nu} / Gamma(nu) t^nu K_nu(t),  nu = n + mu, |mu| <= 1/2.
// With the kernel's table (coef): t <= 2 by the two power series of the
// table (one log, one exp, two Horner sums); t > 2 by the Chebyshev piece of
// e^t sqrt(t) K_nu(t) that holds t.  Without a table, or where its parts do
// not apply (nu within 0.02 of an integer for t <= 2, nu > 8 for t > 2):
// Temme's series for K_mu and K_{mu+1} (t <= 2; N. M. Temme, J. Comput.
// Phys. 19 (1975) 324) or Steed's continued fraction (t > 2), then the upward
// recurrence.  Every loop is bounded.
static __device__ __noinline__ double matern_general_f64(double t, int n, double nu, double mu, double gam1,
                                                         double gam2, double gp, double gm, double fact,
                                                         double lognorm, double sigma2, const double* coef, int iser,
                                                         int cheb) {
    if (!(t > 0.0)) return sigma2;
    const double lt = log(t);
    if (t <= 2.0) {
        if (coef && iser) {
            const double sq = 0.25 * t * t;
            double A = __ldg(coef + KC_ISER - 1), B = __ldg(coef + 2 * KC_ISER - 1);
            for (int k = KC_ISER - 2; k >= 0; --k) {
                A = fma(A, sq, __ldg(coef + k));
                B = fma(B, sq, __ldg(coef + KC_ISER + k));
            }
            return sigma2 * (A - exp(2.0 * nu * lt) * B);
        }
        // Temme: K_mu = sum_k c_k f_k and K_{mu+1} = (2/t) sum_k c_k (p_k - k f_k), c_k = (t^2/4)^k / k!
        const double lx = lt - 0.69314718055994530942;  // log(t / 2)
        const double sg = -mu * lx;                       // mu log(2/t)
        const double e = exp(sg), ie = 1.0 / e;          // (t/2)^{-mu} and its inverse
        const double shs = fabs(sg) < 1e-3 ? 1.0 + sg * sg * (1.0 / 6.0) : 0.5 * (e - ie) / sg;
        double f = fact * (0.5 * (e + ie) * gam1 - shs * lx * gam2);
        double p = 0.5 * e * gp, q = 0.5 * ie * gm;
        const double y = 0.25 * t * t;
        double c = 1.0, s0 = f, s1 = p;
        for (int k = 1; k < 200; ++k) {
            const double dk = (double)k;
            const double r = 1.0 / (dk * dk - mu * mu);  // 1/(k-mu) = (k+mu) r, 1/(k+mu) = (k-mu) r
            f = (dk * f + p + q) * r;
            c *= y / dk;
            p *= (dk + mu) * r;
            q *= (dk - mu) * r;
            const double tf = c * f;
            s0 += tf;
            s1 += c * (p - dk * f);
            if (fabs(tf) < 1e-17 * fabs(s0)) break;
        }
        const double kv = k_upward(t, mu, n, s0, s1 * (2.0 / t));
        if (kv == 0.0) return 0.0;
        return sigma2 * exp(lognorm + nu * lt) * kv;
    }
    if (t >= (double)(2 << KC_CHEB_P)) return 0.0;  // G < e^{-t} t^nu: far below the double range
    double g;
    if (coef && cheb) {
        const int pc = ilogb(t) - 1;                   // t in [2^{pc+1}, 2^{pc+2})
        const double x = ldexp(t, -pc) - 3.0;          // mapped to [-1, 1]
        const double* cc = coef + 2 * KC_ISER + pc * KC_CHEB_N;
        double b1 = 0.0, b2 = 0.0;
        for (int k = KC_CHEB_N - 1; k > 0; --k) {
            const double bn = fma(2.0 * x, b1, __ldg(cc + k) - b2);
            b2 = b1;
            b1 = bn;
        }
        g = fma(x, b1, 0.5 * __ldg(cc) - b2);
    } else {
        double g0, g1;
        steed_scaled(t, mu, g0, g1);
        g = k_upward(t, mu, n, g0, g1);
    }
    return sigma2 * exp(lognorm + (nu - 0.5) * lt - t) * g;
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
                                  kp.lognorm, kp.sigma2, kp.coef, kp.iser, kp.cheb);
    return cauchy_f64(r * kp.scale, kp.alpha, kp.expo, kp.sigma2);
}

// As the FP32 form evaluates it: closed forms and the Cauchy class in float;
// a Matern of other nu in double, rounded.
__device__ __forceinline__ float cov_f32(const KernelParams& kp, float r) {
    if (kp.nu_code <= 2) return matern_f32(r, kp.nu_code, (float)kp.scale, (float)kp.sigma2);
    if (kp.nu_code == 3)
        return (float)matern_general_f64((double)r * kp.scale, kp.n, kp.nu, kp.mu, kp.gam1, kp.gam2, kp.gp, kp.gm,
                                         kp.fact, kp.lognorm, kp.sigma2, kp.coef, kp.iser, kp.cheb);
    return cauchy_f32(__fmul_rn(r, (float)kp.scale), (float)kp.alpha, (float)kp.expo, (float)kp.sigma2);
}

}  // namespace kc
