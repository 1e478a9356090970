// Voigt function H(a, x) in FP64 for the table build.
//
// H(a, x) = Re w(x + i a), w the Faddeeva function (Sec. 2.1 defines the
// profile; the function itself is standard). Two regimes:
//
//  * |x| < 8: Weideman's rational expansion (J.A.C. Weideman, SIAM J.
//    Numer. Anal. 31 (1994) 1497): with t = L tan(theta/2) the function
//    (L^2 + t^2) exp(-t^2) is expanded in Fourier modes exp(i n theta) =
//    ((L + i t)/(L - i t))^n, which turns the Cauchy integral for w into
//      w(z) ~ 2 p(Z) / (L - i z)^2 + 1 / (sqrt(pi) (L - i z)),
//      Z = (L + i z)/(L - i z),  p(Z) = sum_{n=0}^{N-1} c_{n+1} Z^n,
//    c_n the Fourier coefficients (computed on the host by a direct DFT).
//  * |x| >= 8: the asymptotic series w(z) ~ (i / (sqrt(pi) z))
//    sum_k (2k-1)!! / (2 z^2)^k, summed until the terms stop shrinking. Its
//    real part is formed without cancellation, which keeps H accurate deep
//    in the Lorentz wing where Re w << |w|.
//  * a < 1e-6 and |x| < 8: the expansion of Re w(x + i a) in powers of a
//    (Taylor series of w about the real axis, w' = -2 z w + 2 i / sqrt(pi)):
//      H = exp(-x^2) + (2a/sqrt(pi)) (2 x D(x) - 1) + a^2 (1 - 2x^2) exp(-x^2),
//    D the Dawson function; the rational expansion's absolute error
//    (~1e-16 |w|) would swamp H there, which falls to ~1e-15 near |x| = 6.
//    D(x) = exp(-x^2) sum_n x^(2n+1) / (n! (2n+1)), a series of positive
//    terms (no cancellation).
#pragma once

#include <cmath>

#ifndef KRL_HD
#define KRL_HD __host__ __device__
#endif

namespace krl {

constexpr int kWeidemanN = 48;

struct cplx {
    double re, im;
};
KRL_HD inline cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
KRL_HD inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
KRL_HD inline cplx cdiv(cplx a, cplx b)
{
    double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// Weideman's scale for N terms.
inline double weideman_L(int N) { return std::sqrt(N / std::sqrt(2.0)); }

// Fourier coefficients c_1..c_N of f(theta) = (L^2 + t^2) exp(-t^2),
// t = L tan(theta/2), by the trapezoidal rule on 2M points (M = 2N); f is
// even in theta, so the coefficients are real cosine sums. Host only.
inline void weideman_coefficients(double* c, int N)
{
    const double L = weideman_L(N);
    const int M = 2 * N;
    const double pi = 3.14159265358979323846;
    for (int n = 1; n <= N; ++n) {
        double s = 0.0;
        for (int k = -M + 1; k <= M - 1; ++k) {
            double th = k * pi / M;
            double t = L * std::tan(0.5 * th);
            double f = (L * L + t * t) * std::exp(-t * t);
            s += f * std::cos(n * th);
        }
        c[n - 1] = s / (2.0 * M);
    }
}

// w(z) for Im z >= 0, |Re z| < 8, from the coefficients above.
KRL_HD inline cplx faddeeva_rational(double x, double y, const double* c, int N, double L)
{
    // iz = -y + i x
    cplx lmiz = {L + y, -x};           // L - i z
    cplx lpiz = {L - y, x};            // L + i z
    cplx Z = cdiv(lpiz, lmiz);
    cplx p = {c[N - 1], 0.0};          // Horner: p = sum c_{n+1} Z^n
    for (int n = N - 2; n >= 0; --n) p = cadd(cmul(p, Z), cplx{c[n], 0.0});
    cplx den = cmul(lmiz, lmiz);
    cplx t1 = cdiv(cplx{2.0 * p.re, 2.0 * p.im}, den);
    const double rsqrtpi = 0.56418958354775628695;
    cplx t2 = cdiv(cplx{rsqrtpi, 0.0}, lmiz);
    return cadd(t1, t2);
}

// Re w(z) by the asymptotic series, |z| large.
KRL_HD inline double faddeeva_asymptotic_re(double x, double y)
{
    const double rsqrtpi = 0.56418958354775628695;
    cplx z = {x, y};
    cplx iz = cdiv(cplx{0.0, 1.0}, z);                  // i / z
    cplx z2 = cmul(z, z);
    cplx inv2z2 = cdiv(cplx{0.5, 0.0}, z2);             // 1 / (2 z^2)
    cplx term = {1.0, 0.0};
    cplx sum = {1.0, 0.0};
    double prev = 1.0;
    for (int k = 1; k < 60; ++k) {
        term = cmul(term, inv2z2);
        term.re *= (2 * k - 1);
        term.im *= (2 * k - 1);
        double mag = std::fabs(term.re) + std::fabs(term.im);
        if (mag > prev) break;                         // divergent tail
        sum = cadd(sum, term);
        prev = mag;
        if (mag < 1e-18) break;
    }
    cplx w = cmul(iz, sum);
    return rsqrtpi * w.re;
}

// Dawson's function for 0 <= x < 8 by the erfi power series.
KRL_HD inline double dawson(double x)
{
    const double x2 = x * x;
    double term = x;              // x^(2n+1) / n!
    double sum = x;
    for (int n = 1; n < 400; ++n) {
        term *= x2 / n;
        double add = term / (2 * n + 1);
        sum += add;
        if (add < 1e-17 * sum) break;
    }
    return std::exp(-x2) * sum;
}

// H(a, x) for a > 0.
KRL_HD inline double voigt_H(double a, double x, const double* c, int N, double L)
{
    double ax = std::fabs(x);
    if (ax >= 8.0) return faddeeva_asymptotic_re(ax, a);
    if (a < 1e-6) {
        const double e = std::exp(-ax * ax);
        const double rsqrtpi2 = 1.1283791670955125739;   // 2 / sqrt(pi)
        return e + a * rsqrtpi2 * (2.0 * ax * dawson(ax) - 1.0) + a * a * (1.0 - 2.0 * ax * ax) * e;
    }
    return faddeeva_rational(ax, a, c, N, L).re;
}

}  // namespace krl
