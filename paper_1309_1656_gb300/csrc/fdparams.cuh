// Parameters of the matrix-valued Fermi-Dirac equilibrium of one site
// (Sec. 2.2, Prop. 1; Eqs. rhoFDstdOmega, nFDstdOmega, energyFDstdOmega),
// in double precision on the GPU.
//
// Given the site's density matrix rho = (n 1 + S.sigma)/2 and internal energy
// eps: the analytic 2x2 eigen-decomposition gives the occupations
// n_up/dn = (n +- |S|)/2 and the Bloch axis S/|S| of U (Sec. 2.2: U is the
// eigenbasis of rho); then (beta, nu_up, nu_dn), nu = beta mu,
// solve
//   n_s = (2 pi/beta)^h F_{h-1}(nu_s),   n eps = h beta^-1 (2 pi/beta)^h sum_s F_h(nu_s),
// h = d/2.  The three equations are solved together by Newton's method on
// their logarithms in the unknowns (log beta, nu_up, nu_dn), started from the
// classical limit F_k(x) ~ e^x (where the logarithmic system is linear), with
// the Jacobian from dF_k/dx = F_{k-1}; each iteration evaluates F_{h-2},
// F_{h-1}, F_h of both species in one pass.  A site on which that iteration
// does not settle is solved again by the nested method: for a trial beta each
// species is inverted on its own (closed form in 2D, F_0(nu) = log(1 + e^nu);
// Newton on log F_{1/2} in 3D), and beta is found by a bracketed Newton
// iteration on log beta of the energy equation, using
// d nu_s / d beta = h F_{h-1}(nu_s) / (beta F_{h-2}(nu_s)).
#pragma once

#include <math_constants.h>

#include "fd_tables.h"
#include "lattice.cuh"

namespace qlbm {

// Flag bit: a site whose Fermi-Dirac parameters could not be recovered.
constexpr unsigned FLAG_FD_UNRESOLVED = 4u;

// Table index: 0 -> k = -1/2, 1 -> 1/2, 2 -> 3/2, 3 -> 1.
__device__ __forceinline__ double fd_eval(int ki, double x)
{
    if (x <= -1.0) {   // alternating series in q = e^x
        const double q = exp(x);
        double acc = 0.0;
        for (int n = FD_NSER - 1; n >= 0; --n) acc = fma(q, acc, (n & 1) ? -FD_SERIES[ki][n] : FD_SERIES[ki][n]);
        return q * acc;
    }
    if (x < 1.0) {     // Taylor series about 0: eta(k+1-j) x^j / j!
        double acc = 0.0;
        for (int j = FD_NTAY - 1; j >= 0; --j) acc = fma(x, acc, FD_TAYLOR[ki][j]);
        return acc;
    }
    if (ki == 3) {     // F_1(x) = x^2/2 + pi^2/6 - F_1(-x)
        const double q = exp(-x);
        double acc = 0.0;
        for (int n = FD_NSER - 1; n >= 0; --n) acc = fma(q, acc, (n & 1) ? -FD_SERIES[3][n] : FD_SERIES[3][n]);
        return 0.5 * x * x + 1.6449340668482264 - q * acc;
    }
    if (x < FD_X0 + FD_NINT * FD_WIDTH) {   // Chebyshev (Clenshaw)
        const int i = (int)((x - FD_X0) / FD_WIDTH);
        const double a = FD_X0 + FD_WIDTH * i;
        const double t = (x - a - 0.5 * FD_WIDTH) / (0.5 * FD_WIDTH);
        const double *c = FD_CHEB[ki][i];
        double b1 = 0.0, b2 = 0.0;
        for (int j = FD_NCHEB - 1; j >= 1; --j) {
            const double b0 = fma(2.0 * t, b1, c[j] - b2);
            b2 = b1;
            b1 = b0;
        }
        return fma(t, b1, c[0] - b2);
    }
    // Sommerfeld: x^(k+1)/Gamma(k+2) (1 + sum_n a_n x^-2n)
    const double r = 1.0 / (x * x);
    double acc = 0.0;
    for (int n = FD_NASYM - 1; n >= 1; --n) acc = fma(r, acc, FD_ASYM[ki][n]);
    const double k = ki == 0 ? -0.5 : (ki == 1 ? 0.5 : 1.5);
    return pow(x, k + 1.0) * FD_ASYM[ki][0] * fma(r, acc, 1.0);
}

__device__ __forceinline__ double fd_m1(double x)   // F_-1(x) = (1 + e^-x)^-1
{
    return x > 0.0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x));
}
__device__ __forceinline__ double fd_0(double x)    // F_0(x) = log(1 + e^x)
{
    return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

// F_{h-2}, F_{h-1}, F_h for h = D/2.
template <int D> __device__ __forceinline__ double fd_hm2(double x) { return D == 2 ? fd_m1(x) : fd_eval(0, x); }
template <int D> __device__ __forceinline__ double fd_hm1(double x) { return D == 2 ? fd_0(x) : fd_eval(1, x); }
template <int D> __device__ __forceinline__ double fd_h(double x) { return D == 2 ? fd_eval(3, x) : fd_eval(2, x); }

constexpr double kTwoPi = 6.283185307179586;

// nu with (2 pi/beta)^h F_{h-1}(nu) = ns.
template <int D> __device__ __forceinline__ double species_nu(double beta, double ns)
{
    if (D == 2) {
        const double y = ns * beta / kTwoPi;
        return y > 30.0 ? y + log(-expm1(-y)) : log(expm1(y));
    }
    const double y = ns * pow(beta / kTwoPi, 1.5);
    const double ly = log(y);
    double nu = y < 1.0 ? ly : pow(y * 1.3293403881791355, 2.0 / 3.0);   // Gamma(5/2)
    double lo = -1e300, hi = 1e300;
    for (int it = 0; it < 60; ++it) {
        const double F = fd_eval(1, nu), Fm = fd_eval(0, nu);
        const double phi = log(F) - ly;
        if (phi > 0.0) hi = nu;
        else lo = nu;
        double nn = nu - phi * F / Fm;
        if (!(nn > lo && nn < hi)) nn = (lo > -1e299 && hi < 1e299) ? 0.5 * (lo + hi) : (phi > 0.0 ? nu - 5.0 : nu + 5.0);
        const bool done = fabs(nn - nu) <= 4e-15 * (1.0 + fabs(nu));
        nu = nn;
        if (done) break;
    }
    return nu;
}

struct FdParams {
    double beta, mu_up, mu_dn, ax, ay, az;
    double n_up, n_dn;   // (2 pi/beta)^h F_{h-1}(beta mu_s) at the solution
    int status;          // 0 ok, 1 rho not positive definite, 2 no beta fits / no convergence
};

// Alternating series sum_{n>=1} (-1)^(n+1) q^n / n^(k+1), q = e^x <= 1/e, for
// the NK tables from K0, truncated after NT terms: the series alternates with
// decreasing terms, so the error is below q^(NT+1), and F_k >= q/2.
template <int NT, int K0, int NK>
__device__ __forceinline__ void fd_series_nt(double q, double *out)
{
    double acc[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) acc[k] = 0.0;
#pragma unroll
    for (int n = NT - 1; n >= 0; --n) {
#pragma unroll
        for (int k = 0; k < NK; ++k)
            acc[k] = fma(q, acc[k], (n & 1) ? -FD_SERIES[K0 + k][n] : FD_SERIES[K0 + k][n]);
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) out[k] = q * acc[k];
}

// The same at q = e^x, x <= -1, with as many terms as keep 2 q^NT below
// 1e-17 relative: 6 for x <= -8, 14 for x <= -3, else the full table.
template <int K0, int NK>
__device__ __forceinline__ void fd_series(double x, double q, double *out)
{
    if (x <= -8.0) fd_series_nt<6, K0, NK>(q, out);
    else if (x <= -3.0) fd_series_nt<14, K0, NK>(q, out);
    else fd_series_nt<FD_NSER, K0, NK>(q, out);
}

// F_{h-2}, F_{h-1}, F_h (h = D/2) at one argument, sharing the exponential,
// the interval and the powers between the three.
struct Fd3 {
    double m2, m1, h;
};

template <int D> __device__ __forceinline__ Fd3 fd3(double x)
{
    Fd3 r;
    if (D == 2) {   // F_-1 = (1 + e^-x)^-1, F_0 = log(1 + e^x), F_1 (tables)
        double o[1];
        if (x <= -1.0) {
            const double q = exp(x);
            r.m2 = q / (1.0 + q);
            r.m1 = log1p(q);
            fd_series<3, 1>(x, q, o);
            r.h = o[0];
        } else if (x < 1.0) {
            const double e = exp(x);
            r.m2 = e / (1.0 + e);
            r.m1 = log1p(e);
            double acc = 0.0;
            for (int j = FD_NTAY - 1; j >= 0; --j) acc = fma(x, acc, FD_TAYLOR[3][j]);
            r.h = acc;
        } else {        // F_1(x) = x^2/2 + pi^2/6 - F_1(-x)
            const double q = exp(-x);
            r.m2 = 1.0 / (1.0 + q);
            r.m1 = x + log1p(q);
            fd_series<3, 1>(-x, q, o);
            r.h = 0.5 * x * x + 1.6449340668482264 - o[0];
        }
        return r;
    }
    double o[3];
    if (x <= -1.0) {
        fd_series<0, 3>(x, exp(x), o);
    } else if (x < 1.0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int j = FD_NTAY - 1; j >= 0; --j) acc = fma(x, acc, FD_TAYLOR[k][j]);
            o[k] = acc;
        }
    } else if (x < FD_X0 + FD_NINT * FD_WIDTH) {
        const int i = (int)((x - FD_X0) / FD_WIDTH);
        const double a = FD_X0 + FD_WIDTH * i;
        const double t = (x - a - 0.5 * FD_WIDTH) / (0.5 * FD_WIDTH);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double *c = FD_CHEB[k][i];
            double b1 = 0.0, b2 = 0.0;
            for (int j = FD_NCHEB - 1; j >= 1; --j) {
                const double b0 = fma(2.0 * t, b1, c[j] - b2);
                b2 = b1;
                b1 = b0;
            }
            o[k] = fma(t, b1, c[0] - b2);
        }
    } else {        // Sommerfeld: x^(k+1)/Gamma(k+2) (1 + sum_n a_n x^-2n), k + 1 = 1/2, 3/2, 5/2
        const double r2 = 1.0 / (x * x), sq = sqrt(x);
        const double xp[3] = {sq, x * sq, x * x * sq};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int n = FD_NASYM - 1; n >= 1; --n) acc = fma(r2, acc, FD_ASYM[k][n]);
            o[k] = xp[k] * FD_ASYM[k][0] * fma(r2, acc, 1.0);
        }
    }
    r.m2 = o[0];
    r.m1 = o[1];
    r.h = o[2];
    return r;
}

// Single-precision F_{h-2}, F_{h-1}, F_h from the float tables FDF_*
// (truncated where the dropped terms are below ~1e-9 relative).
template <int NT, int K0, int NK>
__device__ __forceinline__ void fd_series_ntf(float q, float *out)
{
    float acc[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) acc[k] = 0.f;
#pragma unroll
    for (int n = NT - 1; n >= 0; --n) {
#pragma unroll
        for (int k = 0; k < NK; ++k)
            acc[k] = fmaf(q, acc[k], (n & 1) ? -FDF_SERIES[K0 + k][n] : FDF_SERIES[K0 + k][n]);
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) out[k] = q * acc[k];
}

// q = e^x, x <= -1; 2 q^NT below 1e-8 relative: 3 terms for x <= -8, 7 for
// x <= -3, else 20.
template <int K0, int NK>
__device__ __forceinline__ void fd_seriesf(float x, float q, float *out)
{
    if (x <= -8.f) fd_series_ntf<3, K0, NK>(q, out);
    else if (x <= -3.f) fd_series_ntf<7, K0, NK>(q, out);
    else fd_series_ntf<FDF_NSER, K0, NK>(q, out);
}

struct Fd3f {
    float m2, m1, h;
};

template <int D> __device__ __forceinline__ Fd3f fd3f(float x)
{
    Fd3f r;
    if (D == 2) {
        float o[1];
        if (x <= -1.f) {
            const float q = expf(x);
            r.m2 = q / (1.f + q);
            r.m1 = log1pf(q);
            fd_seriesf<3, 1>(x, q, o);
            r.h = o[0];
        } else if (x < 1.f) {
            const float e = expf(x);
            r.m2 = e / (1.f + e);
            r.m1 = log1pf(e);
            float acc = 0.f;
            for (int j = FDF_NTAY - 1; j >= 0; --j) acc = fmaf(x, acc, FDF_TAYLOR[3][j]);
            r.h = acc;
        } else {
            const float q = expf(-x);
            r.m2 = 1.f / (1.f + q);
            r.m1 = x + log1pf(q);
            fd_seriesf<3, 1>(-x, q, o);
            r.h = 0.5f * x * x + 1.64493407f - o[0];
        }
        return r;
    }
    float o[3];
    if (x <= -1.f) {
        fd_seriesf<0, 3>(x, expf(x), o);
    } else if (x < 1.f) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float acc = 0.f;
            for (int j = FDF_NTAY - 1; j >= 0; --j) acc = fmaf(x, acc, FDF_TAYLOR[k][j]);
            o[k] = acc;
        }
    } else if (x < FD_X0 + FD_NINT * FD_WIDTH) {
        const int i = (int)((x - FD_X0) / FD_WIDTH);
        const float a = FD_X0 + FD_WIDTH * i;
        const float t = (x - a - 0.5f * FD_WIDTH) / (0.5f * FD_WIDTH);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float *c = FDF_CHEB[k][i];
            float b1 = 0.f, b2 = 0.f;
            for (int j = FDF_NCHEB - 1; j >= 1; --j) {
                const float b0 = fmaf(2.f * t, b1, c[j] - b2);
                b2 = b1;
                b1 = b0;
            }
            o[k] = fmaf(t, b1, c[0] - b2);
        }
    } else {
        const float r2 = 1.f / (x * x), sq = sqrtf(x);
        const float xp[3] = {sq, x * sq, x * x * sq};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float acc = 0.f;
            for (int n = FDF_NASYM - 1; n >= 1; --n) acc = fmaf(r2, acc, FDF_ASYM[k][n]);
            o[k] = xp[k] * FDF_ASYM[k][0] * fmaf(r2, acc, 1.f);
        }
    }
    r.m2 = o[0];
    r.m1 = o[1];
    r.h = o[2];
    return r;
}

// The Newton iteration of fd_params_site in single precision, from the
// classical start: true and (t = log beta, nu_up, nu_dn) to ~1e-6 when it
// settles within 20 iterations.
template <int D>
__device__ bool fd_newton_f(float nup, float ndn, float n, float eps, float &t, float &nu1, float &nu2)
{
    constexpr float h = 0.5f * D;
    constexpr float hl2pi = h * 1.83787707f;   // h log 2 pi
    if (!(ndn > 0.f) || !(eps > 0.f) || !(n * eps > 0.f)) return false;
    const float lA = logf(nup), lB = logf(ndn), lC = logf(n * eps / h);
    t = logf(h / eps);
    nu1 = lA - hl2pi + h * t;
    nu2 = lB - hl2pi + h * t;
    for (int it = 0; it < 20; ++it) {
        const Fd3f F1 = fd3f<D>(nu1), F2 = fd3f<D>(nu2);
        const float sFh = F1.h + F2.h;
        const float r1 = logf(F1.m1) - h * t + hl2pi - lA;
        const float r2 = logf(F2.m1) - h * t + hl2pi - lB;
        const float r3 = logf(sFh) - (h + 1.f) * t + hl2pi - lC;
        const float ig1 = F1.m1 / F1.m2, ig2 = F2.m1 / F2.m2;
        const float c1 = F1.m1 / sFh, c2 = F2.m1 / sFh;
        const float den = -(h + 1.f) + h * (c1 * ig1 + c2 * ig2);
        float dt = (c1 * ig1 * r1 + c2 * ig2 * r2 - r3) / den;
        if (!(dt == dt)) return false;
        dt = fmaxf(-1.f, fminf(1.f, dt));
        const float d1 = fmaxf(-10.f, fminf(10.f, (h * dt - r1) * ig1));
        const float d2 = fmaxf(-10.f, fminf(10.f, (h * dt - r2) * ig2));
        t += dt;
        nu1 += d1;
        nu2 += d2;
        if (fmaxf(fabsf(dt), fmaxf(fabsf(d1), fabsf(d2))) <= 4e-6f * (1.f + fabsf(nu1))) return true;
    }
    return false;
}

// The nested solve (bracketed Newton on log beta around the per-species
// inversion); the fallback of fd_params_site.
template <int D>
__device__ FdParams fd_params_nested(double n, double Sx, double Sy, double Sz, double eps)
{
    constexpr double h = 0.5 * D;
    FdParams p;
    p.beta = p.mu_up = p.mu_dn = p.ax = p.ay = p.az = p.n_up = p.n_dn = CUDART_NAN;
    const double nS = sqrt(Sx * Sx + Sy * Sy + Sz * Sz);
    const double nup = 0.5 * (n + nS), ndn = 0.5 * (n - nS);
    if (!(ndn > 0.0)) {
        p.status = 1;
        return p;
    }
    if (nS > 0.0) {
        p.ax = Sx / nS;
        p.ay = Sy / nS;
        p.az = Sz / nS;
    } else {
        p.ax = p.ay = p.az = 0.0;
    }
    if (!(eps > 0.0)) {
        p.status = 2;
        return p;
    }
    const double nE = n * eps;
    const double pre = h * pow(kTwoPi, h);
    double lb = log(h / eps), lo = -1e300, hi = 1e300;
    double nu1 = 0.0, nu2 = 0.0, gres = 1e300;
    bool ok = false;
    for (int it = 0; it < 100; ++it) {
        const double beta = exp(lb);
        nu1 = species_nu<D>(beta, nup);
        nu2 = nS > 0.0 ? species_nu<D>(beta, ndn) : nu1;
        const double e = exp(-(h + 1.0) * lb);
        const double Fh = fd_h<D>(nu1) + fd_h<D>(nu2);
        const double f1 = fd_hm1<D>(nu1), f2 = fd_hm1<D>(nu2);
        const double g = pre * e * Fh - nE;
        gres = fabs(g);
        const double dg = pre * e * (-(h + 1.0) * Fh + h * (f1 * f1 / fd_hm2<D>(nu1) + f2 * f2 / fd_hm2<D>(nu2)));
        if (g > 0.0) lo = lb;
        else hi = lb;
        double step = -g / dg;
        if (!(step == step)) step = g > 0.0 ? 1.0 : -1.0;
        step = fmax(-2.0, fmin(2.0, step));
        double nb = lb + step;
        if (!(nb > lo && nb < hi)) nb = (lo > -1e299 && hi < 1e299) ? 0.5 * (lo + hi) : nb;
        const bool done = fabs(nb - lb) <= 4e-15 * (1.0 + fabs(lb));
        lb = nb;
        if (done) {
            ok = true;
            break;
        }
    }
    if (!ok && gres <= 1e-12 * nE) ok = true;   // converged to rounding level
    if (!ok) {
        p.status = 2;
        return p;
    }
    p.beta = exp(lb);
    nu1 = species_nu<D>(p.beta, nup);
    nu2 = nS > 0.0 ? species_nu<D>(p.beta, ndn) : nu1;
    p.mu_up = nu1 / p.beta;
    p.mu_dn = nu2 / p.beta;
    const double A = pow(kTwoPi / p.beta, h);
    p.n_up = A * fd_hm1<D>(nu1);
    p.n_dn = nS > 0.0 ? A * fd_hm1<D>(nu2) : p.n_up;
    p.status = 0;
    return p;
}

// Newton's method on
//   r_1 = log F_{h-1}(nu_up) - h t + h log 2 pi - log n_up
//   r_2 = log F_{h-1}(nu_dn) - h t + h log 2 pi - log n_dn
//   r_3 = log(F_h(nu_up) + F_h(nu_dn)) - (h+1) t + h log 2 pi - log(n eps / h),
// t = log beta.  With g_s = F_{h-2}/F_{h-1}(nu_s) and c_s = F_{h-1}(nu_s)/sum F_h
// the Jacobian is [[-h, g_up, 0], [-h, 0, g_dn], [-(h+1), c_up, c_dn]]; its
// Schur complement -(h+1) + h sum_s c_s/g_s is negative (positive heat
// capacity), so the step is always defined.
template <int D>
__device__ FdParams fd_params_site(double n, double Sx, double Sy, double Sz, double eps)
{
    constexpr double h = 0.5 * D;
    constexpr double hl2pi = h * 1.8378770664093453;   // h log 2 pi
    FdParams p;
    p.beta = p.mu_up = p.mu_dn = p.ax = p.ay = p.az = p.n_up = p.n_dn = CUDART_NAN;
    const double nS = sqrt(Sx * Sx + Sy * Sy + Sz * Sz);
    const double nup = 0.5 * (n + nS), ndn = 0.5 * (n - nS);
    if (!(ndn > 0.0)) {
        p.status = 1;
        return p;
    }
    if (nS > 0.0) {
        p.ax = Sx / nS;
        p.ay = Sy / nS;
        p.az = Sz / nS;
    } else {
        p.ax = p.ay = p.az = 0.0;
    }
    if (!(eps > 0.0)) {
        p.status = 2;
        return p;
    }
    const bool split = nS > 0.0;
    const double lA = log(nup), lB = split ? log(ndn) : lA, lC = log(n * eps / h);
    double t = log(h / eps);
    double nu1 = lA - hl2pi + h * t, nu2 = lB - hl2pi + h * t;
    // start from the single-precision solution (~1e-6) where it settles: two
    // double iterations then reach rounding level instead of four
    float tf, n1f, n2f;
    if (fd_newton_f<D>((float)nup, (float)ndn, (float)n, (float)eps, tf, n1f, n2f)) {
        t = tf;
        nu1 = n1f;
        nu2 = split ? (double)n2f : nu1;
    }
    Fd3 F1, F2;
    bool settled = false;
    for (int it = 0;; ++it) {
        F1 = fd3<D>(nu1);
        F2 = split ? fd3<D>(nu2) : F1;
        if (settled || it == 40) break;
        const double sFh = F1.h + F2.h;
        const double r1 = log(F1.m1) - h * t + hl2pi - lA;
        const double r2 = split ? log(F2.m1) - h * t + hl2pi - lB : r1;
        const double r3 = log(sFh) - (h + 1.0) * t + hl2pi - lC;
        const double ig1 = F1.m1 / F1.m2, ig2 = F2.m1 / F2.m2;   // 1/g_s
        const double c1 = F1.m1 / sFh, c2 = F2.m1 / sFh;
        const double den = -(h + 1.0) + h * (c1 * ig1 + c2 * ig2);
        double dt = (c1 * ig1 * r1 + c2 * ig2 * r2 - r3) / den;
        if (!(dt == dt)) break;
        dt = fmax(-1.0, fmin(1.0, dt));
        const double d1 = fmax(-10.0, fmin(10.0, (h * dt - r1) * ig1));
        const double d2 = fmax(-10.0, fmin(10.0, (h * dt - r2) * ig2));
        t += dt;
        nu1 += d1;
        nu2 = split ? nu2 + d2 : nu1;
        // quadratic convergence: once a step is below 1e-9 the iterate is exact
        // to rounding; one more evaluation gives the outputs at it
        settled = fmax(fabs(dt), fmax(fabs(d1), fabs(d2))) <= 1e-9;
    }
    if (!settled) return fd_params_nested<D>(n, Sx, Sy, Sz, eps);
    const double A = exp(hl2pi - h * t);
    p.beta = exp(t);
    p.mu_up = nu1 / p.beta;
    p.mu_dn = nu2 / p.beta;
    p.n_up = A * F1.m1;
    p.n_dn = A * F2.m1;
    p.status = 0;
    return p;
}

// ---------------------------------------------------------------------------
// Single-precision solve (fd_newton_f, float tables FDF_*).  Parameters come
// out to ~1e-6 relative; the
// spin splitting mu_up - mu_dn, a difference of two solved numbers, to
// ~1e-6 |mu| absolute -- what float outputs can hold (a double solve would
// not survive their rounding).  Sites where the float iteration does not
// settle, and invalid ones, go through the double solve (fd_params_site),
// which also decides their status.
// ---------------------------------------------------------------------------
struct FdParamsF {
    float beta, mu_up, mu_dn, ax, ay, az;
    int status;   // as FdParams
};

template <int D>
__device__ FdParamsF fd_params_site_f(float n, float Sx, float Sy, float Sz, float eps)
{
    FdParamsF p;
    const float nS = sqrtf(Sx * Sx + Sy * Sy + Sz * Sz);
    float t, nu1, nu2;
    if (!fd_newton_f<D>(0.5f * (n + nS), 0.5f * (n - nS), n, eps, t, nu1, nu2)) {
        // invalid or unsettled: the double solve decides
        const FdParams q = fd_params_site<D>(n, Sx, Sy, Sz, eps);
        p.beta = (float)q.beta;
        p.mu_up = (float)q.mu_up;
        p.mu_dn = (float)q.mu_dn;
        p.ax = (float)q.ax;
        p.ay = (float)q.ay;
        p.az = (float)q.az;
        p.status = q.status;
        return p;
    }
    const float rS = nS > 0.f ? 1.f / nS : 0.f;
    p.beta = expf(t);
    p.mu_up = nu1 / p.beta;
    p.mu_dn = nu2 / p.beta;
    p.ax = Sx * rS;
    p.ay = Sy * rS;
    p.az = Sz * rS;
    p.status = 0;
    return p;
}

}  // namespace qlbm
