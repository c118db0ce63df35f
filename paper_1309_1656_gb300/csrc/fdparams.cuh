// Parameters of the matrix-valued Fermi-Dirac equilibrium of one site
// (Sec. 2.2, Prop. 1; Eqs. rhoFDstdOmega, nFDstdOmega, energyFDstdOmega),
// in double precision on the GPU.
//
// Given the site's density matrix rho = (n 1 + S.sigma)/2 and internal energy
// eps: the analytic 2x2 eigen-decomposition gives the occupations
// n_up/dn = (n +- |S|)/2 and the Bloch axis S/|S| of U (Sec. 2.2, "U ... can
// be recovered by diagonalizing rho"); then (beta, nu_up, nu_dn), nu = beta mu,
// solve
//   n_s = (2 pi/beta)^h F_{h-1}(nu_s),   n eps = h beta^-1 (2 pi/beta)^h sum_s F_h(nu_s),
// h = d/2.  For a trial beta each species is inverted on its own (closed form
// in 2D, F_0(nu) = log(1 + e^nu); Newton on log F_{1/2} in 3D), and beta is
// found by a bracketed Newton iteration on log beta of the energy equation,
// using d nu_s / d beta = h F_{h-1}(nu_s) / (beta F_{h-2}(nu_s)) (from
// dF_k/dx = F_{k-1}).
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
    int status;   // 0 ok, 1 rho not positive definite, 2 no beta fits / no convergence
};

template <int D>
__device__ FdParams fd_params_site(double n, double Sx, double Sy, double Sz, double eps)
{
    constexpr double h = 0.5 * D;
    FdParams p;
    p.beta = p.mu_up = p.mu_dn = p.ax = p.ay = p.az = CUDART_NAN;
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
    p.status = 0;
    return p;
}

}  // namespace qlbm
