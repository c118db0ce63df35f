// Lattice constants of the quadrature (Sec. 3.1) and of the polynomial
// equilibrium (Sec. 3.2), computed on the host in double.
//
// The library derives them from the defining moment conditions rather than
// from the printed closed forms.  Write <.> for the mean under the weight
// (exp(beta0 w) + 1)^-1, w = |p|^2/2, at mu0 = 0 (Eq. Ih), h = d/2, and
//   c = beta0 <w> = h F_h(0)/F_{h-1}(0),
//   m = beta0^2 <w^2> = h(h+1) F_{h+1}(0)/F_{h-1}(0),
// using F_k(0) = -Li_{k+1}(-1) = (1 - 2^-k) zeta(k+1), F_0(0) = log 2
// (Sec. 2.2).
//
// Quadrature (Eqs. quadrature2D/3D).  By symmetry the degree-5 conditions
// reduce to <1>, <p1^2>, <p1^4> and <p1^2 p2^2>.  Isotropy gives
// <p1^4> = 3 <p1^2 p2^2>, which fixes the ratio of axis to diagonal weights
// (w_axis = 4 w_diag on D2Q9, 2 w_diag on D3Q19), and then
//   xi^2 = <p1^4>/<p1^2> = 6 m / ((d+2) c beta0),
//   a = w_axis = <p1^2> / (k xi^2),  <p1^2> = 2c/(d beta0),  k = 3 (D2Q9), 6 (D3Q19),
//   w_rest = 1 - (sum of the other weights).
// Equilibrium (Eq. WeqPoly, appendix).  Requiring sum w_i P_i = 1,
// sum w_i e_i P_i = u and sum w_i |e_i|^2/2 P_i = eps + |u|^2/2 for all u
// gives
//   alpha3 = d/(2c),  alpha4 = d/(4(m - c^2)),  alpha5 = -(4c/d) alpha4,
//   alpha2 = (beta0 eps - c)/(m - c^2),  alpha1 = 1 - c alpha2.
#include <math.h>

#include "internal.h"

namespace qlbm {

// Riemann zeta for real s > 1 by Euler-Maclaurin summation: the first
// n-1 terms, the integral tail, the half term and eight Bernoulli
// corrections (error far below double rounding for n = 16, s <= 4).
static double zeta_em(double s)
{
    const int n = 16;
    static const double B2j[8] = {1.0 / 6.0,   -1.0 / 30.0, 1.0 / 42.0,      -1.0 / 30.0,
                                  5.0 / 66.0,  -691.0 / 2730.0, 7.0 / 6.0, -3617.0 / 510.0};
    double sum = 0.0;
    for (int k = n - 1; k >= 1; --k) sum += pow((double)k, -s);
    const double N = (double)n;
    sum += pow(N, 1.0 - s) / (s - 1.0) + 0.5 * pow(N, -s);
    // term_j = B_2j/(2j)! * s(s+1)...(s+2j-2) * N^(-s-2j+1)
    double rising = s;          // s (s+1) ... (s+2j-2)
    double fact = 2.0;          // (2j)!
    double npow = pow(N, -s - 1.0);
    for (int j = 1; j <= 8; ++j) {
        sum += B2j[j - 1] / fact * rising * npow;
        rising *= (s + 2 * j - 1) * (s + 2 * j);
        fact *= (double)(2 * j + 1) * (double)(2 * j + 2);
        npow /= N * N;
    }
    return sum;
}

// Complete Fermi-Dirac integral at zero argument.
static double fd_at_zero(double k)
{
    if (k == 0.0) return log(2.0);
    return (1.0 - pow(2.0, -k)) * zeta_em(k + 1.0);
}

int compute_constants(int d, double beta0, HostConsts *o)
{
    if ((d != 2 && d != 3) || !(beta0 > 0.0)) return -1;
    const double h = 0.5 * d;
    const double Fm1 = fd_at_zero(h - 1.0), F0 = fd_at_zero(h), F1 = fd_at_zero(h + 1.0);
    o->d = d;
    o->b = (d == 2) ? 9 : 19;
    o->beta0 = beta0;
    o->c = h * F0 / Fm1;
    o->m = h * (h + 1.0) * F1 / Fm1;
    const double xi2 = 6.0 * o->m / ((d + 2.0) * o->c * beta0);
    o->xi = sqrt(xi2);
    const double p1sq = 2.0 * o->c / (d * beta0);
    const double kk = (d == 2) ? 3.0 : 6.0;
    o->a = p1sq / (kk * xi2);
    o->w[1] = o->a;
    o->w[2] = (d == 2) ? o->a / 4.0 : o->a / 2.0;
    o->w[0] = (d == 2) ? 1.0 - 4.0 * o->w[1] - 4.0 * o->w[2] : 1.0 - 6.0 * o->w[1] - 12.0 * o->w[2];
    o->alpha3 = d / (2.0 * o->c);
    o->alpha4 = d / (4.0 * (o->m - o->c * o->c));
    o->alpha5 = -(4.0 * o->c / d) * o->alpha4;
    o->K = 0.5 * beta0 * xi2;
    o->eps0 = o->c / beta0;
    return 0;
}

}  // namespace qlbm
