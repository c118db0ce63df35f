// Kernels of the Fermi-Dirac parameter recovery: the per-site side output and
// the double-precision step variant whose equilibrium is built through the
// recovered parameters (Eq. WeqDiscr) instead of directly from rho
// (Eq. WeqAlgo).  The two equilibria agree to the accuracy of the solve,
// U diag(n_up, n_dn) U* = rho (Sec. 3.3).
#pragma once

#include "fdparams.cuh"
#include "kernels.cuh"

namespace qlbm {

struct FdArgs {
    double beta0, xi;
};

// Per-site (beta, mu_up, mu_dn, Bloch axis) of the current state.
template <int D, class Codec, bool SWAPPED>
__global__ void __launch_bounds__(kStepBlock)
k_fd_params(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Codec codec, FdArgs a,
            double *__restrict__ beta, double *__restrict__ mu_up, double *__restrict__ mu_dn,
            double *__restrict__ axis, unsigned long long *__restrict__ nfail)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    R f[Q], sx[Q], sy[Q], sz[Q];
    gather<D, Codec, SWAPPED>(pl, g, si, codec, f, sx, sy, sz);
    double fd[Q], xd[Q], yd[Q], zd[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cls = cnorm2<D>(q);
        fd[q] = codec.to_double(f[q], 0, cls);
        xd[q] = codec.to_double(sx[q], 1, cls);
        yd[q] = codec.to_double(sy[q], 2, cls);
        zd[q] = codec.to_double(sz[q], 3, cls);
    }
    const SiteMoments<D, double> m = site_moments<D, double>(fd, xd, yd, zd);
    const double eps = 0.5 * a.xi * a.xi * (m.e2n - (m.jx * m.jx + m.jy * m.jy + m.jz * m.jz));
    const FdParams p = fd_params_site<D>(m.n, m.Sx, m.Sy, m.Sz, eps);
    const int64_t N = g.N, s = si.s;
    if (beta) beta[s] = p.beta;
    if (mu_up) mu_up[s] = p.mu_up;
    if (mu_dn) mu_dn[s] = p.mu_dn;
    if (axis) {
        axis[s] = p.ax;
        axis[N + s] = p.ay;
        axis[2 * N + s] = p.az;
    }
    if (p.status != 0) atomicAdd(nfail, 1ull);
}

// Reverse mode of qlbm_fd_params by the implicit-function rule.  The
// parameters p = (beta, nu_up, nu_dn), nu = beta mu, solve G(p; m) = 0 with
// m = (n_up, n_dn, E = n eps) and
//   G_s = A F_{h-1}(nu_s) - n_s,  G_3 = h beta^-1 A sum_s F_h(nu_s) - E,  A = (2 pi/beta)^h,
// so dp/dm = J^-1 with J = dG/dp (dG/dm = -1), and a cotangent pbar of p
// gives mbar = J^-T pbar.  Then n_up/dn = (n +- |S|)/2, axis = S/|S| and
// E = xi^2/2 (E2 - |J_lat|^2/n) (J_lat = sum i f, E2 = sum |i|^2 f) carry it
// to the populations: lambda_f,i = nbar + i.Jbar + |i|^2 E2bar, lambda_s,i = Sbar.
// Output: the cotangent of the current state in the canonical layout.
template <int D, class Codec, bool SWAPPED>
__global__ void __launch_bounds__(kStepBlock)
k_fd_params_adjoint(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Codec codec, FdArgs a,
                    const double *__restrict__ gbeta, const double *__restrict__ gmu_up,
                    const double *__restrict__ gmu_dn, const double *__restrict__ gaxis,
                    double *__restrict__ lam)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    constexpr double h = 0.5 * D;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    R f[Q], sx[Q], sy[Q], sz[Q];
    gather<D, Codec, SWAPPED>(pl, g, si, codec, f, sx, sy, sz);
    double fd[Q], xd[Q], yd[Q], zd[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cls = cnorm2<D>(q);
        fd[q] = codec.to_double(f[q], 0, cls);
        xd[q] = codec.to_double(sx[q], 1, cls);
        yd[q] = codec.to_double(sy[q], 2, cls);
        zd[q] = codec.to_double(sz[q], 3, cls);
    }
    const SiteMoments<D, double> m = site_moments<D, double>(fd, xd, yd, zd);
    const double jj = m.jx * m.jx + m.jy * m.jy + m.jz * m.jz;
    const double eps = 0.5 * a.xi * a.xi * (m.e2n - jj);
    const FdParams p = fd_params_site<D>(m.n, m.Sx, m.Sy, m.Sz, eps);
    const int64_t N = g.N, s = si.s;
    double nbar = 0.0, Sbx = 0.0, Sby = 0.0, Sbz = 0.0, Jbx = 0.0, Jby = 0.0, Jbz = 0.0, E2bar = 0.0;
    if (p.status == 0) {
        const double beta = p.beta, nu1 = beta * p.mu_up, nu2 = beta * p.mu_dn;
        const double bb = gbeta ? gbeta[s] : 0.0, b1 = gmu_up ? gmu_up[s] : 0.0, b2 = gmu_dn ? gmu_dn[s] : 0.0;
        // cotangent of (beta, nu_up, nu_dn)
        const double pb0 = bb - (b1 * p.mu_up + b2 * p.mu_dn) / beta, pb1 = b1 / beta, pb2 = b2 / beta;
        const double A = pow(kTwoPi / beta, h);
        const Fd3 G1 = fd3<D>(nu1), G2 = fd3<D>(nu2);
        const double F1 = G1.m1, F2 = G2.m1, Fh = G1.h + G2.h;
        // J rows: G1, G2, G3; columns: beta, nu_up, nu_dn
        const double J00 = -h / beta * A * F1, J01 = A * G1.m2;
        const double J10 = -h / beta * A * F2, J12 = A * G2.m2;
        const double J20 = -(h + 1.0) / beta * h / beta * A * Fh, J21 = h / beta * A * F1, J22 = h / beta * A * F2;
        // solve J^T mbar = pbar:
        //   J00 m0 + J10 m1 + J20 m2 = pb0
        //   J01 m0 +            J21 m2 = pb1
        //              J12 m1 + J22 m2 = pb2
        // m0 = (pb1 - J21 m2)/J01, m1 = (pb2 - J22 m2)/J12, substitute into the first
        const double den = J20 - J00 * J21 / J01 - J10 * J22 / J12;
        const double m2 = (pb0 - J00 * pb1 / J01 - J10 * pb2 / J12) / den;
        const double m0 = (pb1 - J21 * m2) / J01, m1 = (pb2 - J22 * m2) / J12;
        nbar = 0.5 * (m0 + m1);
        const double nS = sqrt(m.Sx * m.Sx + m.Sy * m.Sy + m.Sz * m.Sz);
        if (nS > 0.0) {
            const double sbar = 0.5 * (m0 - m1);
            double ax = 0.0, ay = 0.0, az = 0.0;
            if (gaxis) {
                ax = gaxis[s];
                ay = gaxis[N + s];
                az = gaxis[2 * N + s];
            }
            const double adot = ax * p.ax + ay * p.ay + az * p.az;
            Sbx = sbar * p.ax + (ax - adot * p.ax) / nS;
            Sby = sbar * p.ay + (ay - adot * p.ay) / nS;
            Sbz = sbar * p.az + (az - adot * p.az) / nS;
        }
        // E = xi^2/2 (E2 - |J_lat|^2 / n): its cotangent m2
        const double c = 0.5 * a.xi * a.xi * m2;
        E2bar = c;
        Jbx = -2.0 * c * m.jx;
        Jby = -2.0 * c * m.jy;
        Jbz = -2.0 * c * m.jz;
        nbar += c * jj;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        double *o = lam + (int64_t)(4 * q) * N + s;
        o[0] = nbar + cx<D>(q) * Jbx + cy<D>(q) * Jby + cz<D>(q) * Jbz + cnorm2<D>(q) * E2bar;
        o[N] = Sbx;
        o[2 * N] = Sby;
        o[3 * N] = Sbz;
    }
}

// Equilibrium initial state from physical Fermi-Dirac parameters: per site
// n_s = (2 pi/beta)^h F_{h-1}(beta mu_s) (Eq. nFDstdOmega),
// eps = h beta^-1 sum_s F_h(beta mu_s) / sum_s F_{h-1}(beta mu_s)
// (Eq. energyFDstdOmega), rho = U diag(n_up, n_dn) U* with U's Bloch axis
// `axis` (tr rho = n_up + n_dn, S = (n_up - n_dn) axis), and W_i = W_i^eq of
// Eq. WeqAlgo with the given velocity.
template <int D, class Codec>
__global__ void __launch_bounds__(kStepBlock)
k_init_fd(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, InitConsts ic, Codec codec,
          const double *__restrict__ beta, const double *__restrict__ mu_up, const double *__restrict__ mu_dn,
          const double *__restrict__ axis, const double *__restrict__ u)
{
    constexpr int Q = Lattice<D>::Q;
    constexpr double h = 0.5 * D;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    const int64_t N = g.N, s = si.s;
    const double b = beta[s], nu1 = b * mu_up[s], nu2 = b * mu_dn[s];
    const double pre = pow(kTwoPi / b, h);
    const Fd3 G1 = fd3<D>(nu1), G2 = fd3<D>(nu2);
    const double F1 = G1.m1, F2 = G2.m1;
    const double nup = pre * F1, ndn = pre * F2;
    const double n = nup + ndn;
    const double e = h / b * (G1.h + G2.h) / (F1 + F2);
    const double Sx = (nup - ndn) * axis[s], Sy = (nup - ndn) * axis[N + s], Sz = (nup - ndn) * axis[2 * N + s];
    const double jx = u[s] / ic.xi, jy = u[N + s] / ic.xi, jz = (D == 3) ? u[2 * N + s] / ic.xi : 0.0;
    const double be = ic.beta0 * e;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cls = cnorm2<D>(q);
        const double wp = ic.w[cls] * poly_P_d<D>(ic, q, jx, jy, jz, be);
        codec.store4(pl.p[q] + s, codec.load(codec.from_double(wp * n, 0, cls)),
                     codec.load(codec.from_double(wp * Sx, 1, cls)), codec.load(codec.from_double(wp * Sy, 2, cls)),
                     codec.load(codec.from_double(wp * Sz, 3, cls)));
    }
}

// Collision whose equilibrium density matrix is rebuilt from the recovered
// parameters: rho' = U diag(n_up', n_dn') U*, n_s' = (2 pi/beta)^h F_{h-1}(beta mu_s)
// (Eq. WeqDiscr), i.e. n' = n_up' + n_dn', S' = (n_up' - n_dn') axis; u and
// eps (hence P_i) are the site's moments as in Eq. WeqAlgo.  A site whose
// parameters cannot be recovered keeps rho' = rho and is counted.
template <int D>
__device__ __forceinline__ unsigned collide_fd(double *f, double *sx, double *sy, double *sz,
                                               const Coll<double> &k, const FdArgs &a)
{
    constexpr int Q = Lattice<D>::Q;
    SiteMoments<D, double> m = site_moments<D, double>(f, sx, sy, sz);
    const double jj = m.jx * m.jx + m.jy * m.jy + m.jz * m.jz;
    const double be = k.K * (m.e2n - jj);   // beta0 * eps
    double n2 = m.n, Sx2 = m.Sx, Sy2 = m.Sy, Sz2 = m.Sz;
    unsigned flag = 0u;
    const FdParams p = fd_params_site<D>(m.n, m.Sx, m.Sy, m.Sz, be / a.beta0);
    if (p.status == 0) {
        const double nu = p.n_up, nd = p.n_dn;
        n2 = nu + nd;
        Sx2 = (nu - nd) * p.ax;
        Sy2 = (nu - nd) * p.ay;
        Sz2 = (nu - nd) * p.az;
    } else {
        flag |= FLAG_FD_UNRESOLVED;
    }
    const double a2 = (be - k.c) * k.inv_mc2;
    const double a1 = 1.0 - k.c * a2;
    const double b0 = fma(k.c5, jj, a1);
    const double a2K = a2 * k.K;
    const double bq[3] = {b0, b0 + a2K, b0 + 2.0 * a2K};
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const double t = cx<D>(q) * m.jx + cy<D>(q) * m.jy + cz<D>(q) * m.jz;
        const double hq = k.w[cnorm2<D>(q)] * fma(t, fma(k.c4, t, k.c3), bq[cnorm2<D>(q)]);
        f[q] = fma(k.omega, fma(hq, n2, -f[q]), f[q]);
        sx[q] = fma(k.omega, fma(hq, Sx2, -sx[q]), sx[q]);
        sy[q] = fma(k.omega, fma(hq, Sy2, -sy[q]), sy[q]);
        sz[q] = fma(k.omega, fma(hq, Sz2, -sz[q]), sz[q]);
    }
    if (!(m.n > 0.0)) flag |= (m.n == m.n) ? FLAG_NONPOSITIVE : FLAG_NONFINITE;
    return flag;
}

template <int D, bool ODD, int FIELD>
__global__ void __launch_bounds__(kStepBlock)
k_step_aa_fd(const Planes<double, Lattice<D>::Q> pl, Grid g, Coll<double> k, FdArgs a,
             unsigned *__restrict__ flags)
{
    constexpr int Q = Lattice<D>::Q;
    const CodecF64 codec;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    double f[Q], sx[Q], sy[Q], sz[Q];
    gather<D, CodecF64, ODD>(pl, g, si, codec, f, sx, sy, sz);
    const unsigned flag = collide_fd<D>(f, sx, sy, sz, k, a);
    apply_field<D, FIELD, double>(sx, sy, sz, k, si.s);
    SiteIdx so = si;
    so.s += g.zero;
    so.x += g.zero;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int slot = ODD ? q : opposite<D>(q);
        const int s = ODD ? neighbour(g, so, cx<D>(q), cy<D>(q), cz<D>(q)) : so.s;
        stq(pl.p[slot] + s, f[q], sx[q], sy[q], sz[q]);
    }
    if (flag) atomicOr(flags, flag);
}

// One single-precision AA step (the step kernel's collision and addressing,
// bit for bit) that also writes the Fermi-Dirac parameters of the state it
// started from: after the stores, the site's conserved moments (which the
// collision leaves unchanged) go through the single-precision solve
// (fd_params_site_f; double near degenerate eigenvalues).  The solve runs
// while the stores drain.  Outputs float [N] (axis [3][N]).
template <int D, class Codec, bool ODD, int FIELD>
__global__ void __launch_bounds__(kStepBlock, step_min_blocks<D, Codec>())
k_step_aa_fdout(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Coll<float> k, Codec codec,
                float beta0, unsigned *__restrict__ flags, float *__restrict__ beta, float *__restrict__ mu_up,
                float *__restrict__ mu_dn, float *__restrict__ axis, unsigned long long *__restrict__ nfail)
{
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    float f[Q], sx[Q], sy[Q], sz[Q];
    gather<D, Codec, ODD>(pl, g, si, codec, f, sx, sy, sz);
    float mom[5];
    const unsigned flag = collide_dev<D, true>(f, sx, sy, sz, k, mom);
    apply_field<D, FIELD, float>(sx, sy, sz, k, si.s);
    SiteIdx so = si;
    so.s += g.zero;
    so.x += g.zero;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int slot = ODD ? q : opposite<D>(q);
        const int s = ODD ? neighbour(g, so, cx<D>(q), cy<D>(q), cz<D>(q)) : so.s;
        codec.store4(pl.p[slot] + s, f[q], sx[q], sy[q], sz[q]);
    }
    if (flag) atomicOr(flags, flag);
    const FdParamsF p = fd_params_site_f<D>(mom[0], mom[1], mom[2], mom[3], mom[4] / beta0);
    const int64_t N = g.N, s = si.s;
    beta[s] = p.beta;
    mu_up[s] = p.mu_up;
    mu_dn[s] = p.mu_dn;
    axis[s] = p.ax;
    axis[N + s] = p.ay;
    axis[2 * N + s] = p.az;
    if (p.status != 0) atomicAdd(nfail, 1ull);
}

}  // namespace qlbm
