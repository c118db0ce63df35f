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
    constexpr double h = 0.5 * D;
    SiteMoments<D, double> m = site_moments<D, double>(f, sx, sy, sz);
    const double jj = m.jx * m.jx + m.jy * m.jy + m.jz * m.jz;
    const double be = k.K * (m.e2n - jj);   // beta0 * eps
    double n2 = m.n, Sx2 = m.Sx, Sy2 = m.Sy, Sz2 = m.Sz;
    unsigned flag = 0u;
    const FdParams p = fd_params_site<D>(m.n, m.Sx, m.Sy, m.Sz, be / a.beta0);
    if (p.status == 0) {
        const double pre = pow(kTwoPi / p.beta, h);
        const double nu = pre * fd_hm1<D>(p.beta * p.mu_up), nd = pre * fd_hm1<D>(p.beta * p.mu_dn);
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

template <int D, bool ODD>
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
    SiteIdx so = si;
    so.s += g.zero;
    so.x += g.zero;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int slot = ODD ? q : opposite<D>(q);
        const int s = ODD ? neighbour(g, so, cx<D>(q), cy<D>(q), cz<D>(q)) : so.s;
        pl.p[4 * slot][s] = f[q];
        pl.p[4 * slot + 1][s] = sx[q];
        pl.p[4 * slot + 2][s] = sy[q];
        pl.p[4 * slot + 3][s] = sz[q];
    }
    if (flag) atomicOr(flags, flag);
}

}  // namespace qlbm
