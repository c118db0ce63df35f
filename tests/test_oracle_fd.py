"""Pins of the oracle's Fermi-Dirac integrals and parameter inversion
(Sec. 2.2: Eqs. rhoFDstdOmega, nFDstdOmega, energyFDstdOmega, Prop. 1).

F_k is checked against what fixes it independently of the oracle's
quadrature: the derivative relation dF_k/dx = F_{k-1} stated in the paper
(which ties F_1 to the closed form F_0 and F_{1/2} to F_{-1/2}), the values
F_k(0) = (1 - 2^-k) zeta(k+1), the dilogarithm (F_1 = -Li_2(-e^x)), the
classical and degenerate limits, and mpmath's polylogarithm.  The forward
map (n_s, eps) of the parameters is checked against direct numerical
integration of the Fermi-Dirac distribution in d dimensions, and the
inversion by round trips from known parameters.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

KS = [-0.5, 0.5, 1.0, 1.5]


@pytest.mark.parametrize("k", KS)
def test_fd_at_zero(oracle_mod, k):
    eta = math.log(2.0) if k == 0 else (1.0 - 2.0 ** (-k)) * special.zeta(k + 1.0)
    assert oracle_mod.fd(k, 0.0) == pytest.approx(eta, rel=2e-15)


@pytest.mark.parametrize("k", [0.5, 1.0, 1.5])
def test_fd_derivative_relation(oracle_mod, k):
    h = 1e-4
    for x in (-8.0, -1.3, 0.4, 2.7, 11.0, 35.0):
        d = (oracle_mod.fd(k, x + h) - oracle_mod.fd(k, x - h)) / (2 * h)
        assert d == pytest.approx(oracle_mod.fd(k - 1.0, x), rel=1e-8), (k, x)


def test_fd1_is_dilogarithm(oracle_mod):
    # F_1(x) = -Li_2(-e^x), Li_2(z) = spence(1 - z)
    for x in np.linspace(-20, 30, 41):
        ref = -special.spence(1.0 + math.exp(x))
        assert oracle_mod.fd(1.0, x) == pytest.approx(ref, rel=1e-13), x


@pytest.mark.parametrize("k", KS)
def test_fd_limits(oracle_mod, k):
    # classical: F_k(x) = e^x - e^{2x}/2^{k+1} + ...
    x = -12.0
    assert oracle_mod.fd(k, x) == pytest.approx(math.exp(x) - math.exp(2 * x) / 2 ** (k + 1), rel=1e-14)
    # degenerate (Sommerfeld): x^{k+1}/Gamma(k+2) [1 + pi^2/6 (k+1)k/x^2
    #                                             + 7 pi^4/360 (k+1)k(k-1)(k-2)/x^4]
    x = 150.0   # the next Sommerfeld term is below 1e-11 here
    som = x ** (k + 1) / math.gamma(k + 2) * (1 + math.pi ** 2 / 6 * (k + 1) * k / x ** 2 +
                                              7 * math.pi ** 4 / 360 * (k + 1) * k * (k - 1) * (k - 2) / x ** 4)
    assert oracle_mod.fd(k, x) == pytest.approx(som, rel=1e-11)


@pytest.mark.parametrize("k", [-0.5, 0.5, 1.5])
def test_fd_against_polylog(oracle_mod, k):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for x in np.linspace(-40, 45, 35):
        ref = float(-mp.polylog(k + 1, -mp.exp(x)).real)
        assert oracle_mod.fd(k, x) == pytest.approx(ref, rel=3e-15), x


def _fd_distribution_moments(d, beta, mu):
    """n and sum |p|^2/2 of (exp(beta(|p|^2/2 - mu)) + 1)^-1 on R^d, by
    radial quadrature (independent of the F_k route)."""
    area = 2 * math.pi ** (d / 2) / math.gamma(d / 2)
    f = lambda r: special.expit(-beta * (0.5 * r * r - mu))
    top = math.sqrt(2 * max(mu, 0.0) + 120.0 / beta)
    n = area * integrate.quad(lambda r: r ** (d - 1) * f(r), 0, top, epsabs=0, epsrel=1e-13, limit=400)[0]
    e = area * integrate.quad(lambda r: 0.5 * r * r * r ** (d - 1) * f(r), 0, top, epsabs=0, epsrel=1e-13,
                              limit=400)[0]
    return n, e


@pytest.mark.parametrize("d", [2, 3])
def test_fd_moments_against_direct_integration(oracle_mod, d):
    for beta, mu_up, mu_dn in ((1.0, -1.5, -2.5), (0.7, 0.2, -0.35), (2.3, 1.4, 0.3)):
        nu, nd, eps = oracle_mod.fd_moments(d, beta, mu_up, mu_dn)
        n1, e1 = _fd_distribution_moments(d, beta, mu_up)
        n2, e2 = _fd_distribution_moments(d, beta, mu_dn)
        assert nu == pytest.approx(n1, rel=1e-11)
        assert nd == pytest.approx(n2, rel=1e-11)
        assert eps == pytest.approx((e1 + e2) / (n1 + n2), rel=1e-11)


def _rho_of(oracle_mod, d, beta, mu_up, mu_dn, axis):
    nu, nd, eps = oracle_mod.fd_moments(d, beta, mu_up, mu_dn)
    a = np.asarray(axis, float)
    return np.r_[nu + nd, (nu - nd) * a], eps


@pytest.mark.parametrize("d", [2, 3])
def test_fd_params_round_trip(oracle_mod, d):
    rng = np.random.default_rng(d)
    for _ in range(8):
        beta = rng.uniform(0.3, 3.0)
        mu_up = rng.uniform(-4.0, 2.0)
        mu_dn = mu_up - rng.uniform(0.05, 2.0)
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        rho4, eps = _rho_of(oracle_mod, d, beta, mu_up, mu_dn, axis)
        rc, out = oracle_mod.fd_params(d, rho4, eps)
        assert rc == 0
        assert out[0] == pytest.approx(beta, rel=1e-10)
        assert out[1] == pytest.approx(mu_up, rel=1e-9, abs=1e-10)
        assert out[2] == pytest.approx(mu_dn, rel=1e-9, abs=1e-10)
        assert np.allclose(out[3:], axis, atol=1e-10)


def test_fd_params_degenerate_and_invalid(oracle_mod):
    # equal chemical potentials: rho ~ 1, no preferred axis
    rho4, eps = _rho_of(oracle_mod, 3, 1.2, -1.0, -1.0, [0, 0, 1])
    rc, out = oracle_mod.fd_params(3, rho4, eps)
    assert rc == 0 and out[1] == pytest.approx(-1.0, rel=1e-10) and out[2] == pytest.approx(-1.0, rel=1e-10)
    assert np.all(out[3:] == 0.0)
    # not positive definite
    rc, out = oracle_mod.fd_params(3, np.array([1.0, 0.0, 0.0, 1.2]), 1.0)
    assert rc == 1 and np.all(np.isnan(out[:3]))
    # energy below the degenerate (zero-temperature) limit
    rc, out = oracle_mod.fd_params(3, np.array([1.0, 0.0, 0.0, 0.0]), 1e-6)
    assert rc == 2 and np.isnan(out[0])
