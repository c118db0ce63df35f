"""Pins of the oracle's lattice constants (Sec. 3.1, Sec. 3.2, appendix).

Each check ties the oracle to something other than itself: the decimals the
paper prints, closed forms of the zeta function, the defining moment
conditions of the Fermi-Dirac cubature computed by independent numerical
integration, and the moment identities the polynomial equilibrium must
satisfy by construction.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import expit, gamma

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "printed_constants.txt")


def _printed():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, d, val = line.split()[:3]
        rows.append((name, int(d), val))
    return rows


@pytest.mark.parametrize("name,d,val", _printed())
def test_printed_constants(oracle_mod, name, d, val):
    c = oracle_mod.constants(d, 1.0)
    got = {"a": c["a"], "xi_sqrt_beta0": c["xi"], "xi_at_beta0_1": c["xi"],
           "alpha_fac": c["alpha_fac"]}[name]
    decimals = len(val.split(".")[1])
    assert abs(got - float(val)) <= 0.5 * 10.0 ** (-decimals), (name, d, got, val)


def test_xi_scales_as_inverse_sqrt_beta0(oracle_mod):
    # Eqs. QuadSolution2Dmu0/3Dmu0: xi = const / sqrt(beta0)
    for d in (2, 3):
        x1 = oracle_mod.constants(d, 1.0)["xi"]
        for b0 in (0.8, 1.2, 3.0):
            assert oracle_mod.constants(d, b0)["xi"] == pytest.approx(x1 / math.sqrt(b0), rel=1e-15)


def test_zeta_closed_forms_and_library(oracle_mod):
    # Euler's closed forms and scipy's independent implementation.
    from scipy.special import zeta as sz
    assert oracle_mod.zeta(2.0) == pytest.approx(math.pi ** 2 / 6, rel=1e-15)
    assert oracle_mod.zeta(4.0) == pytest.approx(math.pi ** 4 / 90, rel=1e-15)
    assert oracle_mod.zeta(6.0) == pytest.approx(math.pi ** 6 / 945, rel=1e-15)
    for s in (1.5, 2.5, 3.0, 3.5):
        assert oracle_mod.zeta(s) == pytest.approx(float(sz(s, 1)), rel=2e-15)


def test_lattice_tables(oracle_mod):
    # D2Q9: 9 directions {-1,0,1}^2; D3Q19: |i1|+|i2|+|i3| <= 2 (Sec. 3.1).
    for d, b in ((2, 9), (3, 19)):
        c = oracle_mod.constants(d, 1.0)
        assert c["b"] == b
        idx = c["idx"]
        assert len({tuple(r) for r in idx}) == b
        assert np.all(np.abs(idx).sum(axis=1) <= 2)
        # opposite of q is b-1-q
        assert np.array_equal(idx[::-1], -idx)
        # enumeration order: i1 varies fastest, then i2, then i3
        keys = [(r[2], r[1], r[0]) for r in idx]
        assert keys == sorted(keys)
        assert c["w"].sum() == pytest.approx(1.0, abs=1e-15)
        assert np.all(c["w"] > 0)


def _fd_weight_moment(d, beta0, m):
    """<p^m> under (exp(beta0 |p|^2/2) + 1)^-1 on R^d, by radial quadrature
    and the sphere-monomial formula of Folland (Amer. Math. Monthly 2001)."""
    if any(k % 2 for k in m):
        return 0.0
    bk = [(k + 1) / 2.0 for k in m]
    sphere = 2.0 * np.prod([gamma(v) for v in bk]) / gamma(sum(bk))
    sphere0 = 2.0 * gamma(0.5) ** d / gamma(d / 2.0)
    deg = sum(m)

    def radial(power):
        f = lambda r: r ** power * expit(-beta0 * r * r / 2.0)
        return integrate.quad(f, 0.0, 60.0 / math.sqrt(beta0), epsabs=0, epsrel=1e-13, limit=200)[0]

    return sphere * radial(deg + d - 1) / (sphere0 * radial(d - 1))


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("beta0", [0.8, 1.0, 1.7])
def test_quadrature_degree_five(oracle_mod, d, beta0):
    # Eqs. quadrature2D / quadrature3D: exact for every monomial of degree <= 5,
    # not exact for at least one monomial of degree 6.
    c = oracle_mod.constants(d, beta0)
    pts = c["xi"] * c["idx"][:, :d].astype(float)
    w = c["w"]
    for deg in range(0, 6):
        for m in itertools.product(range(deg + 1), repeat=d):
            if sum(m) != deg:
                continue
            q = np.sum(w * np.prod(pts ** np.array(m), axis=1))
            ref = _fd_weight_moment(d, beta0, m)
            assert q == pytest.approx(ref, rel=1e-11, abs=1e-13), (m, q, ref)
    worst = 0.0
    for m in itertools.product(range(7), repeat=d):
        if sum(m) != 6:
            continue
        q = np.sum(w * np.prod(pts ** np.array(m), axis=1))
        ref = _fd_weight_moment(d, beta0, m)
        worst = max(worst, abs(q - ref) / max(abs(ref), 1e-300))
    assert worst > 1e-3


@pytest.mark.parametrize("d", [2, 3])
def test_eps0_is_fd_mean_energy(oracle_mod, d):
    # Eq. energyFDstdOmega at mu = 0, by direct integration, and the
    # appendix coefficients reduce to alpha1 = 1, alpha2 = 0 there.
    for beta0 in (0.8, 1.0, 1.7):
        e0 = oracle_mod.eps0(d, beta0)
        ref = 0.5 * sum(_fd_weight_moment(d, beta0, tuple(2 if j == k else 0 for j in range(d)))
                        for k in range(d))
        assert e0 == pytest.approx(ref, rel=1e-12)
        c = oracle_mod.constants(d, beta0)
        assert c["A1_0"] + c["A1_1"] * beta0 * e0 == pytest.approx(1.0, rel=1e-14)
        assert abs(c["A2_0"] + c["A2_1"] * beta0 * e0) < 1e-14


def _moments_of(d, xi, idx, pops):
    """Eq. DiscrAvr for one site's populations [b][4] (numpy)."""
    e = xi * idx[:, :d].astype(float)
    f = pops[:, 0]
    n = f.sum()
    S = pops[:, 1:].sum(axis=0)
    u = (e * f[:, None]).sum(axis=0) / n
    eps = (0.5 * ((e - u) ** 2).sum(axis=1) * f).sum() / n
    return n, S, u, eps


@pytest.mark.parametrize("d", [2, 3])
def test_equilibrium_moment_identities(oracle_mod, d):
    # Sec. 3.2 / Eq. WeqAlgo: the discrete equilibrium has exactly the
    # density matrix, velocity and internal energy it is built from.
    rng = np.random.default_rng(7 + d)
    for beta0 in (0.7, 1.0, 1.6):
        c = oracle_mod.constants(d, beta0)
        for _ in range(25):
            n = rng.uniform(0.3, 2.0)
            S = rng.normal(size=3)
            S *= rng.uniform(0, 0.95) * n / np.linalg.norm(S)
            u = rng.uniform(-0.4, 0.4, size=d)
            eps = oracle_mod.eps0(d, beta0) * rng.uniform(0.6, 1.5)
            weq = oracle_mod.equilibrium_site(d, beta0, np.r_[n, S], u, eps)
            n2, S2, u2, e2 = _moments_of(d, c["xi"], c["idx"], weq)
            assert n2 == pytest.approx(n, rel=1e-13)
            assert np.allclose(S2, S, rtol=1e-12, atol=1e-13)
            assert np.allclose(u2, u, rtol=1e-11, atol=1e-13)
            assert e2 == pytest.approx(eps, rel=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_alpha_coefficients_unique(oracle_mod, d):
    # The five coefficients are fixed by the moment conditions: perturbing
    # any one of them breaks an identity (guards against a term that the
    # identities above could not see).
    beta0 = 1.0
    c = oracle_mod.constants(d, beta0)
    xi, idx, w = c["xi"], c["idx"], c["w"]
    e = xi * idx[:, :d].astype(float)
    u = np.array([0.21, -0.13, 0.17][:d])
    eps = 1.3 * oracle_mod.eps0(d, beta0)

    def moments_with(delta):
        k = dict(c)
        for key, v in delta.items():
            k[key] = k[key] + v
        a1 = k["A1_0"] + k["A1_1"] * beta0 * eps
        a2 = k["A2_0"] + k["A2_1"] * beta0 * eps
        eu = e @ u
        P = (a1 + a2 * beta0 * 0.5 * (e ** 2).sum(1) + k["alpha3"] * beta0 * eu
             + k["alpha4"] * (beta0 * eu) ** 2 + k["alpha5"] * beta0 * 0.5 * (u @ u))
        f = w * P
        return np.r_[f.sum() - 1.0, (e * f[:, None]).sum(0) - u,
                     (0.5 * (e ** 2).sum(1) * f).sum() - (eps + 0.5 * u @ u)]

    assert np.max(np.abs(moments_with({}))) < 1e-13
    for key in ("A1_0", "A1_1", "A2_0", "A2_1", "alpha3", "alpha4", "alpha5"):
        assert np.max(np.abs(moments_with({key: 1e-3}))) > 1e-6, key
