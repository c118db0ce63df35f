"""The paper's Riemann problem (Sec. 4) as a physical pin of the oracle:
2048 x 2 D2Q9 periodic, tau = 10, 385 steps, beta = 1, u = 0, left
(mu_up, mu_dn) = (-3/2, -5/2), right (-2, -3); beta0 = 1 (not stated in the
paper).  The lattice Boltzmann moments are compared with the exact solution
of the Euler equations (Eq. Euler, gamma = 1 + 2/d = 2, P = (gamma - 1)
tr[rho] eps) around the central membrane, away from the waves of the second
(periodic) interface.  The paper reports qualitative agreement "albeit with
a small jump in velocity close to x = 0"; the bounds below encode that:
a few per cent in density and pressure, the shock front within 1 % of the
distance it travelled, and the velocity jump at the membrane."""
import numpy as np
import pytest

from euler_riemann import sample, star_state

NX, NY, TAU, T = 2048, 2, 10.0, 385
LEFT, RIGHT = (-1.5, -2.5), (-2.0, -3.0)


def riemann_initial(oracle_mod, beta=1.0):
    N = NX * NY
    rho4 = np.zeros((4, N))
    eps = np.zeros(N)
    sides = {}
    for name, mu in (("L", LEFT), ("R", RIGHT)):
        nu, nd, e = oracle_mod.fd_moments(2, beta, mu[0], mu[1])
        sides[name] = (nu + nd, nu - nd, e)
    x = np.arange(N) % NX
    for s in range(N):
        n, sz, e = sides["L" if x[s] < NX // 2 else "R"]
        rho4[0, s], rho4[3, s], eps[s] = n, sz, e
    return rho4, np.zeros((2, N)), eps, sides


@pytest.fixture(scope="module")
def run(oracle_mod):
    rho4, u, eps, sides = riemann_initial(oracle_mod)
    st = oracle_mod.init_equilibrium(2, (NX, NY, 1), 1.0, rho4, u, eps)
    st = oracle_mod.run(2, (NX, NY, 1), TAU, 1.0, T, st)
    r, uu, e = oracle_mod.moments(2, (NX, NY, 1), 1.0, st)
    xi = oracle_mod.constants(2, 1.0)["xi"]
    return r[0, :NX], uu[0, :NX], r[0, :NX] * e[:NX], sides, xi


def test_riemann_against_exact_euler(run):
    n, ux, P, sides, xi = run
    (nL, _, eL), (nR, _, eR) = sides["L"], sides["R"]
    L, R = (nL, 0.0, nL * eL), (nR, 0.0, nR * eR)
    i0 = NX // 2
    win = np.arange(i0 - 400, i0 + 400)
    ex = sample(L, R, 2.0, (win - i0 + 0.5) * xi / T)
    l1 = lambda a, b: np.sum(np.abs(a - b)) / np.sum(np.abs(b))
    assert l1(n[win], ex[0]) < 0.04
    assert l1(P[win], ex[2]) < 0.04
    # star pressure (plateau between the rarefaction and the shock)
    ps, us = star_state(L, R, 2.0)
    plateau = P[i0 + 100:i0 + 250]
    assert np.median(plateau) == pytest.approx(ps, rel=0.03)
    # shock front: where the pressure crosses (P* + P_R)/2
    mid = 0.5 * (ps + R[2])
    lbm = win[np.where(np.diff(np.sign(P[win] - mid)) != 0)[0][-1]]
    exa = win[np.where(np.diff(np.sign(ex[2] - mid)) != 0)[0][-1]]
    assert abs(lbm - exa) <= 0.01 * (exa - i0) + 2
    # the paper's "small jump in velocity close to x = 0"
    assert ux[i0 + 40] - ux[i0 - 40] > 0.02
