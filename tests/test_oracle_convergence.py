"""The paper's 3D convergence-to-equilibrium example (Sec. 4, Fig. 6) as a
pin of the oracle: 32^3 D3Q19, tau = 10, beta0 = 1, uniform tr[rho],
Bloch vectors along z with a dichotomic outline and u_x proportional to
r_z.  The paper reports exponential convergence of rho, u and the total
energy to their (conserved) global averages, with an oscillatory pattern
from waves crossing the periodic box; the spin fluctuations, which carry no
waves, decay on a clean exponential."""
import numpy as np
import pytest

from paper_1309_1656_gb300 import fields

L, TAU, STEP, T = 32, 10.0, 25, 300


def deviations(oracle_mod, st):
    r, u, e = oracle_mod.moments(3, (L, L, L), 1.0, st)
    et = r[0] * (e + 0.5 * (u ** 2).sum(0))
    return np.array([np.abs(r[0] - r[0].mean()).max(),
                     np.abs(r[1:] - r[1:].mean(1, keepdims=True)).max(),
                     np.abs(u - u.mean(1, keepdims=True)).max(),
                     np.abs(et - et.mean()).max()])


@pytest.fixture(scope="module")
def history(oracle_mod):
    fl = fields.dichotomic3d(L)
    st = oracle_mod.init_equilibrium(3, (L, L, L), 1.0, fl["rho4"], fl["u"], fl["eps"])
    c0 = oracle_mod.conserved(3, (L, L, L), 1.0, st)
    rows = []
    for t in range(0, T + 1, STEP):
        rows.append(deviations(oracle_mod, st))
        if t < T:
            st = oracle_mod.run(3, (L, L, L), TAU, 1.0, STEP, st)
    return np.array(rows), c0, oracle_mod.conserved(3, (L, L, L), 1.0, st)


def test_spin_fluctuations_decay_exponentially(history):
    rows, _, _ = history
    t = np.arange(len(rows)) * STEP
    ls = np.log(rows[1:, 1])
    slope, icpt = np.polyfit(t[1:], ls, 1)
    resid = ls - (slope * t[1:] + icpt)
    assert slope < -0.03                      # > 1e3 per 230 steps
    assert np.max(np.abs(resid)) < 0.5        # a straight line in log scale
    assert rows[-1, 1] < 1e-6 * rows[0, 1]


def test_density_velocity_energy_converge(history):
    rows, c0, c1 = history
    for k in (0, 2, 3):                       # tr rho, u, total energy
        assert rows[-1, k] < 2e-2 * rows[1:4, k].max()
    assert np.max(np.abs(c1 - c0)) < 1e-12 * np.max(np.abs(c0))
