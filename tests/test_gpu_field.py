"""GPU parity of the magnetic-field term (Sec. 5, Eq. sigmaB_comm) against
the oracle: forward steps (FP64 per step, including the graph-replay path;
FP32 moment fields) and the checkpointed reverse mode."""
import numpy as np
import pytest

from paper_1309_1656_gb300 import fields

pytestmark = pytest.mark.gpu

MU, B = 0.3, (0.4, -0.25, 0.9)


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1309_1656_gb300 import qlbm
    return qlbm


@pytest.fixture
def ofield(oracle_mod):
    oracle_mod.set_field(MU, B)
    yield oracle_mod
    oracle_mod.set_field(0.0, (0, 0, 0))


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("d,dims", [(2, (37, 5, 1)), (3, (9, 7, 5))])
@pytest.mark.parametrize("nsteps", [1, 2, 7, 70])
def test_field_fp64_vs_oracle(q, ofield, d, dims, nsteps):
    st = fields.random_populations(d, dims, seed=120 + d)
    with q.Lattice(d, dims, 0.75, 1.0, precision="fp64") as lat:
        lat.set_magnetic_field(MU, B)
        lat.set_state(st)
        lat.step(nsteps)
        got = lat.get_state()
    exp = ofield.run(d, dims, 0.75, 1.0, nsteps, st)
    assert rel(got, exp) < 1e-12 * nsteps


@pytest.mark.parametrize("d,dims", [(2, (48, 40, 1)), (3, (16, 14, 12))])
def test_field_fp32_moments(q, ofield, d, dims):
    fl = fields.modes(d, dims, seed=13, amp=0.05, umax=0.1)
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp32") as lat:
        lat.set_magnetic_field(MU, B)
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(200)
        r, u, e = lat.moments()
    st = ofield.init_equilibrium(d, dims, 1.0, fl["rho4"], fl["u"], fl["eps"])
    st = ofield.run(d, dims, 0.7, 1.0, 200, st)
    r0, u0, e0 = ofield.moments(d, dims, 1.0, st)
    assert rel(r[0], r0[0]) < 1e-5 and rel(r[1:], r0[1:]) < 1e-5
    assert rel(u, u0) < 1e-5 and rel(e, e0) < 1e-5


@pytest.mark.parametrize("d,dims", [(2, (13, 6, 1)), (3, (6, 5, 4))])
def test_field_rollout_adjoint_fp64(q, ofield, d, dims):
    tau, nsteps = 0.8, 6
    st = fields.random_populations(d, dims, seed=140 + d)
    lam_T = np.random.default_rng(7).normal(size=st.shape)
    with q.Lattice(d, dims, tau, 1.0, precision="fp64") as lat:
        lat.set_magnetic_field(MU, B)
        lat.set_state(st)
        lat.rollout(nsteps, 2)
        lam0, g = lat.rollout_adjoint(lam_T)
    traj = [st]
    for _ in range(nsteps):
        traj.append(ofield.run(d, dims, tau, 1.0, 1, traj[-1]))
    lam, g_o = lam_T, 0.0
    for k in reversed(range(nsteps)):
        lam, gk = ofield.adjoint_step(d, dims, tau, 1.0, traj[k], lam)
        g_o += gk
    assert rel(lam0, lam) < 1e-11 * nsteps
    assert g == pytest.approx(g_o, rel=1e-10)
