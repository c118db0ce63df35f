"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerances (normwise, max |gpu - oracle| / max |oracle| per compared array):
  * FP64 storage: 1e-12 relative per step (the target stated for the FP64
    path), i.e. k * 1e-12 after k steps;
  * FP32 storage: 1e-5 relative on each moment field after 1000 steps;
  * FP16 deviation storage: bound derived from half precision (see
    test_fp16dev_parity).
Sizes span several thread blocks with ragged row tails (nx not a multiple
of the block width) and both AA parities (odd and even step counts).
"""
import numpy as np
import pytest

from paper_1309_1656_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1309_1656_gb300 import qlbm
    return qlbm


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


SHAPES = [(2, (37, 29, 1)), (2, (130, 7, 1)), (3, (9, 7, 5)), (3, (33, 6, 4))]


@pytest.mark.parametrize("d,dims", SHAPES)
@pytest.mark.parametrize("nsteps", [1, 2, 7])
def test_fp64_state_parity(q, oracle_mod, d, dims, nsteps):
    tau, beta0 = 0.7, 1.1
    st = fields.random_populations(d, dims, seed=100 + d)
    with q.Lattice(d, dims, tau, beta0, precision="fp64") as lat:
        lat.set_state(st)
        lat.step(nsteps)
        got = lat.get_state()
        assert lat.time() == nsteps
    exp = oracle_mod.run(d, dims, tau, beta0, nsteps, st)
    assert rel(got, exp) < 1e-12 * nsteps


@pytest.mark.parametrize("d,dims", SHAPES)
def test_fp64_init_moments_conserved_parity(q, oracle_mod, d, dims):
    beta0 = 0.9
    fl = fields.random_fields(d, dims, seed=7)
    with q.Lattice(d, dims, 0.8, beta0, precision="fp64") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        st = lat.get_state()
        ref = oracle_mod.init_equilibrium(d, dims, beta0, fl["rho4"], fl["u"], fl["eps"])
        assert rel(st, ref) < 1e-13
        r, u, e = lat.moments()
        assert rel(r, fl["rho4"]) < 1e-13
        assert rel(u, fl["u"]) < 1e-12
        assert rel(e, fl["eps"]) < 1e-13
        lat.step(3)
        st3 = oracle_mod.run(d, dims, 0.8, beta0, 3, ref)
        r2, u2, e2 = lat.moments()
        r3, u3, e3 = oracle_mod.moments(d, dims, beta0, st3)
        assert rel(r2, r3) < 3e-12 and rel(u2, u3) < 3e-12 and rel(e2, e3) < 3e-12
        c = lat.conserved()
        c_ref = oracle_mod.conserved(d, dims, beta0, st3)
        assert np.allclose(c, c_ref, rtol=1e-13, atol=1e-13 * np.max(np.abs(c_ref)))


def test_default_eps_is_eps0(q, oracle_mod):
    for d, dims in ((2, (8, 6, 1)), (3, (5, 4, 3))):
        fl = fields.random_fields(d, dims, seed=3)
        with q.Lattice(d, dims, 0.8, 1.3) as lat:
            lat.init_equilibrium(fl["rho4"], fl["u"])
            _, _, e = lat.moments()
            assert np.allclose(e, oracle_mod.eps0(d, 1.3), rtol=1e-13)


DRIFT_CASES = [(2, (128, 96, 1), "fp64"), (3, (32, 24, 20), "fp64"),
               (2, (128, 96, 1), "fp32"), (3, (32, 24, 20), "fp32")]


def _drift(q, d, dims, prec, state=None, fl=None, nsteps=100):
    with q.Lattice(d, dims, 0.6, 1.0, precision=prec) as lat:
        if state is not None:
            lat.set_state(state)
        else:
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        c0 = lat.conserved()
        lat.step(nsteps)
        c1 = lat.conserved()
    return float(np.max(np.abs(c1 - c0)) / np.max(np.abs(c0)))


@pytest.mark.parametrize("d,dims,prec", DRIFT_CASES)
def test_conservation_drift_near_equilibrium(q, d, dims, prec):
    # Eqs. GlobalDensity/GlobalVelocity/GlobalTotalEnergy over 100 steps of
    # paper-shaped Fourier-mode fields (flow develops, collisions active).
    # Single precision leaves an unbiased random walk of roundings of
    # ~1e-9 here; a biased equilibrium moment (rounded constants) would
    # drift by ~1e-7 per step, i.e. >= 1e-5.
    fl = fields.modes(d, dims, seed=8, amp=0.05, umax=0.1)
    tol = 1e-13 if prec == "fp64" else 2e-8
    assert _drift(q, d, dims, prec, fl=fl) <= tol


@pytest.mark.parametrize("d,dims,prec", DRIFT_CASES)
def test_conservation_drift_far_from_equilibrium(q, d, dims, prec):
    # Random populations (n ~ 2, far from the n = 1 deviation reference,
    # strongly non-equilibrium): single-precision rounding is then of the
    # order of the values themselves; the bound allows a bias of at most
    # 0.1 ulp per site and step (1e-6 over 100 steps).
    st = fields.random_populations(d, dims, seed=5)
    tol = 1e-13 if prec == "fp64" else 1e-6
    assert _drift(q, d, dims, prec, state=st) <= tol


@pytest.mark.parametrize("d,dims,tau", [(2, (64, 64, 1), 0.8), (3, (24, 20, 16), 0.7)])
def test_fp32_moments_after_1000_steps(q, oracle_mod, d, dims, tau):
    # FP32 storage and arithmetic against the FP64 oracle on the paper-shaped
    # workloads (2D density wave + spin blob; 3D Fourier-mode fields).
    beta0 = 1.0
    fl = fields.blob2d(dims[0], dims[1]) if d == 2 else fields.modes(3, dims, seed=2)
    with q.Lattice(d, dims, tau, beta0, precision="fp32") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(1000)
        lat.sync()
        r, u, e = lat.moments()
    st = oracle_mod.init_equilibrium(d, dims, beta0, fl["rho4"], fl["u"], fl["eps"])
    st = oracle_mod.run(d, dims, tau, beta0, 1000, st)
    r0, u0, e0 = oracle_mod.moments(d, dims, beta0, st)
    assert rel(r[0], r0[0]) < 1e-5
    assert rel(r[1:], r0[1:]) < 1e-5
    assert rel(u, u0) < 1e-5
    assert rel(e, e0) < 1e-5


def test_error_flags(q):
    from paper_1309_1656_gb300.qlbm import QLBMError, QLBM_ERR_NONFINITE, QLBM_ERR_NONPOSITIVE_DENSITY
    d, dims = 2, (16, 8, 1)
    st = fields.random_populations(d, dims, seed=9)
    with q.Lattice(d, dims, 0.8, 1.0) as lat:
        bad = st.copy()
        bad[3, 2, 17] = np.nan
        lat.set_state(bad)
        lat.step(1)
        with pytest.raises(QLBMError) as e:
            lat.sync()
        assert e.value.code == QLBM_ERR_NONFINITE
        lat.sync()  # cleared
        neg = st.copy()
        neg[:, 0, 5] = -neg[:, 0, 5]
        lat.set_state(neg)
        lat.step(1)
        with pytest.raises(QLBMError) as e:
            lat.sync()
        assert e.value.code == QLBM_ERR_NONPOSITIVE_DENSITY
        lat.set_state(st)
        lat.step(2)
        lat.sync()


def test_device_pointer_paths(q, oracle_mod):
    import torch
    d, dims = 3, (10, 9, 8)
    N = 10 * 9 * 8
    fl = fields.random_fields(d, dims, seed=21)
    with q.Lattice(d, dims, 0.75, 1.0) as lat:
        rho4 = torch.from_numpy(fl["rho4"]).cuda()
        u = torch.from_numpy(fl["u"]).cuda()
        eps = torch.from_numpy(fl["eps"]).cuda()
        q.qlbm_init_equilibrium(lat.h, rho4, u, eps)
        lat.step(5)
        st = torch.zeros((19, 4, N), dtype=torch.float64, device="cuda")
        q.qlbm_get_state(lat.h, st)
        r = torch.zeros_like(rho4)
        uu = torch.zeros_like(u)
        e = torch.zeros_like(eps)
        q.qlbm_moments(lat.h, r, uu, e)
        host = lat.get_state()
        assert np.array_equal(st.cpu().numpy(), host)
        r2, u2, e2 = lat.moments()
        assert np.array_equal(r.cpu().numpy(), r2) and np.array_equal(e.cpu().numpy(), e2)
        q.qlbm_set_state(lat.h, st)
        assert lat.time() == 0
        assert np.array_equal(lat.get_state(), host)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replay_equals_single_launches(q, prec):
    # qlbm_step(n >= 64) replays a captured 32-step graph; the result must be
    # bit-identical to n single-step calls, from either AA parity.
    d, dims = 3, (20, 9, 7)
    st = fields.random_populations(d, dims, seed=61)
    for pre in (0, 1):
        with q.Lattice(d, dims, 0.8, 1.0, precision=prec) as a, \
                q.Lattice(d, dims, 0.8, 1.0, precision=prec) as b:
            a.set_state(st)
            b.set_state(st)
            a.step(pre)
            b.step(pre)
            a.step(101)
            for _ in range(101):
                b.step(1)
            assert a.time() == b.time() == 101 + pre
            assert np.array_equal(a.get_state(), b.get_state())
