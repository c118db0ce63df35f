"""Degenerate inputs on the GPU: zero steps, lattices one site wide (every
neighbour is the site itself), pure density (W proportional to the identity,
Sec. 3.3: the scheme then stays spinless), the uniform equilibrium as a fixed
point, and covariance under a global SU(2) spin rotation (Sec. 2)."""
import numpy as np
import pytest

from paper_1309_1656_gb300 import fields

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "df64", "fp64df", "fp32", "fp16dev"]


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1309_1656_gb300 import qlbm
    return qlbm


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("prec", PRECS)
def test_zero_steps_leave_the_state(q, prec):
    d, dims = 3, (9, 7, 5)
    fl = fields.random_fields(d, dims, seed=2)
    with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        before = lat.get_state()
        lat.step(0)
        assert lat.time() == 0
        assert np.array_equal(lat.get_state(), before)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("df64", 1e-12), ("fp64df", 1e-12)])
@pytest.mark.parametrize("d,dims", [(2, (1, 1, 1)), (2, (1, 7, 1)), (2, (5, 1, 1)),
                                    (3, (1, 1, 1)), (3, (3, 1, 2)), (3, (1, 4, 1))])
def test_lattices_one_site_wide_vs_oracle(q, oracle_mod, prec, tol, d, dims):
    st = fields.random_populations(d, dims, seed=60 + d)
    with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
        lat.set_state(st)
        lat.step(5)
        got = lat.get_state()
    exp = oracle_mod.run(d, dims, 0.7, 1.0, 5, st)
    assert rel(got, exp) < 5 * tol


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d,dims", [(2, (37, 29, 1)), (3, (12, 9, 7))])
def test_pure_density_stays_spinless(q, oracle_mod, prec, d, dims):
    # W_i ~ 1: every spin component is zero and stays exactly zero; the
    # densities follow the oracle (the 64-bit precisions)
    fl = fields.random_fields(d, dims, seed=8)
    fl["rho4"][1:] = 0.0
    with q.Lattice(d, dims, 0.8, 1.0, precision=prec) as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(50)
        st = lat.get_state()
    assert np.all(st[:, 1:, :] == 0.0)
    if prec in ("fp64", "df64", "fp64df"):
        ref = oracle_mod.init_equilibrium(d, dims, 1.0, fl["rho4"], fl["u"], fl["eps"])
        ref = oracle_mod.run(d, dims, 0.8, 1.0, 50, ref)
        assert rel(st, ref) < 50 * 1e-12


@pytest.mark.parametrize("prec", PRECS)
def test_uniform_equilibrium_is_a_fixed_point(q, oracle_mod, prec):
    # n = 1, S = 0, u = 0, eps = eps0: the deviation codecs hold exact zeros
    # and keep them; the 64-bit precisions keep w_i up to rounding
    d, dims = 3, (8, 6, 5)
    N = int(np.prod(dims))
    rho4 = np.zeros((4, N))
    rho4[0] = 1.0
    with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
        lat.init_equilibrium(rho4, np.zeros((d, N)))
        before = lat.get_state()
        lat.step(20)
        after = lat.get_state()
    if prec in ("fp32", "fp16dev"):
        assert np.array_equal(after, before)
    else:
        assert rel(after, before) < 1e-12


def rotation(axis, angle):
    a = np.asarray(axis, float)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("df64", 1e-12), ("fp64df", 1e-12), ("fp32", 1e-6)])
def test_step_commutes_with_a_global_spin_rotation(q, prec, tol):
    # W -> V W V* for a fixed V in SU(2) rotates every Bloch vector by the
    # same R in SO(3); the collision and streaming act on s linearly with
    # scalar coefficients, so rotating then stepping equals stepping then
    # rotating
    d, dims = 3, (11, 8, 6)
    st = fields.random_populations(d, dims, seed=70)
    R = rotation((0.3, -0.7, 0.5), 1.1)
    rot = st.copy()
    rot[:, 1:, :] = np.einsum("ij,qjn->qin", R, st[:, 1:, :])
    out = []
    for s0 in (st, rot):
        with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
            lat.set_state(s0)
            lat.step(6)
            out.append(lat.get_state())
    a = out[0].copy()
    a[:, 1:, :] = np.einsum("ij,qjn->qin", R, out[0][:, 1:, :])
    assert rel(out[1], a) < tol


def test_lattice_larger_than_the_device_is_an_error(q):
    # 6e8 D3Q19 sites in FP64 need ~365 GB: the allocation fails, the call
    # returns QLBM_ERR_OOM, and the device stays usable
    with pytest.raises(q.QLBMError) as e:
        q.qlbm_create(3, (1000, 1000, 600), 0.7, 1.0, 1.0, q.QLBM_FP64)
    assert e.value.code == q.QLBM_ERR_OOM
    d, dims = 2, (16, 8, 1)
    st = fields.random_populations(d, dims, seed=4)
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp64") as lat:
        lat.set_state(st)
        lat.step(3)
        assert np.isfinite(lat.get_state()).all()
