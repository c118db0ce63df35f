"""GPU parity of FP64 storage stepped in double-float arithmetic
(QLBM_FP64_DF) against the FP64 oracle.

The state is stored as IEEE doubles, exactly as in QLBM_FP64; the step
splits each double into a float pair (hi rounded to 24 bits, |lo| <=
ulp(hi)/2, together within 2^-48 of the double), runs the double-float
collision and rounds the result to double.  The per-step error bound is
therefore that of the double-float storage precision, 1e-12 relative
(normwise), and k steps give k * 1e-12.  Everything but the step is the
FP64 code, so state set-up and read-out are exact."""
import numpy as np
import pytest

from paper_1309_1656_gb300 import fields

pytestmark = pytest.mark.gpu

SHAPES = [(2, (37, 29, 1)), (2, (130, 7, 1)), (3, (9, 7, 5)), (3, (33, 6, 4))]


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1309_1656_gb300 import qlbm
    return qlbm


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_set_get_round_trip_is_exact(q):
    st = fields.random_populations(3, (9, 7, 5), seed=3)
    with q.Lattice(3, (9, 7, 5), 0.7, 1.0, precision="fp64df") as lat:
        lat.set_state(st)
        assert np.array_equal(lat.get_state(), st)


@pytest.mark.parametrize("d,dims", SHAPES)
@pytest.mark.parametrize("nsteps", [1, 2, 7, 100])
def test_fp64df_state_parity(q, oracle_mod, d, dims, nsteps):
    tau, beta0 = 0.7, 1.1
    st = fields.random_populations(d, dims, seed=100 + d)
    with q.Lattice(d, dims, tau, beta0, precision="fp64df") as lat:
        lat.set_state(st)
        lat.step(nsteps)
        got = lat.get_state()
        assert lat.time() == nsteps
    exp = oracle_mod.run(d, dims, tau, beta0, nsteps, st)
    assert rel(got, exp) < 1e-12 * nsteps


@pytest.mark.parametrize("d,dims", SHAPES)
def test_fp64df_init_moments_conserved_parity(q, oracle_mod, d, dims):
    beta0 = 0.9
    fl = fields.random_fields(d, dims, seed=7)
    with q.Lattice(d, dims, 0.8, beta0, precision="fp64df") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        ref = oracle_mod.init_equilibrium(d, dims, beta0, fl["rho4"], fl["u"], fl["eps"])
        assert rel(lat.get_state(), ref) < 1e-13
        lat.step(3)
        st3 = oracle_mod.run(d, dims, 0.8, beta0, 3, ref)
        r2, u2, e2 = lat.moments()
        r3, u3, e3 = oracle_mod.moments(d, dims, beta0, st3)
        assert rel(r2, r3) < 3e-12 and rel(u2, u3) < 3e-12 and rel(e2, e3) < 3e-12
        c = lat.conserved()
        c_ref = oracle_mod.conserved(d, dims, beta0, st3)
        assert np.allclose(c, c_ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(c_ref)))


def test_fp64df_agrees_with_fp64_over_1000_steps(q):
    # the D3Q19 workload recipe at 32^3: k * 1e-12 over k = 1000 steps
    d, dims = 3, (32, 32, 32)
    fl = fields.modes(d, dims, seed=2)
    out = {}
    for prec in ("fp64", "fp64df"):
        with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            lat.step(1000)
            out[prec] = lat.moments()
    for a, b in zip(out["fp64df"], out["fp64"]):
        assert rel(a, b) < 1000 * 1e-12


@pytest.mark.parametrize("d,dims", [(2, (128, 96, 1)), (3, (32, 24, 20))])
def test_fp64df_conservation_drift(q, d, dims):
    # Eqs. GlobalDensity/GlobalVelocity/GlobalTotalEnergy over 100 steps of
    # random populations far from equilibrium
    st = fields.random_populations(d, dims, seed=5)
    with q.Lattice(d, dims, 0.6, 1.0, precision="fp64df") as lat:
        lat.set_state(st)
        c0 = lat.conserved()
        lat.step(100)
        c1 = lat.conserved()
    assert float(np.max(np.abs(c1 - c0)) / np.max(np.abs(c0))) <= 1e-12


def test_fp64df_graph_replay_equals_single_launches(q):
    d, dims = 3, (17, 6, 5)
    st = fields.random_populations(d, dims, seed=11)
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp64df") as a, \
            q.Lattice(d, dims, 0.7, 1.0, precision="fp64df") as b:
        a.set_state(st)
        b.set_state(st)
        a.step(70)
        for _ in range(70):
            b.step(1)
        assert np.array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("d,dims", [(2, (37, 5, 1)), (3, (9, 7, 5))])
def test_fp64df_magnetic_field_vs_oracle(q, oracle_mod, d, dims):
    mu, B = 0.3, (0.4, -0.25, 0.9)
    st = fields.random_populations(d, dims, seed=120 + d)
    with q.Lattice(d, dims, 0.75, 1.0, precision="fp64df") as lat:
        lat.set_magnetic_field(mu, B)
        lat.set_state(st)
        lat.step(7)
        got = lat.get_state()
    oracle_mod.set_field(mu, B)
    try:
        exp = oracle_mod.run(d, dims, 0.75, 1.0, 7, st)
    finally:
        oracle_mod.set_field(0.0, (0, 0, 0))
    assert rel(got, exp) < 7e-12


def test_fp64df_values_outside_the_split_range(q, oracle_mod):
    # zero spin components take the short split; values below 2^-74 (and
    # the whole warp that holds one) take the general split; the step must
    # still follow the oracle
    d, dims = 2, (40, 9, 1)
    st = fields.random_populations(d, dims, seed=13)
    st[:, 3, ::3] = 0.0           # s_z exactly zero at every third site
    st[5, 1, ::7] = 1e-30         # tiny spin components
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp64df") as lat:
        lat.set_state(st)
        lat.step(4)
        got = lat.get_state()
    exp = oracle_mod.run(d, dims, 0.7, 1.0, 4, st)
    assert rel(got, exp) < 4e-12


def test_fp64df_small_spin_field_keeps_its_own_precision(q, oracle_mod):
    # a spin field ~2^-75 below the densities (the general split, whose
    # pairs are exact to 2^-47 down to 2^-102) must still be followed to
    # double-float precision relative to its own size, up to the absolute
    # floor of single precision's range (a lo part below 2^-126 is dropped
    # when rounding back: ~1e-38, here ~1e-14 of the spins).  The oracle's
    # complex-matrix storage resolves s_z only to ~ulp(f) (it sits in
    # rho_11 - rho_22), so the expectation uses the step's exact linearity in
    # the spins (u and eps depend on the traces alone, Eq. DiscrAvr):
    # s(T) for lam * s(0) is lam * s(T) for s(0), with f(T) unchanged
    d, dims = 3, (9, 7, 5)
    st = fields.random_populations(d, dims, seed=21)
    lam = 1e-22
    small = st.copy()
    small[:, 1:] *= lam
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp64df") as lat:
        lat.set_state(small)
        lat.step(3)
        got = lat.get_state()
    exp = oracle_mod.run(d, dims, 0.7, 1.0, 3, st)
    assert rel(got[:, 0], exp[:, 0]) < 3e-12
    assert rel(got[:, 1:], lam * exp[:, 1:]) < 3e-12


def test_fp64df_values_below_the_float_range_become_zero(q, oracle_mod):
    # double-float has single precision's exponent range: magnitudes below
    # 2^-126 are read as signed zeros (the densities are unaffected)
    d, dims = 2, (33, 5, 1)
    st = fields.random_populations(d, dims, seed=22)
    st[:, 1:] *= 1e-40
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp64df") as lat:
        lat.set_state(st)
        lat.step(2)
        got = lat.get_state()
    exp = oracle_mod.run(d, dims, 0.7, 1.0, 2, st)
    assert rel(got[:, 0], exp[:, 0]) < 3e-12
    assert np.all(np.abs(got[:, 1:]) < 2.0 ** -126)


def test_fp64df_fd_path_is_the_fp64_one(q):
    # the Fermi-Dirac equilibrium path is stepped by the FP64 kernel on the
    # same storage: bit-identical states
    d, dims = 3, (10, 8, 6)
    fl = fields.modes(d, dims, seed=4)
    out = {}
    for prec in ("fp64", "fp64df"):
        with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            lat.set_equilibrium_path(1)
            lat.step(3)
            out[prec] = lat.get_state()
    assert np.array_equal(out["fp64"], out["fp64df"])


def test_fp64df_has_no_reverse_mode(q):
    d, dims = 2, (8, 6, 1)
    st = fields.random_populations(d, dims, seed=1)
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp64df") as lat:
        lat.set_state(st)
        with pytest.raises(q.QLBMError):
            lat.step_adjoint(np.zeros_like(st))
        with pytest.raises(q.QLBMError):
            lat.rollout(4)
