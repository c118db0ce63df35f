"""GPU parity of the double-float storage precision (QLBM_DF64) against the
FP64 oracle.

A double-float value carries a 48-bit significand, so one stored value is
within 2^-48 ~ 3.6e-15 of the double it represents and every double-float
operation rounds at ~2^-47 of its operands' size.  A step forms each output
population from O(b) such operations on values no larger than max |W|, so
the per-step error bound is the FP64 path's target, 1e-12 relative
(normwise), with a margin of ~10x over the operation count; k steps give
k * 1e-12.  Sizes and shapes are those of the FP64 parity tests (ragged row
tails, both AA parities)."""
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


def test_set_get_round_trip_is_a_double_float_rounding(q):
    st = fields.random_populations(3, (9, 7, 5), seed=3)
    with q.Lattice(3, (9, 7, 5), 0.7, 1.0, precision="df64") as lat:
        lat.set_state(st)
        back = lat.get_state()
    err = np.abs(back - st)
    assert np.all(err <= 2.0 ** -48 * np.abs(st))
    assert not np.array_equal(back, st)    # really stored as two floats


@pytest.mark.parametrize("d,dims", SHAPES)
@pytest.mark.parametrize("nsteps", [1, 2, 7, 100])
def test_df64_state_parity(q, oracle_mod, d, dims, nsteps):
    tau, beta0 = 0.7, 1.1
    st = fields.random_populations(d, dims, seed=100 + d)
    with q.Lattice(d, dims, tau, beta0, precision="df64") as lat:
        lat.set_state(st)
        lat.step(nsteps)
        got = lat.get_state()
        assert lat.time() == nsteps
    exp = oracle_mod.run(d, dims, tau, beta0, nsteps, st)
    assert rel(got, exp) < 1e-12 * nsteps


@pytest.mark.parametrize("d,dims", SHAPES)
def test_df64_init_moments_conserved_parity(q, oracle_mod, d, dims):
    beta0 = 0.9
    fl = fields.random_fields(d, dims, seed=7)
    with q.Lattice(d, dims, 0.8, beta0, precision="df64") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        st = lat.get_state()
        ref = oracle_mod.init_equilibrium(d, dims, beta0, fl["rho4"], fl["u"], fl["eps"])
        assert rel(st, ref) < 1e-13
        lat.step(3)
        st3 = oracle_mod.run(d, dims, 0.8, beta0, 3, ref)
        r2, u2, e2 = lat.moments()
        r3, u3, e3 = oracle_mod.moments(d, dims, beta0, st3)
        assert rel(r2, r3) < 3e-12 and rel(u2, u3) < 3e-12 and rel(e2, e3) < 3e-12
        c = lat.conserved()
        c_ref = oracle_mod.conserved(d, dims, beta0, st3)
        assert np.allclose(c, c_ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(c_ref)))


def test_df64_agrees_with_fp64_over_1000_steps(q):
    # the D3Q19 workload recipe at 32^3: moment fields of the two GPU paths,
    # within the per-step target accumulated over k = 1000 steps (k * 1e-12;
    # measured 2.6e-11 on u, the smallest field)
    d, dims = 3, (32, 32, 32)
    fl = fields.modes(d, dims, seed=2)
    out = {}
    for prec in ("fp64", "df64"):
        with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            lat.step(1000)
            out[prec] = lat.moments()
    for a, b in zip(out["df64"], out["fp64"]):
        assert rel(a, b) < 1000 * 1e-12


@pytest.mark.parametrize("d,dims", [(2, (128, 96, 1)), (3, (32, 24, 20))])
def test_df64_conservation_drift(q, d, dims):
    # Eqs. GlobalDensity/GlobalVelocity/GlobalTotalEnergy over 100 steps of
    # random populations far from equilibrium: double-float rounding is
    # unbiased at ~2^-47 per operation.
    st = fields.random_populations(d, dims, seed=5)
    with q.Lattice(d, dims, 0.6, 1.0, precision="df64") as lat:
        lat.set_state(st)
        c0 = lat.conserved()
        lat.step(100)
        c1 = lat.conserved()
    assert float(np.max(np.abs(c1 - c0)) / np.max(np.abs(c0))) <= 1e-12


def test_df64_graph_replay_equals_single_launches(q):
    d, dims = 3, (17, 6, 5)
    st = fields.random_populations(d, dims, seed=11)
    with q.Lattice(d, dims, 0.7, 1.0, precision="df64") as a, \
            q.Lattice(d, dims, 0.7, 1.0, precision="df64") as b:
        a.set_state(st)
        b.set_state(st)
        a.step(70)
        for _ in range(70):
            b.step(1)
        assert np.array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("d,dims", [(2, (37, 5, 1)), (3, (9, 7, 5))])
def test_df64_magnetic_field_vs_oracle(q, oracle_mod, d, dims):
    mu, B = 0.3, (0.4, -0.25, 0.9)
    st = fields.random_populations(d, dims, seed=120 + d)
    with q.Lattice(d, dims, 0.75, 1.0, precision="df64") as lat:
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


def test_df64_fd_params_match_fp64(q):
    d, dims = 3, (12, 10, 8)
    fl = fields.modes(d, dims, seed=4)
    res = {}
    for prec in ("fp64", "df64"):
        with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            lat.step(5)
            res[prec] = lat.fd_params()
    for a, b in zip(res["df64"][:3], res["fp64"][:3]):
        assert rel(a, b) < 1e-10
    assert res["df64"][4] == 0


def test_df64_has_no_reverse_mode(q):
    d, dims = 2, (8, 6, 1)
    st = fields.random_populations(d, dims, seed=1)
    with q.Lattice(d, dims, 0.7, 1.0, precision="df64") as lat:
        lat.set_state(st)
        with pytest.raises(q.QLBMError):
            lat.step_adjoint(np.zeros_like(st))
        with pytest.raises(q.QLBMError):
            lat.rollout(4)
