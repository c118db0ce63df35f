"""GPU parity of the magnetic-field term (Sec. 5, Eq. sigmaB_comm) against
the oracle: forward steps (FP64 per step, including the graph-replay path;
FP32 moment fields) and the checkpointed reverse mode, for one field over
the whole lattice and for a field B(x) per site (also changing between
steps, on the Fermi-Dirac equilibrium path and in the fused FD-output
step)."""
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


# ---------------------------------------------------------------------------
# A field that varies over the lattice, B(x) (qlbm_set_magnetic_field_array)
# ---------------------------------------------------------------------------

def site_field(dims, seed):
    N = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    Bs = rng.normal(size=(3, N)) * rng.uniform(0.2, 1.5, N)
    Bs[:, ::7] = 0.0
    return Bs


@pytest.fixture
def osite(oracle_mod):
    yield oracle_mod
    oracle_mod.set_field_array(0.0, None)
    oracle_mod.set_field(0.0, (0, 0, 0))


@pytest.mark.parametrize("prec", ["fp64", "fp64df", "df64"])
@pytest.mark.parametrize("d,dims", [(2, (37, 5, 1)), (3, (9, 7, 5)), (3, (33, 6, 4))])
@pytest.mark.parametrize("nsteps", [1, 2, 7, 70])
def test_site_field_fp64_vs_oracle(q, osite, prec, d, dims, nsteps):
    # the 64-bit precisions: FP64 storage stepped in double or in
    # double-float arithmetic, and double-float storage (within 1e-12 per
    # step of the oracle each)
    st = fields.random_populations(d, dims, seed=150 + d)
    Bs = site_field(dims, 3 + d)
    osite.set_field_array(MU, Bs)
    with q.Lattice(d, dims, 0.75, 1.0, precision=prec) as lat:
        lat.set_magnetic_field_array(MU, Bs)
        lat.set_state(st)
        lat.step(nsteps)
        got = lat.get_state()
    exp = osite.run(d, dims, 0.75, 1.0, nsteps, st)
    assert rel(got, exp) < 1e-12 * nsteps


def smooth_field(dims):
    """A weak field varying smoothly over the box (a rough random field
    dephases the spins to rounding level within 200 steps, leaving nothing
    to compare)."""
    nx, ny, nz = dims
    s = np.arange(nx * ny * nz)
    x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
    return np.array([0.05 + 0.04 * np.sin(2 * np.pi * x / nx), 0.03 * np.cos(2 * np.pi * y / ny),
                     0.08 + 0.05 * np.sin(2 * np.pi * z / nz + 1.0)])


@pytest.mark.parametrize("d,dims", [(2, (48, 40, 1)), (3, (16, 14, 12))])
def test_site_field_fp32_moments(q, osite, d, dims):
    import torch
    fl = fields.modes(d, dims, seed=14, amp=0.05, umax=0.1)
    Bs = smooth_field(dims)
    osite.set_field_array(MU, Bs)
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp32") as lat:
        # the field as a device tensor
        lat.set_magnetic_field_array(MU, torch.from_numpy(Bs).cuda())
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(200)
        r, u, e = lat.moments()
    st = osite.init_equilibrium(d, dims, 1.0, fl["rho4"], fl["u"], fl["eps"])
    st = osite.run(d, dims, 0.7, 1.0, 200, st)
    r0, u0, e0 = osite.moments(d, dims, 1.0, st)
    assert np.max(np.abs(r0[1:])) > 1e-3      # the spin field is still there
    assert rel(r[0], r0[0]) < 1e-5 and rel(r[1:], r0[1:]) < 1e-5
    assert rel(u, u0) < 1e-5 and rel(e, e0) < 1e-5


@pytest.mark.parametrize("d,dims", [(2, (150, 37, 1)), (3, (40, 23, 9))])
def test_site_field_fp16_vs_oracle(q, osite, d, dims):
    # the row-pipelined FP16 step with a per-site field, 5 steps: the FP16
    # bound of the storage arithmetic, 5 ((b + 2) 2^-24 + 2^-11) D / max|W|
    n = 5
    fl = fields.random_fields(d, dims, seed=15, umax=0.1)
    Bs = site_field(dims, 10)
    osite.set_field_array(MU, Bs)
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp16dev") as lat:
        lat.set_magnetic_field_array(MU, Bs)
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(n)
        got = lat.get_state()
    st = osite.init_equilibrium(d, dims, 1.0, fl["rho4"], fl["u"], fl["eps"])
    exp = osite.run(d, dims, 0.7, 1.0, n, st)
    c = osite.constants(d, 1.0)
    dev = exp.copy()
    dev[:, 0] -= c["w"][:, None]
    tol = n * ((c["b"] + 2) * 2.0 ** -24 + 2.0 ** -11) * np.max(np.abs(dev)) / np.max(np.abs(exp))
    assert rel(got, exp) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp64df", "df64"])
def test_site_field_changing_in_time(q, osite, prec):
    # B(x, t): a new field before every step, on the GPU and in the oracle
    d, dims, n = 3, (8, 7, 5), 6
    st = fields.random_populations(d, dims, seed=16)
    B0 = site_field(dims, 11)
    exp = st
    with q.Lattice(d, dims, 0.8, 1.0, precision=prec) as lat:
        lat.set_state(st)
        for t in range(n):
            Bt = B0 * np.cos(0.7 * t) + 0.3 * np.sin(0.4 * t)
            lat.set_magnetic_field_array(MU, Bt)
            lat.step(1)
            osite.set_field_array(MU, Bt)
            exp = osite.run(d, dims, 0.8, 1.0, 1, exp)
        got = lat.get_state()
    assert rel(got, exp) < 1e-12 * n


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
@pytest.mark.parametrize("d,dims", [(2, (13, 6, 1)), (3, (6, 5, 4))])
def test_site_field_rollout_adjoint_vs_oracle(q, osite, d, dims, prec, tol):
    tau, nsteps = 0.8, 6
    st = fields.random_populations(d, dims, seed=160 + d)
    Bs = site_field(dims, 12)
    osite.set_field_array(MU, Bs)
    lam_T = np.random.default_rng(8).normal(size=st.shape)
    with q.Lattice(d, dims, tau, 1.0, precision=prec) as lat:
        lat.set_magnetic_field_array(MU, Bs)
        lat.set_state(st)
        lat.rollout(nsteps, 2)
        lam0, g = lat.rollout_adjoint(lam_T)
    traj = [st]
    for _ in range(nsteps):
        traj.append(osite.run(d, dims, tau, 1.0, 1, traj[-1]))
    lam, g_o = lam_T, 0.0
    for k in reversed(range(nsteps)):
        lam, gk = osite.adjoint_step(d, dims, tau, 1.0, traj[k], lam)
        g_o += gk
    assert rel(lam0, lam) < tol * nsteps
    assert g == pytest.approx(g_o, rel=10 * tol)


@pytest.mark.parametrize("kind", ["uniform", "site"])
def test_field_on_the_fermi_dirac_equilibrium_path(q, kind):
    # the FP64 step through the recovered Fermi-Dirac parameters (Eq.
    # WeqDiscr) applies the field exactly as the direct path does
    d, dims = 3, (12, 10, 8)
    fl = fields.modes(d, dims, seed=21)
    Bs = site_field(dims, 13)
    res = []
    for path in (q.QLBM_EQ_DIRECT, q.QLBM_EQ_FD_PARAMS):
        with q.Lattice(d, dims, 0.7, 1.0, precision="fp64") as lat:
            if kind == "uniform":
                lat.set_magnetic_field(MU, B)
            else:
                lat.set_magnetic_field_array(MU, Bs)
            lat.set_equilibrium_path(path)
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            lat.step(7)
            res.append(lat.get_state())
    assert rel(res[1], res[0]) < 7e-12
    # and the field did act
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp64") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(7)
        assert rel(lat.get_state(), res[0]) > 1e-4


@pytest.mark.parametrize("prec", ["fp32", "fp16dev"])
def test_site_field_fused_fd_output_state_equals_plain_step(q, prec):
    d, dims = 3, (16, 14, 12)
    fl = fields.modes(d, dims, seed=22)
    Bs = site_field(dims, 14)
    out = []
    for fused in (False, True):
        with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
            lat.set_magnetic_field_array(MU, Bs)
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            for _ in range(3):
                if fused:
                    lat.step_fd_output()
                else:
                    lat.step(1)
            out.append(lat.get_state())
    assert np.array_equal(out[0], out[1])


def test_site_field_arguments(q):
    d, dims = 2, (8, 6, 1)
    N = int(np.prod(dims))
    st = fields.random_populations(d, dims, seed=17)
    with q.Lattice(d, dims, 0.8, 1.0, precision="fp64") as lat:
        bad = np.ones((3, N))
        bad[1, 5] = np.nan
        with pytest.raises(q.QLBMError) as e:
            lat.set_magnetic_field_array(MU, bad)
        assert e.value.code == q.QLBM_ERR_INVALID_ARG
        with pytest.raises(ValueError):
            lat.set_magnetic_field_array(MU, np.ones((3, N - 1)))
        # the field was left off: the step equals the field-free step
        lat.set_state(st)
        lat.step(3)
        a = lat.get_state()
        # a uniform field with mu = 0 switches a per-site field off
        lat.set_magnetic_field_array(MU, np.ones((3, N)))
        lat.set_magnetic_field(0.0, (0.0, 0.0, 0.0))
        lat.set_state(st)
        lat.step(3)
        assert np.array_equal(lat.get_state(), a)
