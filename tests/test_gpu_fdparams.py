"""GPU parity of the Fermi-Dirac parameter recovery (Prop. 1) against the
oracle's independent inversion (its own F_k quadrature and bisection), round
trips from known parameters, invalid sites, and the step variant that builds
W^eq through the recovered parameters (Eq. WeqDiscr) against the direct
equilibrium (Eq. WeqAlgo)."""
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


@pytest.mark.parametrize("d,dims", [(2, (9, 7, 1)), (3, (5, 4, 3))])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 2e-5)])
def test_fd_params_vs_oracle(q, oracle_mod, d, dims, prec, tol):
    beta0 = 1.0
    fl = fields.random_fields(d, dims, seed=70 + d, umax=0.3)
    with q.Lattice(d, dims, 0.8, beta0, precision=prec) as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(3)
        r4, u, eps = lat.moments()
        beta, mu_up, mu_dn, axis, nfail = lat.fd_params()
    assert nfail == 0
    for s in range(r4.shape[1]):
        rc, ref = oracle_mod.fd_params(d, r4[:, s], eps[s])
        assert rc == 0
        assert beta[s] == pytest.approx(ref[0], rel=tol)
        assert mu_up[s] == pytest.approx(ref[1], rel=tol, abs=tol)
        assert mu_dn[s] == pytest.approx(ref[2], rel=tol, abs=tol)
        assert np.allclose(axis[:, s], ref[3:], atol=tol)


@pytest.mark.parametrize("d", [2, 3])
def test_fd_params_round_trip(q, oracle_mod, d):
    # fields built from known parameters through the oracle's forward map
    dims = (6, 5, 1) if d == 2 else (4, 3, 3)
    N = int(np.prod(dims))
    rng = np.random.default_rng(d + 11)
    beta = rng.uniform(0.4, 2.5, N)
    mu_up = rng.uniform(-4.0, 1.5, N)
    mu_dn = mu_up - rng.uniform(0.0, 1.5, N)
    mu_dn[:2] = mu_up[:2]                    # degenerate occupations
    axis = rng.normal(size=(3, N))
    axis /= np.linalg.norm(axis, axis=0)
    rho4 = np.zeros((4, N))
    eps = np.zeros(N)
    for s in range(N):
        nu, nd, e = oracle_mod.fd_moments(d, beta[s], mu_up[s], mu_dn[s])
        rho4[0, s] = nu + nd
        rho4[1:, s] = (nu - nd) * axis[:, s]
        eps[s] = e
    with q.Lattice(d, dims, 0.8, 1.0) as lat:
        lat.init_equilibrium(rho4, np.zeros((d, N)), eps)
        b, mu, md, ax, nfail = lat.fd_params()
    assert nfail == 0
    assert np.allclose(b, beta, rtol=1e-10)
    assert np.allclose(mu, mu_up, rtol=1e-9, atol=1e-10)
    assert np.allclose(md, mu_dn, rtol=1e-9, atol=1e-10)
    assert np.allclose(ax[:, 2:], axis[:, 2:], atol=1e-9)
    assert np.all(ax[:, :2] == 0.0)


REGIMES = {   # nu_up = beta mu_up range, nu_up - nu_dn range
    "classical": ((-30.0, -8.0), (0.0, 5.0)),
    "intermediate": ((-8.0, 1.0), (0.0, 5.0)),
    "degenerate": ((1.0, 40.0), (0.0, 5.0)),
    # n_dn / n_up down to ~1e-4: n_dn = (n - |S|)/2 keeps ~12 digits
    "polarised": ((0.0, 10.0), (6.0, 9.0)),
}


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("regime", sorted(REGIMES))
def test_fd_params_round_trip_regimes(q, oracle_mod, d, regime):
    # every branch of the device F_k evaluation (series lengths, Taylor,
    # Chebyshev, Sommerfeld) and the Newton solve far from its classical
    # starting point
    dims = (5, 4, 1) if d == 2 else (3, 3, 2)
    N = int(np.prod(dims))
    rng = np.random.default_rng(d + 31 + len(regime))
    (a1, b1), (g1, g2) = REGIMES[regime]
    beta = rng.uniform(0.3, 3.0, N)
    nu_up = rng.uniform(a1, b1, N)
    nu_dn = nu_up - rng.uniform(g1, g2, N)
    axis = rng.normal(size=(3, N))
    axis /= np.linalg.norm(axis, axis=0)
    rho4 = np.zeros((4, N))
    eps = np.zeros(N)
    for s in range(N):
        nu, nd, e = oracle_mod.fd_moments(d, beta[s], nu_up[s] / beta[s], nu_dn[s] / beta[s])
        rho4[0, s] = nu + nd
        rho4[1:, s] = (nu - nd) * axis[:, s]
        eps[s] = e
    with q.Lattice(d, dims, 0.8, 1.0) as lat:
        lat.init_equilibrium(rho4, np.zeros((d, N)), eps)
        b, mu, md, ax, nfail = lat.fd_params()
    assert nfail == 0
    # beta is ill-conditioned in the degenerate limit (eps depends on it only
    # at order (pi/nu)^2): relative error ~ 1e-16 nu^2
    tol_b = 1e-10 if regime != "degenerate" else 1e-8
    assert np.allclose(b, beta, rtol=tol_b)
    assert np.allclose(mu * b, nu_up, rtol=1e-9, atol=1e-9)
    assert np.allclose(md * b, nu_dn, rtol=1e-9, atol=1e-9)
    moved = nu_up != nu_dn
    assert np.allclose(ax[:, moved], axis[:, moved], atol=1e-9)


def test_fd_params_invalid_sites(q):
    d, dims = 3, (4, 2, 2)
    N = 16
    fl = fields.random_fields(d, dims, seed=5)
    fl["rho4"][3, 0] = 1.5 * fl["rho4"][0, 0]     # |S| > n: not positive definite
    fl["eps"][1] = 1e-7                          # below the degenerate limit
    with q.Lattice(d, dims, 0.8, 1.0) as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        b, mu, md, ax, nfail = lat.fd_params()
    assert nfail == 2
    assert np.isnan(b[0]) and np.isnan(b[1]) and np.all(np.isfinite(b[2:]))


@pytest.mark.parametrize("d,dims", [(2, (33, 17, 1)), (3, (12, 9, 7))])
def test_fd_equilibrium_path_matches_direct(q, d, dims):
    fl = fields.random_fields(d, dims, seed=80 + d)
    out = {}
    for path in (q.QLBM_EQ_DIRECT, q.QLBM_EQ_FD_PARAMS):
        with q.Lattice(d, dims, 0.7, 1.0, precision="fp64") as lat:
            lat.set_equilibrium_path(path)
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            lat.step(7)
            lat.sync()
            out[path] = lat.get_state()
    a, b = out[q.QLBM_EQ_DIRECT], out[q.QLBM_EQ_FD_PARAMS]
    assert np.max(np.abs(a - b)) / np.max(np.abs(a)) < 7e-12


def test_fd_path_needs_fp64(q):
    with q.Lattice(2, (8, 8, 1), 0.8, 1.0, precision="fp32") as lat:
        with pytest.raises(q.QLBMError) as e:
            lat.set_equilibrium_path(q.QLBM_EQ_FD_PARAMS)
        assert e.value.code == q.QLBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("d,dims", [(2, (7, 5, 1)), (3, (4, 4, 3))])
def test_fd_params_adjoint_vs_finite_differences(q, d, dims):
    # J(W) = sum_x c_b beta + c_u mu_up + c_d mu_dn + c_a . axis, differentiated
    # through the per-site Newton solve by the implicit-function rule, checked
    # by central differences of the forward recovery in FP64.
    b = 9 if d == 2 else 19
    N = int(np.prod(dims))
    fl = fields.random_fields(d, dims, seed=90 + d, umax=0.25)
    rng = np.random.default_rng(d)
    cb, cu, cd = rng.normal(size=(3, N))
    ca = rng.normal(size=(3, N))
    with q.Lattice(d, dims, 0.8, 1.0, precision="fp64") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(2)
        W = lat.get_state()

        def J(state):
            lat.set_state(state)
            be, mu, md, ax, nf = lat.fd_params()
            assert nf == 0
            return float(np.sum(cb * be + cu * mu + cd * md) + np.sum(ca * ax))

        lat.set_state(W)
        lam = np.zeros((b, 4, N))
        q.qlbm_fd_params_adjoint(lat.h, lam, cb, cu, cd, ca)
        for _ in range(4):
            dv = rng.normal(size=W.shape) * np.abs(W)
            h = 1e-6
            fd = (J(W + h * dv) - J(W - h * dv)) / (2 * h)
            ad = float(np.sum(lam * dv))
            assert ad == pytest.approx(fd, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("d,dims", [(2, (11, 6, 1)), (3, (5, 4, 3))])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-7)])
def test_init_from_fd_parameters(q, oracle_mod, d, dims, prec, tol):
    N = int(np.prod(dims))
    rng = np.random.default_rng(d + 30)
    beta = rng.uniform(0.5, 2.0, N)
    mu_up = rng.uniform(-3.0, 1.0, N)
    mu_dn = mu_up - rng.uniform(0.0, 1.0, N)
    axis = rng.normal(size=(3, N))
    axis /= np.linalg.norm(axis, axis=0)
    u = rng.uniform(-0.1, 0.1, (d, N))
    rho4 = np.zeros((4, N))
    eps = np.zeros(N)
    for s in range(N):
        nu, nd, e = oracle_mod.fd_moments(d, beta[s], mu_up[s], mu_dn[s])
        rho4[:, s] = np.r_[nu + nd, (nu - nd) * axis[:, s]]
        eps[s] = e
    ref = oracle_mod.init_equilibrium(d, dims, 1.0, rho4, u, eps)
    with q.Lattice(d, dims, 0.8, 1.0, precision=prec) as lat:
        q.qlbm_init_fd_params(lat.h, beta, mu_up, mu_dn, axis, u)
        got = lat.get_state()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < tol


@pytest.mark.parametrize("prec", ["fp32", "fp16dev"])
@pytest.mark.parametrize("d,dims", [(2, (37, 29, 1)), (3, (33, 6, 4))])
@pytest.mark.parametrize("field", [False, True])
def test_step_fd_output_state_equals_plain_step(q, prec, d, dims, field):
    # the fused kernel runs the step kernel's collision and addressing (and
    # the field's spin rotation): the state after it is the state after a
    # plain step, in both AA parities
    fl = fields.random_fields(d, dims, seed=21)
    with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as a, q.Lattice(d, dims, 0.7, 1.0, precision=prec) as b:
        for lat in (a, b):
            if field:
                lat.set_magnetic_field(0.3, (0.4, -0.25, 0.9))
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            lat.step(3)
        for _ in range(2):
            a.step(1)
            out = b.step_fd_output()
            assert out[4] == 0
            assert np.array_equal(a.get_state(), b.get_state())
        assert a.time() == b.time() == 5


@pytest.mark.parametrize("prec", ["fp32", "fp16dev"])
@pytest.mark.parametrize("d,dims", [(2, (48, 40, 1)), (3, (16, 14, 12))])
def test_step_fd_output_params_vs_double_solve(q, prec, d, dims):
    # single-precision solve fused into the step against the double solve of
    # the same state (qlbm_fd_params); a quarter of the sites are near
    # degenerate (|S| < 0.005 n), where the float splitting keeps ~1e-6 |mu|
    fl = fields.modes(d, dims, seed=17, amp=0.05, umax=0.1)
    N = int(np.prod(dims))
    rng = np.random.default_rng(5)
    deg = rng.random(N) < 0.25
    fl["rho4"][1:, deg] *= rng.uniform(0.0, 0.005, deg.sum()) / np.maximum(
        np.linalg.norm(fl["rho4"][1:, deg], axis=0) / fl["rho4"][0, deg], 1e-300)
    with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(2)
        b64, mu64, md64, ax64, nf64 = lat.fd_params()
        b, mu, md, ax, nf = lat.step_fd_output()
    assert nf == 0 and nf64 == 0
    assert np.allclose(b, b64, rtol=2e-5, atol=0)
    scale = 1.0 / b64
    assert np.all(np.abs(mu - mu64) <= 2e-5 * (np.abs(mu64) + scale))
    assert np.all(np.abs(md - md64) <= 2e-5 * (np.abs(md64) + scale))
    # spin splitting, including the near-degenerate sites
    split64 = mu64 - md64
    assert np.all(np.abs((mu - md) - split64) <= 1e-4 * np.abs(split64) + 2e-6 * scale)
    S = np.linalg.norm(fl["rho4"][1:], axis=0)
    ok = S > 0
    assert np.allclose(ax[:, ok], ax64[:, ok], atol=2e-5)


def test_step_fd_output_needs_single_precision_storage(q):
    with q.Lattice(2, (8, 6, 1), 0.7, 1.0, precision="fp64") as lat:
        lat.init_equilibrium(np.r_[np.ones((1, 48)), np.zeros((3, 48))], np.zeros((2, 48)))
        with pytest.raises(q.QLBMError):
            lat.step_fd_output()


def test_step_fd_output_device_pointers_match_host(q):
    # device float32 tensors (asynchronous when not counting) and host arrays
    # give the same parameters and the same state
    import torch
    d, dims = 3, (20, 9, 7)
    N = int(np.prod(dims))
    fl = fields.modes(d, dims, seed=23)
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp32") as a, q.Lattice(d, dims, 0.7, 1.0, precision="fp32") as b:
        for lat in (a, b):
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        host = a.step_fd_output()
        dev = [torch.empty(N, dtype=torch.float32, device="cuda") for _ in range(3)]
        ax = torch.empty((3, N), dtype=torch.float32, device="cuda")
        assert q.qlbm_step_fd_output(b.h, *dev, ax, count=False) is None
        b.sync()
        for x, y in zip(host[:3], dev):
            assert np.array_equal(x, y.cpu().numpy())
        assert np.array_equal(host[3], ax.cpu().numpy())
        assert np.array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("prec,abs_tol,beta_tol", [("fp32", 2e-6, 2e-5), ("fp16dev", 2e-5, 3e-4)])
@pytest.mark.parametrize("d", [2, 3])
def test_step_fd_output_splitting_near_degeneracy_vs_oracle(q, oracle_mod, prec, abs_tol, beta_tol, d):
    # sites with |S|/n log-uniform in [1e-8, 1e-2]: the fused single-
    # precision output's spin splitting mu_up - mu_dn against the oracle's
    # double inversion of the same fields (its own init state and moments).
    # Bound (header of qlbm_step_fd_output): 1e-4 |mu_up - mu_dn| relative
    # plus abs_tol / beta absolute -- 2e-6 / beta for FP32 storage, 2e-5 /
    # beta for FP16, whose spin components are stored in half precision
    # (absolute storage error ~2^-25 per value)
    dims = (15, 11, 1) if d == 2 else (7, 6, 4)
    N = int(np.prod(dims))
    fl = fields.modes(d, dims, seed=19, amp=0.05, umax=0.1)
    rng = np.random.default_rng(29 + d)
    ratio = 10.0 ** rng.uniform(-8, -2, N)
    ax = rng.normal(size=(3, N))
    ax /= np.linalg.norm(ax, axis=0)
    fl["rho4"][1:] = ratio * fl["rho4"][0] * ax
    with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        b, mu, md, axg, nf = lat.step_fd_output()
    assert nf == 0
    st = oracle_mod.init_equilibrium(d, dims, 1.0, fl["rho4"], fl["u"], fl["eps"])
    r4, _, eps = oracle_mod.moments(d, dims, 1.0, st)
    worst = 0.0
    for s in range(N):
        rc, out = oracle_mod.fd_params(d, r4[:, s], eps[s])
        assert rc == 0
        split_o = out[1] - out[2]
        split_g = float(mu[s]) - float(md[s])
        bound = 1e-4 * abs(split_o) + abs_tol / out[0]
        worst = max(worst, abs(split_g - split_o) / bound)
        assert abs(split_g - split_o) <= bound, (s, ratio[s], split_g, split_o)
        # beta against the oracle's: FP16 storage rounds the energy moments
        assert float(b[s]) == pytest.approx(out[0], rel=beta_tol)
    assert worst <= 1.0
