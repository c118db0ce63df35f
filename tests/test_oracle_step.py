"""Pins of the oracle's time step (Sec. 3.3) against what the paper fixes.

* streaming alone (dt/tau = 0) is a periodic shift of every direction by its
  lattice vector, checked against numpy.roll (Eq. TransportStep);
* dt/tau = 1 replaces every population by the streamed local equilibrium;
* global density matrix, momentum and total energy are conserved
  (Eqs. GlobalDensity, GlobalVelocity, GlobalTotalEnergy), and the collision
  conserves them site by site; on an equilibrium state they equal the site
  means of rho, n u and n (eps + |u|^2/2) formed from the input fields;
* a homogeneous equilibrium is a fixed point; a homogeneous non-equilibrium
  state relaxes as (1 - dt/tau)^n exactly (streaming is the identity there);
* Hermiticity is preserved exactly; the step commutes with a global SU(2)
  rotation (Sec. 2.1); W proportional to the identity stays so, diagonal W
  stays diagonal, the spin part evolves linearly (Pauli split of Eq. WeqAlgo);
* linear sound waves travel at the speed that the equilibrium's pressure
  and energy flux imply (derived from Sec. 3.2 with FD moments integrated
  independently), an independent physical check of its moments;
* the adjoint step matches central finite differences of the forward step.
"""
import math

import numpy as np
import pytest

from paper_1309_1656_gb300 import fields

SIGMA = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]),
         np.array([[1, 0], [0, -1]], complex)]


def to_matrices(state):
    """Pauli [b][4][N] -> complex W[N][b][2][2] (test-side conversion)."""
    f = state[:, 0].T
    s = np.moveaxis(state[:, 1:], 1, 2).transpose(1, 0, 2)  # [N][b][3]
    W = 0.5 * f[..., None, None] * np.eye(2)
    for k in range(3):
        W = W + 0.5 * s[..., k, None, None] * SIGMA[k]
    return W


def from_matrices(W):
    b = W.shape[1]
    out = np.empty((b, 4, W.shape[0]))
    out[:, 0] = np.trace(W, axis1=2, axis2=3).real.T
    for k in range(3):
        out[:, 1 + k] = np.einsum("nbij,ji->nb", W, SIGMA[k]).real.T
    return out


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def nq(d):
    return 9 if d == 2 else 19


CASES = [(2, (5, 4, 1)), (2, (7, 3, 1)), (3, (4, 3, 5)), (3, (3, 3, 3))]


@pytest.mark.parametrize("d,dims", CASES)
def test_pure_streaming_is_roll(oracle_mod, d, dims):
    st = fields.random_populations(d, dims, seed=11)
    out = oracle_mod.run(d, dims, tau=1.0, beta0=1.0, nsteps=1, state=st, dt=0.0)
    c = oracle_mod.constants(d, 1.0)
    nx, ny, nz = dims
    for q in range(nq(d)):
        i1, i2, i3 = c["idx"][q]
        g = st[q].reshape(4, nz, ny, nx)
        exp = np.roll(g, shift=(i3, i2, i1), axis=(1, 2, 3)).reshape(4, -1)
        # exact up to the ulp of the Pauli <-> matrix conversion
        assert np.max(np.abs(out[q] - exp)) <= 4e-16 * np.max(np.abs(exp)), q


@pytest.mark.parametrize("d,dims", CASES)
def test_omega_one_gives_streamed_equilibrium(oracle_mod, d, dims):
    beta0 = 1.2
    st = fields.random_populations(d, dims, seed=12)
    out = oracle_mod.run(d, dims, tau=1.0, beta0=beta0, nsteps=1, state=st, dt=1.0)
    rho4, u, eps = oracle_mod.moments(d, dims, beta0, st)
    c = oracle_mod.constants(d, beta0)
    nx, ny, nz = dims
    N = nx * ny * nz
    weq = np.empty_like(st)
    for s in range(N):
        weq[:, :, s] = oracle_mod.equilibrium_site(d, beta0, rho4[:, s], u[:, s], eps[s])
    for q in range(nq(d)):
        i1, i2, i3 = c["idx"][q]
        exp = np.roll(weq[q].reshape(4, nz, ny, nx), (i3, i2, i1), axis=(1, 2, 3)).reshape(4, -1)
        assert rel(out[q], exp) < 1e-14


@pytest.mark.parametrize("d,dims", CASES)
def test_global_conservation(oracle_mod, d, dims):
    beta0 = 1.0
    st = fields.random_populations(d, dims, seed=13)
    c0 = oracle_mod.conserved(d, dims, beta0, st)
    st2 = oracle_mod.run(d, dims, tau=0.7, beta0=beta0, nsteps=6, state=st)
    c1 = oracle_mod.conserved(d, dims, beta0, st2)
    scale = np.max(np.abs(c0))
    assert np.max(np.abs(c1 - c0)) < 1e-14 * scale * 10
    # the state did change
    assert rel(st2, st) > 1e-3


@pytest.mark.parametrize("d,dims", CASES)
def test_global_averages_of_an_equilibrium_state(oracle_mod, d, dims):
    # Eqs. GlobalDensity, GlobalVelocity, GlobalTotalEnergy on an
    # equilibrium-initialised state.  The discrete equilibrium reproduces
    # rho, u and eps at every site (its moment constraints, Sec. 3.3), so the
    # averages are the site means of rho, n u and n (eps + |u|^2 / 2), formed
    # here from the input fields alone; conservation in time (above) cannot
    # see a wrong factor in these sums, this pin does.
    beta0 = 0.9
    fl = fields.random_fields(d, dims, seed=17)
    st = oracle_mod.init_equilibrium(d, dims, beta0, fl["rho4"], fl["u"], fl["eps"])
    c = oracle_mod.conserved(d, dims, beta0, st)
    n, u, eps = fl["rho4"][0], fl["u"][:d], fl["eps"]
    assert np.allclose(c[:4], fl["rho4"].mean(axis=1), rtol=0, atol=1e-14)
    assert np.allclose(c[4:4 + d], (n * u).mean(axis=1), rtol=0, atol=1e-14)
    assert np.all(c[4 + d:7] == 0.0)
    assert c[7] == pytest.approx((n * (eps + 0.5 * (u ** 2).sum(axis=0))).mean(), rel=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_local_conservation_of_collision(oracle_mod, d):
    rng = np.random.default_rng(3)
    c = oracle_mod.constants(d, 1.0)
    e = c["xi"] * c["idx"][:, :d].astype(float)
    for k in range(10):
        pops = fields.random_populations(d, (1, 1, 1), seed=100 + k)[:, :, 0]
        out = oracle_mod.collide_site(d, tau=rng.uniform(0.55, 3.0), beta0=1.0, pops=pops)
        assert np.allclose(out[:, :4].sum(0), pops.sum(0), rtol=0, atol=1e-14)
        assert np.allclose(e.T @ out[:, 0], e.T @ pops[:, 0], rtol=0, atol=1e-14)
        en = lambda p: 0.5 * ((e ** 2).sum(1) * p[:, 0]).sum()
        assert en(out) == pytest.approx(en(pops), rel=1e-14)


@pytest.mark.parametrize("d,dims", CASES)
def test_homogeneous_equilibrium_is_fixed_point(oracle_mod, d, dims):
    beta0 = 0.9
    N = int(np.prod(dims))
    rho4 = np.tile(np.array([[1.1], [0.2], [-0.3], [0.15]]), (1, N))
    u = np.tile(np.array([[0.12], [-0.07], [0.05]])[:d], (1, N))
    eps = np.full(N, 1.15 * oracle_mod.eps0(d, beta0))
    st = oracle_mod.init_equilibrium(d, dims, beta0, rho4, u, eps)
    out = oracle_mod.run(d, dims, tau=0.6, beta0=beta0, nsteps=5, state=st)
    assert rel(out, st) < 5e-14


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("tau", [0.6, 1.0, 2.5])
def test_homogeneous_relaxation_closed_form(oracle_mod, d, tau):
    # Uniform W: streaming is the identity and moments are conserved, so
    # W^n - W^eq = (1 - dt/tau)^n (W^0 - W^eq) exactly.
    beta0, dims, n = 1.0, (3, 2, 2), 7
    N = int(np.prod(dims)) if d == 3 else 6
    dims = dims if d == 3 else (3, 2, 1)
    one = fields.random_populations(d, (1, 1, 1), seed=21)
    st = np.repeat(one, N, axis=2)
    rho4, u, eps = oracle_mod.moments(d, dims, beta0, st)
    weq = oracle_mod.equilibrium_site(d, beta0, rho4[:, 0], u[:, 0], eps[0])
    out = oracle_mod.run(d, dims, tau=tau, beta0=beta0, nsteps=n, state=st)
    exp = weq + (1.0 - 1.0 / tau) ** n * (one[:, :, 0] - weq)
    for s in range(N):
        # rounding of the re-evaluated equilibrium accumulates ~1 ulp per step
        assert np.allclose(out[:, :, s], exp, rtol=0, atol=5e-15 * n)


@pytest.mark.parametrize("d,dims", CASES[:3])
def test_hermiticity_exact(oracle_mod, d, dims):
    st = fields.random_populations(d, dims, seed=14)
    W = to_matrices(st)
    out = oracle_mod.run_matrix(d, dims, tau=0.8, beta0=1.0, nsteps=4, W=W)
    assert np.array_equal(out[..., 0, 1], np.conj(out[..., 1, 0]))
    assert np.all(out[..., 0, 0].imag == 0) and np.all(out[..., 1, 1].imag == 0)


def random_su2(rng):
    a = rng.normal(size=4)
    a /= np.linalg.norm(a)
    return np.array([[a[0] + 1j * a[1], a[2] + 1j * a[3]],
                     [-a[2] + 1j * a[3], a[0] - 1j * a[1]]])


@pytest.mark.parametrize("d,dims", CASES)
def test_su2_covariance(oracle_mod, d, dims):
    # Sec. 2.1: C[U W U*] = U C[W] U* for constant U in SU(2); the discrete
    # step inherits it.
    rng = np.random.default_rng(5)
    st = fields.random_populations(d, dims, seed=15)
    W = to_matrices(st)
    for _ in range(3):
        U = random_su2(rng)
        assert np.allclose(U @ U.conj().T, np.eye(2), atol=1e-15)
        rot = U @ W @ U.conj().T
        a = oracle_mod.run_matrix(d, dims, tau=0.7, beta0=1.0, nsteps=3, W=rot)
        b = U @ oracle_mod.run_matrix(d, dims, tau=0.7, beta0=1.0, nsteps=3, W=W) @ U.conj().T
        assert rel(a, b) < 5e-14


@pytest.mark.parametrize("d,dims", CASES[:3])
def test_scalar_and_diagonal_reduction(oracle_mod, d, dims):
    st = fields.random_populations(d, dims, seed=16)
    scal = st.copy()
    scal[:, 1:] = 0.0
    out = oracle_mod.run(d, dims, tau=0.75, beta0=1.0, nsteps=5, state=scal)
    assert np.all(out[:, 1:] == 0.0)  # W proportional to 1 stays so
    diag = st.copy()
    diag[:, 1:3] = 0.0
    out2 = oracle_mod.run(d, dims, tau=0.75, beta0=1.0, nsteps=5, state=diag)
    assert np.all(out2[:, 1:3] == 0.0)  # diagonal W stays diagonal
    # the trace channel does not see the spin at all
    full = oracle_mod.run(d, dims, tau=0.75, beta0=1.0, nsteps=5, state=st)
    assert rel(full[:, 0], out[:, 0]) < 5e-14


@pytest.mark.parametrize("d,dims", CASES[:3])
def test_spin_superposition(oracle_mod, d, dims):
    st = fields.random_populations(d, dims, seed=17)
    s2 = fields.random_populations(d, dims, seed=18)[:, 1:]
    a, b = 0.3, -0.7
    run = lambda s: oracle_mod.run(d, dims, tau=0.65, beta0=1.0, nsteps=4,
                                   state=np.concatenate([st[:, :1], s], axis=1))
    lhs = run(a * st[:, 1:] + b * s2)[:, 1:]
    rhs = a * run(st[:, 1:])[:, 1:] + b * run(s2)[:, 1:]
    assert rel(lhs, rhs) < 1e-13


def _fd_mean(d, beta0, power):
    """<(|p|^2/2)^power> under the weight (exp(beta0 |p|^2/2) + 1)^-1 on R^d."""
    from scipy import integrate
    from scipy.special import expit
    rad = lambda k: integrate.quad(lambda r: r ** k * expit(-beta0 * r * r / 2.0), 0.0,
                                   60.0 / math.sqrt(beta0), epsabs=0, epsrel=1e-13, limit=200)[0]
    return rad(2 * power + d - 1) / (2.0 ** power * rad(d - 1))


@pytest.mark.parametrize("d", [2, 3])
def test_linear_sound_speed(oracle_mod, d):
    # Linearising the scheme about (n, u, eps) = (1, 0, eps0): the pressure
    # tensor of W^eq is exactly (2/d) n eps (degree-4 moments, exact under the
    # rule), and its energy flux is n alpha3 beta0 <w p p> u = n m/(c beta0) u
    # with c = beta0 <w>, m = beta0^2 <w^2>, w = |p|^2/2 (Sec. 3.2).  Hence
    # small waves travel at c_s^2 = (2/d) m / (c beta0).  This is slower than
    # the Euler-limit speed gamma (2/d) eps0 of Eq. Euler (the polynomial
    # equilibrium matches rho, u, eps but not the heat flux of W_FD), by
    # 3.9 % (d = 2) and 2.9 % (d = 3).  A standing wave of u_x with
    # wavelength L cells (dx = xi) crosses zero after a quarter period.
    beta0, tau, L = 1.0, 0.55, 96
    dims = (L, 1, 1) if d == 3 else (L, 1)
    N = L
    xi = oracle_mod.constants(d, beta0)["xi"]
    cc = beta0 * _fd_mean(d, beta0, 1)
    mm = beta0 ** 2 * _fd_mean(d, beta0, 2)
    eps = cc / beta0
    x = np.arange(L)
    rho4 = np.zeros((4, N))
    rho4[0] = 1.0
    u = np.zeros((d, N))
    u[0] = 1e-5 * np.sin(2 * np.pi * x / L)
    st = oracle_mod.init_equilibrium(d, dims, beta0, rho4, u, np.full(N, eps))
    cs = math.sqrt((2.0 / d) * mm / (cc * beta0))
    cs_euler = math.sqrt((1 + 2.0 / d) * (2.0 / d) * eps)
    period = L * xi / cs
    amps = []
    for t in range(int(0.4 * period)):
        r, uu, _ = oracle_mod.moments(d, dims, beta0, st)
        amps.append(np.dot(uu[0], np.sin(2 * np.pi * x / L)))
        st = oracle_mod.run(d, dims, tau=tau, beta0=beta0, nsteps=1, state=st)
    a = np.array(amps)
    k = np.argmax(a < 0)
    assert k > 0
    t0 = k - 1 + a[k - 1] / (a[k - 1] - a[k])
    assert t0 / (0.25 * period) == pytest.approx(1.0, abs=2e-3), (t0, period)
    # and the measurement resolves the difference to the Euler speed
    assert abs(t0 / (0.25 * L * xi / cs_euler) - 1.0) > 0.02


@pytest.mark.parametrize("d,dims", [(2, (4, 3)), (3, (3, 3, 2))])
def test_adjoint_matches_finite_differences(oracle_mod, d, dims):
    rng = np.random.default_rng(9)
    beta0, tau, nsteps = 1.0, 0.7, 3
    st = fields.random_populations(d, dims, seed=19)
    cvec = rng.normal(size=st.shape)  # J = <cvec, W^n>
    J = lambda s, t=tau: float(np.sum(cvec * oracle_mod.run(d, dims, t, beta0, nsteps, s)))
    # reverse sweep
    traj = [st]
    for _ in range(nsteps):
        traj.append(oracle_mod.run(d, dims, tau, beta0, 1, traj[-1]))
    lam = cvec.copy()
    gtau = 0.0
    for k in reversed(range(nsteps)):
        lam, g = oracle_mod.adjoint_step(d, dims, tau, beta0, traj[k], lam)
        gtau += g
    for _ in range(3):
        dirv = rng.normal(size=st.shape)
        h = 1e-6
        fd = (J(st + h * dirv) - J(st - h * dirv)) / (2 * h)
        ad = float(np.sum(lam * dirv))
        assert ad == pytest.approx(fd, rel=1e-6, abs=1e-8)
    h = 1e-6
    fdt = (J(st, tau + h) - J(st, tau - h)) / (2 * h)
    assert gtau == pytest.approx(fdt, rel=1e-6, abs=1e-8)
