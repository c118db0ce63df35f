"""Pins of the oracle's magnetic-field term (Sec. 5, Eq. sigmaB_comm):
-i[mu sigma.B, W] gives ds/dt = 2 mu B x s, so over n steps without
collisions every Bloch vector turns by 2 mu |B| n dt about B (Rodrigues'
formula, computed here independently of the oracle's matrix conjugation);
with collisions the total spin precesses the same way while density,
momentum and energy are conserved; the step stays SU(2) covariant when the
field is rotated with the state; the adjoint matches finite differences.
The same for a field B(x) that varies over the lattice: each population
turns at the site it leaves (followed along its path with Rodrigues'
formula per site), a field parallel to every spin changes nothing, a
constant array equals the uniform field, and covariance, conservation and
the adjoint hold as before."""
import math

import numpy as np
import pytest

from paper_1309_1656_gb300 import fields


def rodrigues(B, theta):
    b = np.asarray(B, float) / np.linalg.norm(B)
    K = np.array([[0, -b[2], b[1]], [b[2], 0, -b[0]], [-b[1], b[0], 0]])
    return np.eye(3) + math.sin(theta) * K + (1 - math.cos(theta)) * K @ K


@pytest.fixture
def field(oracle_mod):
    yield oracle_mod
    oracle_mod.set_field(0.0, (0, 0, 0))


@pytest.mark.parametrize("d,dims", [(2, (5, 4, 1)), (3, (3, 3, 2))])
def test_free_precession(field, d, dims):
    o = field
    mu, B, n = 0.37, (0.3, -1.1, 0.8), 5
    o.set_field(mu, B)
    st = fields.random_populations(d, dims, seed=3)
    out = o.run(d, dims, tau=1e15, beta0=1.0, nsteps=n, state=st)
    R = rodrigues(B, 2 * mu * np.linalg.norm(B) * n)
    exp = st.copy()
    exp[:, 1:] = np.einsum("ij,qjn->qin", R, st[:, 1:])
    # streaming moves populations; compare site-independent totals per direction
    assert np.allclose(out[:, 0].sum(1), st[:, 0].sum(1), rtol=1e-13)
    assert np.allclose(out[:, 1:].sum(2), exp[:, 1:].sum(2), rtol=1e-12, atol=1e-13)
    # a uniform state is not moved by streaming: check site by site
    one = np.repeat(st[:, :, :1], st.shape[2], axis=2)
    out1 = o.run(d, dims, tau=1e15, beta0=1.0, nsteps=n, state=one)
    assert np.allclose(out1[:, 1:], np.einsum("ij,qjn->qin", R, one[:, 1:]), rtol=1e-12, atol=1e-14)
    # sense of rotation: B along z turns x towards +y
    o.set_field(0.1, (0, 0, 1.0))
    s = one.copy()
    s[:, 1:] = 0.0
    s[:, 1] = 0.01
    o2 = o.run(d, dims, tau=1e15, beta0=1.0, nsteps=1, state=s)
    assert np.all(o2[:, 2] > 0)


@pytest.mark.parametrize("d,dims", [(2, (6, 5, 1)), (3, (4, 3, 3))])
def test_total_spin_precesses_with_collisions(field, d, dims):
    o = field
    mu, B, n = 0.21, (0.5, 0.2, -0.9), 6
    o.set_field(mu, B)
    st = fields.random_populations(d, dims, seed=4)
    c0 = o.conserved(d, dims, 1.0, st)
    out = o.run(d, dims, tau=0.7, beta0=1.0, nsteps=n, state=st)
    c1 = o.conserved(d, dims, 1.0, out)
    R = rodrigues(B, 2 * mu * np.linalg.norm(B) * n)
    assert np.allclose(c1[1:4], R @ c0[1:4], rtol=1e-12, atol=1e-14)
    assert c1[0] == pytest.approx(c0[0], rel=1e-14)
    assert np.allclose(c1[4:], c0[4:], rtol=1e-13, atol=1e-14)


def test_su2_covariance_with_rotated_field(field):
    o = field
    d, dims = 3, (3, 3, 2)
    rng = np.random.default_rng(1)
    a = rng.normal(size=4)
    a /= np.linalg.norm(a)
    V = np.array([[a[0] + 1j * a[1], a[2] + 1j * a[3]], [-a[2] + 1j * a[3], a[0] - 1j * a[1]]])
    sig = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    # rotation matrix of V: (V s.sigma V*) = (Rv s).sigma
    Rv = np.array([[0.5 * np.trace(V @ sig[j] @ V.conj().T @ sig[i]).real for j in range(3)] for i in range(3)])
    B = np.array([0.4, -0.3, 0.7])
    st = fields.random_populations(d, dims, seed=6)
    from test_oracle_step import to_matrices
    W = to_matrices(st)
    o.set_field(0.3, B)
    a1 = V @ o.run_matrix(d, dims, 0.8, 1.0, 3, W) @ V.conj().T
    o.set_field(0.3, Rv @ B)
    a2 = o.run_matrix(d, dims, 0.8, 1.0, 3, V @ W @ V.conj().T)
    assert np.max(np.abs(a1 - a2)) < 1e-13 * np.max(np.abs(a1))


def test_adjoint_with_field(field):
    o = field
    d, dims, tau, beta0, nsteps = 3, (3, 3, 2), 0.7, 1.0, 3
    o.set_field(0.45, (0.2, 0.9, -0.4))
    rng = np.random.default_rng(12)
    st = fields.random_populations(d, dims, seed=19)
    cvec = rng.normal(size=st.shape)
    J = lambda s, t=tau: float(np.sum(cvec * o.run(d, dims, t, beta0, nsteps, s)))
    traj = [st]
    for _ in range(nsteps):
        traj.append(o.run(d, dims, tau, beta0, 1, traj[-1]))
    lam, gtau = cvec.copy(), 0.0
    for k in reversed(range(nsteps)):
        lam, g = o.adjoint_step(d, dims, tau, beta0, traj[k], lam)
        gtau += g
    h = 1e-6
    for _ in range(3):
        dv = rng.normal(size=st.shape)
        fd = (J(st + h * dv) - J(st - h * dv)) / (2 * h)
        assert float(np.sum(lam * dv)) == pytest.approx(fd, rel=1e-6, abs=1e-8)
    fdt = (J(st, tau + h) - J(st, tau - h)) / (2 * h)
    assert gtau == pytest.approx(fdt, rel=1e-6, abs=1e-8)


# ---------------------------------------------------------------------------
# A field that varies over the lattice, B(x) (Sec. 5: -i[mu sigma.B(x,t), W])
# ---------------------------------------------------------------------------

def site_field(d, dims, seed):
    N = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(3, N)) * rng.uniform(0.2, 1.5, N)
    B[:, :: 7] = 0.0          # some sites without field
    return B


def shift_index(dims, e):
    """flat index of x + e for every site x"""
    nx, ny, nz = dims
    s = np.arange(nx * ny * nz)
    x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
    return ((x + e[0]) % nx) + nx * (((y + e[1]) % ny) + ny * ((z + e[2]) % nz))


def lattice_vectors(d):
    out = []
    for i3 in ((-1, 0, 1) if d == 3 else (0,)):
        for i2 in (-1, 0, 1):
            for i1 in (-1, 0, 1):
                if abs(i1) + abs(i2) + abs(i3) <= 2:
                    out.append((i1, i2, i3))
    return out


@pytest.fixture
def site_field_off(oracle_mod):
    yield oracle_mod
    oracle_mod.set_field_array(0.0, None)
    oracle_mod.set_field(0.0, (0, 0, 0))


@pytest.mark.parametrize("d,dims", [(2, (5, 4, 1)), (3, (4, 3, 3))])
def test_site_field_free_precession_rodrigues(site_field_off, d, dims):
    # without collisions (tau -> infinity) a population's Bloch vector turns,
    # at every site it leaves, by 2 mu |B(x)| dt about B(x) and then streams
    # to x + e_i: follow each population along its path for n steps with
    # Rodrigues' formula per site
    o = site_field_off
    mu, n = 0.31, 3
    B = site_field(d, dims, 5)
    o.set_field_array(mu, B)
    st = fields.random_populations(d, dims, seed=13)
    out = o.run(d, dims, tau=1e15, beta0=1.0, nsteps=n, state=st)
    exp = st.copy()
    N = int(np.prod(dims))
    Rs = [rodrigues(B[:, x], 2 * mu * np.linalg.norm(B[:, x])) if np.any(B[:, x]) else np.eye(3) for x in range(N)]
    for _ in range(n):
        nxt = np.empty_like(exp)
        for q, e in enumerate(lattice_vectors(d)):
            t = shift_index(dims, e)
            rot = np.einsum("xij,jx->ix", np.array(Rs), exp[q, 1:])
            nxt[q, 0, t] = exp[q, 0]
            nxt[q][1:, t] = rot
        exp = nxt
    assert np.allclose(out, exp, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("d,dims", [(2, (6, 5, 1)), (3, (4, 3, 3))])
def test_site_field_parallel_to_every_spin_changes_nothing(site_field_off, d, dims):
    # every Bloch vector along z and B(x) along z with a varying magnitude:
    # each rotation leaves every spin as it is, so the run equals the run
    # without field
    o = site_field_off
    st = fields.random_populations(d, dims, seed=14)
    st[:, 1] = 0.0
    st[:, 2] = 0.0
    N = int(np.prod(dims))
    B = np.zeros((3, N))
    B[2] = np.linspace(-1.3, 2.1, N)
    ref = o.run(d, dims, 0.7, 1.0, 4, st)
    o.set_field_array(0.8, B)
    got = o.run(d, dims, 0.7, 1.0, 4, st)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
    # a field not parallel to the spins does change them (the pin has teeth)
    B[0] = 0.5
    o.set_field_array(0.8, B)
    assert np.max(np.abs(o.run(d, dims, 0.7, 1.0, 4, st) - ref)) > 1e-3


def test_site_field_constant_equals_uniform_field(site_field_off):
    o = site_field_off
    d, dims = 3, (4, 3, 3)
    N = int(np.prod(dims))
    Bv = (0.3, -1.1, 0.8)
    st = fields.random_populations(d, dims, seed=15)
    o.set_field(0.37, Bv)
    a = o.run(d, dims, 0.7, 1.0, 3, st)
    o.set_field_array(0.37, np.repeat(np.array(Bv)[:, None], N, axis=1))
    b = o.run(d, dims, 0.7, 1.0, 3, st)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("d,dims", [(2, (6, 5, 1)), (3, (4, 3, 3))])
def test_site_field_conserves_density_momentum_energy(site_field_off, d, dims):
    o = site_field_off
    st = fields.random_populations(d, dims, seed=16)
    o.set_field_array(0.4, site_field(d, dims, 6))
    c0 = o.conserved(d, dims, 1.0, st)
    c1 = o.conserved(d, dims, 1.0, o.run(d, dims, 0.7, 1.0, 5, st))
    assert c1[0] == pytest.approx(c0[0], rel=1e-14)
    assert np.allclose(c1[4:], c0[4:], rtol=1e-13, atol=1e-14)
    # the total spin is not conserved by a non-uniform field
    assert np.max(np.abs(c1[1:4] - c0[1:4])) > 1e-6


def test_site_field_su2_covariance(site_field_off):
    # rotating the state by V and every site's field by the same rotation
    # commutes with the step
    o = site_field_off
    d, dims = 3, (3, 3, 2)
    rng = np.random.default_rng(2)
    a = rng.normal(size=4)
    a /= np.linalg.norm(a)
    V = np.array([[a[0] + 1j * a[1], a[2] + 1j * a[3]], [-a[2] + 1j * a[3], a[0] - 1j * a[1]]])
    sig = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    Rv = np.array([[0.5 * np.trace(V @ sig[j] @ V.conj().T @ sig[i]).real for j in range(3)] for i in range(3)])
    B = site_field(d, dims, 7)
    st = fields.random_populations(d, dims, seed=17)
    from test_oracle_step import to_matrices
    W = to_matrices(st)
    o.set_field_array(0.3, B)
    a1 = V @ o.run_matrix(d, dims, 0.8, 1.0, 3, W) @ V.conj().T
    o.set_field_array(0.3, Rv @ B)
    a2 = o.run_matrix(d, dims, 0.8, 1.0, 3, V @ W @ V.conj().T)
    assert np.max(np.abs(a1 - a2)) < 1e-13 * np.max(np.abs(a1))


def test_site_field_adjoint_vs_finite_differences(site_field_off):
    o = site_field_off
    d, dims, tau, beta0, nsteps = 3, (3, 3, 2), 0.7, 1.0, 3
    o.set_field_array(0.45, site_field(d, dims, 8))
    rng = np.random.default_rng(22)
    st = fields.random_populations(d, dims, seed=23)
    cvec = rng.normal(size=st.shape)
    J = lambda s, t=tau: float(np.sum(cvec * o.run(d, dims, t, beta0, nsteps, s)))
    traj = [st]
    for _ in range(nsteps):
        traj.append(o.run(d, dims, tau, beta0, 1, traj[-1]))
    lam, gtau = cvec.copy(), 0.0
    for k in reversed(range(nsteps)):
        lam, g = o.adjoint_step(d, dims, tau, beta0, traj[k], lam)
        gtau += g
    h = 1e-6
    for _ in range(3):
        dv = rng.normal(size=st.shape)
        fd = (J(st + h * dv) - J(st - h * dv)) / (2 * h)
        assert float(np.sum(lam * dv)) == pytest.approx(fd, rel=1e-6, abs=1e-8)
    fdt = (J(st, tau + h) - J(st, tau - h)) / (2 * h)
    assert gtau == pytest.approx(fdt, rel=1e-6, abs=1e-8)


def test_site_field_size_must_match_the_lattice(site_field_off):
    o = site_field_off
    o.set_field_array(0.3, np.ones((3, 10)))
    with pytest.raises(RuntimeError):
        o.run(2, (4, 4, 1), 0.7, 1.0, 1, fields.random_populations(2, (4, 4, 1), seed=1))
