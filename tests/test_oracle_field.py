"""Pins of the oracle's magnetic-field term (Sec. 5, Eq. sigmaB_comm):
-i[mu sigma.B, W] gives ds/dt = 2 mu B x s, so over n steps without
collisions every Bloch vector turns by 2 mu |B| n dt about B (Rodrigues'
formula, computed here independently of the oracle's matrix conjugation);
with collisions the total spin precesses the same way while density,
momentum and energy are conserved; the step stays SU(2) covariant when the
field is rotated with the state; the adjoint matches finite differences."""
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
