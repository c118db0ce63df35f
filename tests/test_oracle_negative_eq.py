"""Pins of the oracle's negative-eigenvalue diagnostic of the discrete
equilibrium (Sec. 3.2 end, Sec. 3.3 end: W_i^eq = w_i rho P_i, Eq. WeqAlgo,
can have negative eigenvalues; the scheme neither clips them nor adapts tau).

The expected sign patterns follow from the appendix coefficients without
evaluating them here: at u = 0, P_i = alpha1 + alpha2 beta0 |e_i|^2/2 with
alpha1 = 1 - c alpha2 and alpha2 proportional to beta0 eps - c, so
  * far above the reference temperature (beta0 eps >> c) only the rest
    direction has P_i < 0 (its P is alpha1, the others gain alpha2 K |i|^2);
  * far below it (beta0 eps << c) only the diagonal class |i|^2 = 2 has
    P_i < 0 (alpha2 < 0 weighs most there) while P_rest = alpha1 > 1;
  * at eps = eps0 every P_i = 1 > 0.
The eigenvalues of w_i P_i rho are w_i P_i (n +- |S|)/2, so an indefinite rho
(|S| > n) makes every direction with P_i > 0 negative, and a pure state
(|S| = n) has a zero eigenvalue, which is not negative.  The directions are
enumerated here in the documented order (i1 fastest, then i2, then i3;
D3Q19 without the corners), independently of the oracle's tables."""
import numpy as np
import pytest

from paper_1309_1656_gb300 import fields


def lattice_vectors(d):
    out = []
    for i3 in ((-1, 0, 1) if d == 3 else (0,)):
        for i2 in (-1, 0, 1):
            for i1 in (-1, 0, 1):
                if abs(i1) + abs(i2) + abs(i3) <= 2:
                    out.append((i1, i2, i3))
    return np.array(out)


def mask_of(directions):
    m = 0
    for q in directions:
        m |= 1 << int(q)
    return m


def uniform_state(o, d, dims, n, S, eps, u=None):
    N = int(np.prod(dims))
    r4 = np.zeros((4, N))
    r4[0] = n
    r4[1:] = np.asarray(S, float)[:, None]
    uu = np.zeros((d, N)) if u is None else np.repeat(np.asarray(u, float)[:d, None], N, axis=1)
    e = None if eps is None else np.full(N, float(eps))
    return o.init_equilibrium(d, dims, 1.0, r4, uu, e)


CASES = [(2, (4, 3, 1)), (3, (3, 3, 2))]
S_GENERIC = (0.21, -0.33, 0.17)    # |S| = 0.43 < n = 1, components along every axis


@pytest.mark.parametrize("d,dims", CASES)
def test_hot_equilibrium_negative_in_the_rest_direction_only(oracle_mod, d, dims):
    iv = lattice_vectors(d)
    rest = [q for q, v in enumerate(iv) if not v.any()]
    N = int(np.prod(dims))
    st = uniform_state(oracle_mod, d, dims, 1.0, S_GENERIC, eps=4.0)
    count, mask = oracle_mod.negative_eq(d, dims, 1.0, st)
    assert count == N
    assert np.all(mask == mask_of(rest))


@pytest.mark.parametrize("d,dims", CASES)
def test_cold_equilibrium_negative_in_the_diagonal_class_only(oracle_mod, d, dims):
    iv = lattice_vectors(d)
    diag = [q for q, v in enumerate(iv) if (v * v).sum() == 2]
    N = int(np.prod(dims))
    st = uniform_state(oracle_mod, d, dims, 1.3, S_GENERIC, eps=0.15)
    count, mask = oracle_mod.negative_eq(d, dims, 1.0, st)
    assert count == len(diag) * N
    assert np.all(mask == mask_of(diag))


@pytest.mark.parametrize("d,dims", CASES)
def test_reference_temperature_has_no_negative_equilibrium(oracle_mod, d, dims):
    st = uniform_state(oracle_mod, d, dims, 0.8, S_GENERIC, eps=None)
    count, mask = oracle_mod.negative_eq(d, dims, 1.0, st)
    assert count == 0 and not mask.any()
    lmin = oracle_mod.eq_min_eigenvalues(d, dims, 1.0, st)
    # at eps0 and u = 0, P_i = 1: the smallest eigenvalue of w_i rho is
    # w_i (n - |S|)/2, in every direction
    w = np.array([st[q, 0, 0] / 0.8 for q in range(st.shape[0])])
    exp = w * (0.8 - np.linalg.norm(S_GENERIC)) / 2
    assert np.allclose(lmin[:, 0], exp, rtol=1e-13)


@pytest.mark.parametrize("d,dims", CASES)
def test_indefinite_density_matrix_makes_every_direction_negative(oracle_mod, d, dims):
    b = len(lattice_vectors(d))
    N = int(np.prod(dims))
    S = np.array(S_GENERIC) / np.linalg.norm(S_GENERIC) * 1.4      # |S| = 1.4 > n = 1
    st = uniform_state(oracle_mod, d, dims, 1.0, S, eps=None)
    count, mask = oracle_mod.negative_eq(d, dims, 1.0, st)
    assert count == b * N
    assert np.all(mask == (1 << b) - 1)


@pytest.mark.parametrize("d,dims", CASES)
def test_pure_state_is_not_negative(oracle_mod, d, dims):
    # |S| = n exactly along z: rho = diag(n, 0), eigenvalue 0 is not negative
    st = uniform_state(oracle_mod, d, dims, 1.0, (0.0, 0.0, 1.0), eps=None)
    count, _ = oracle_mod.negative_eq(d, dims, 1.0, st)
    assert count == 0
    assert np.all(oracle_mod.eq_min_eigenvalues(d, dims, 1.0, st) == 0.0)


@pytest.mark.parametrize("d,dims", [(2, (6, 5, 1)), (3, (4, 3, 3))])
def test_mask_invariant_under_spin_rotation_and_positive_scaling(oracle_mod, d, dims):
    # a global SU(2) rotation turns every Bloch vector by the same SO(3)
    # rotation R, and scaling all populations by a > 0 leaves u and eps
    # unchanged: neither changes which W_i^eq have a negative eigenvalue
    st = fields.random_populations(d, dims, seed=8, fmin=0.005, fmax=0.3, spin_frac=0.95)
    count, mask = oracle_mod.negative_eq(d, dims, 1.0, st)
    assert count > 0     # random populations far from equilibrium give some
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(1.1), -np.sin(1.1)], [0, np.sin(1.1), np.cos(1.1)]])
    rot = st.copy()
    rot[:, 1:] = np.einsum("ij,qjn->qin", R, st[:, 1:])
    c2, m2 = oracle_mod.negative_eq(d, dims, 1.0, rot)
    assert c2 == count and np.array_equal(m2, mask)
    c3, m3 = oracle_mod.negative_eq(d, dims, 1.0, 2.5 * st)
    assert c3 == count and np.array_equal(m3, mask)
