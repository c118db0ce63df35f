"""The paper's Riemann problem on the GPU, initialised from its Fermi-Dirac
parameters (qlbm_init_fd_params), against the oracle run of
test_oracle_riemann (FP64 per-step tolerance; FP32 moment fields)."""
import numpy as np
import pytest

from test_oracle_riemann import LEFT, NX, NY, RIGHT, T, TAU, riemann_initial

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1309_1656_gb300 import qlbm
    return qlbm


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12 * T), ("fp32", 1e-5)])
def test_riemann_gpu_vs_oracle(q, oracle_mod, prec, tol):
    N = NX * NY
    x = np.arange(N) % NX
    left = x < NX // 2
    beta = np.ones(N)
    mu_up = np.where(left, LEFT[0], RIGHT[0]).astype(float)
    mu_dn = np.where(left, LEFT[1], RIGHT[1]).astype(float)
    axis = np.zeros((3, N))
    axis[2] = 1.0
    with q.Lattice(2, (NX, NY, 1), TAU, 1.0, precision=prec) as lat:
        q.qlbm_init_fd_params(lat.h, beta, mu_up, mu_dn, axis, np.zeros((2, N)))
        lat.step(T)
        r, u, e = lat.moments()
    rho4, uu, eps, _ = riemann_initial(oracle_mod)
    st = oracle_mod.init_equilibrium(2, (NX, NY, 1), 1.0, rho4, uu, eps)
    st = oracle_mod.run(2, (NX, NY, 1), TAU, 1.0, T, st)
    r0, u0, e0 = oracle_mod.moments(2, (NX, NY, 1), 1.0, st)
    rel = lambda a, b: np.max(np.abs(a - b)) / np.max(np.abs(b))
    assert rel(r, r0) < tol and rel(e, e0) < tol and rel(u, u0) < tol


def test_convergence_example_fp32(q, oracle_mod):
    # the 3D convergence example (test_oracle_convergence) in FP32 on the GPU
    from paper_1309_1656_gb300 import fields
    L, T = 32, 200
    fl = fields.dichotomic3d(L)
    with q.Lattice(3, (L, L, L), 10.0, 1.0, precision="fp32") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(T)
        r, u, e = lat.moments()
    st = oracle_mod.init_equilibrium(3, (L, L, L), 1.0, fl["rho4"], fl["u"], fl["eps"])
    st = oracle_mod.run(3, (L, L, L), 10.0, 1.0, T, st)
    r0, u0, e0 = oracle_mod.moments(3, (L, L, L), 1.0, st)
    # relative to the initial amplitudes of the fluctuations (0.1 spin, 0.05 u)
    assert np.max(np.abs(r[1:] - r0[1:])) < 1e-6 * 0.1
    assert np.max(np.abs(u - u0)) < 1e-6 * 0.05
    assert np.max(np.abs(r[0] - r0[0])) < 1e-6
    assert np.max(np.abs(e - e0)) / np.max(np.abs(e0)) < 1e-6
