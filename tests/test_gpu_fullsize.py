"""Parity at the full workload sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes one by one.

Two steps from the equilibrium initial state: the collision leaves an
equilibrium unchanged, so W^1_j(y) = W^eq_j(fields(y - e_j)) and
W^2_i(x) = C_i(W^1(x - e_i)) with C the oracle's one-site collision.  The
oracle's inputs are the generator's fields at those sites (direct mode
sums); nothing comes from the GPU.  Sampled sites include the periodic
faces, edges and corners.
"""
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


def sample_sites(dims, n, seed):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    xs = list(rng.integers(0, nx, n)) + [0, nx - 1, 0, nx - 1, 0, nx - 1]
    ys = list(rng.integers(0, ny, n)) + [0, ny - 1, ny - 1, 0, 0, ny - 1]
    zs = list(rng.integers(0, nz, n)) + [0, nz - 1, 0, nz - 1, nz - 1, 0]
    return np.array([x + nx * (y + ny * z) for x, y, z in zip(xs, ys, zs)], np.int64)


def shift(dims, s, e):
    nx, ny, nz = dims
    x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
    return ((x + e[0]) % nx) + nx * (((y + e[1]) % ny) + ny * ((z + e[2]) % nz))


def expected_after_two_steps(oracle_mod, d, dims, tau, beta0, field_at, sites):
    c = oracle_mod.constants(d, beta0)
    idx = c["idx"]
    b = len(idx)
    # all sites x - e_i - e_j
    need = set()
    for s in sites:
        for i in range(b):
            y = shift(dims, s, -idx[i])
            for j in range(b):
                need.add(int(shift(dims, y, -idx[j])))
    need = np.array(sorted(need), np.int64)
    fl = field_at(need)
    pos = {int(s): k for k, s in enumerate(need)}
    eps0 = oracle_mod.eps0(d, beta0)
    weq_cache = {}

    def weq(z):
        if z not in weq_cache:
            k = pos[z]
            e = eps0 if fl["eps"] is None else fl["eps"][k]
            weq_cache[z] = oracle_mod.equilibrium_site(d, beta0, fl["rho4"][:, k], fl["u"][:, k], e)
        return weq_cache[z]

    out = np.empty((len(sites), b, 4))
    for a, s in enumerate(sites):
        for i in range(b):
            y = shift(dims, s, -idx[i])
            w1 = np.array([weq(int(shift(dims, y, -idx[j])))[j] for j in range(b)])
            out[a, i] = oracle_mod.collide_site(d, tau, beta0, w1)[i]
    return out


def run_and_sample(q, d, dims, tau, beta0, prec, fl, sites):
    import torch
    b = 9 if d == 2 else 19
    N = int(np.prod(dims))
    with q.Lattice(d, dims, tau, beta0, precision=prec) as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(2)
        lat.sync()
        st = torch.empty((b, 4, N), dtype=torch.float64, device="cuda")
        q.qlbm_get_state(lat.h, st)
        idx = torch.from_numpy(sites).cuda()
        got = st[:, :, idx].permute(2, 0, 1).cpu().numpy()
        del st
    return got


def check(got, exp, tol):
    err = np.max(np.abs(got - exp)) / np.max(np.abs(exp))
    assert err < tol, err


def storage_tol(oracle_mod, d, beta0, exp, prec):
    """Bound for single/half storage, derived from the arithmetic.  The
    kernels hold deviations from the reference equilibrium (f_i - w_i, and
    s_i) of size at most D = max|deviation|.  Per step, each stored value is
    rounded once to the storage unit roundoff u_s (2^-24 single, 2^-11
    half), and the rest population, which takes the exact mass and spin
    balance, collects the float (u_a = 2^-24) roundings of a b-term sum
    plus two more operations.  Over the two steps, normwise relative to the
    largest population:  2 ((b + 2) u_a + u_s) D / max|W|."""
    if prec in ("fp64", "fp64df", "df64"):
        return 2e-12
    c = oracle_mod.constants(d, beta0)
    w, b = c["w"], c["b"]
    dev = exp.copy()
    dev[:, :, 0] -= w[None, :]
    ua = 2.0 ** -24
    us = ua if prec == "fp32" else 2.0 ** -11
    return 2.0 * ((b + 2) * ua + us) * np.max(np.abs(dev)) / np.max(np.abs(exp))


@pytest.mark.parametrize("prec", ["fp64", "fp64df", "df64", "fp32", "fp16dev"])
def test_d3q19_128_bench_configuration(q, oracle_mod, prec):
    d, dims, tau, beta0 = 3, (128, 128, 128), 0.7, 1.0
    fl = fields.modes(3, dims, seed=2)
    sites = sample_sites(dims, 96, seed=1)
    got = run_and_sample(q, d, dims, tau, beta0, prec, fl, sites)
    exp = expected_after_two_steps(oracle_mod, d, dims, tau, beta0,
                                   lambda s: fields.modes(3, dims, seed=2, sites=s), sites)
    check(got, exp, storage_tol(oracle_mod, d, beta0, exp, prec))


@pytest.mark.parametrize("prec", ["fp32", "fp16dev", "df64", "fp64df"])
def test_d2q9_4096_shear_layer(q, oracle_mod, prec):
    d, dims, tau, beta0 = 2, (4096, 4096, 1), 0.7, 1.0
    fl = fields.shear2d(4096, 4096, seed=3)

    def field_at(s):
        return {k: (v[..., s] if v is not None else None) for k, v in fl.items()}

    sites = sample_sites(dims, 96, seed=2)
    got = run_and_sample(q, d, dims, tau, beta0, prec, fl, sites)
    exp = expected_after_two_steps(oracle_mod, d, dims, tau, beta0, field_at, sites)
    check(got, exp, storage_tol(oracle_mod, d, beta0, exp, prec))


@pytest.mark.slow
def test_d3q19_512_throughput_configuration(q, oracle_mod):
    """The 512^3 workload bench.py times: fields synthesised on the device
    (qlbm_fourier_field) and fed to the init as device tensors, exactly as
    the bench does; expected values from the generator's direct mode sums
    at the sampled sites."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 140e9:
        pytest.skip("needs ~130 GB of free device memory")
    d, dims, tau, beta0 = 3, (512, 512, 512), 0.6, 1.0
    fl = q.fields_on_device(fields.mode_spec(3, dims, seed=5), dims)
    sites = sample_sites(dims, 32, seed=3)
    got = run_and_sample(q, d, dims, tau, beta0, "fp32", fl, sites)
    del fl
    torch.cuda.empty_cache()
    exp = expected_after_two_steps(oracle_mod, d, dims, tau, beta0,
                                   lambda s: fields.modes(3, dims, seed=5, sites=s), sites)
    check(got, exp, storage_tol(oracle_mod, d, beta0, exp, "fp32"))
