"""The device synthesis of the Fourier-mode input fields (qlbm_fourier_field).

Its values must equal the generator's own direct mode sum
(``fields.ModeField.at``, numpy, float64) at sampled sites, including the
periodic faces, edges and corners, at the 128^3 and 512^3 workload sizes and
on ragged boxes; on a small box also against the host inverse-FFT grid.  The
bound, 1e-14 absolute on the scaled fields (amplitude ~0.02, density ~1), is
a few hundred roundings of the ~130-term sums.  The result must not depend
on the launch (deterministic), and bad arguments are refused."""
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
    xs = list(rng.integers(0, nx, n)) + [0, nx - 1, 0, nx - 1, 0, nx - 1, nx - 1]
    ys = list(rng.integers(0, ny, n)) + [0, ny - 1, ny - 1, 0, 0, ny - 1, ny - 1]
    zs = list(rng.integers(0, nz, n)) + [0, nz - 1, 0, nz - 1, nz - 1, 0, nz - 1]
    return np.array([x + nx * (y + ny * z) for x, y, z in zip(xs, ys, zs)], np.int64)


@pytest.mark.parametrize("d,dims,seed", [(3, (128, 128, 128), 2), (3, (512, 512, 512), 5),
                                         (3, (37, 29, 11), 3), (2, (300, 77, 1), 7), (2, (4096, 4096, 1), 9)])
def test_device_fields_match_direct_sum(q, d, dims, seed):
    import torch
    spec = fields.mode_spec(d, dims, seed=seed)
    dev = q.fields_on_device(spec, dims)
    sites = sample_sites(dims, 512, seed=seed)
    ref = fields.modes(d, dims, seed=seed, sites=sites)
    idx = torch.from_numpy(sites).cuda()
    for key in ("rho4", "u"):
        got = dev[key][:, idx].cpu().numpy()
        err = float(np.max(np.abs(got - ref[key])))
        assert err <= 1e-14, (key, err)
    del dev
    torch.cuda.empty_cache()


def test_device_fields_match_host_grid(q):
    d, dims, seed = 3, (24, 20, 16), 11
    dev = q.fields_on_device(fields.mode_spec(d, dims, seed=seed), dims)
    host = fields.modes(d, dims, seed=seed)
    for key in ("rho4", "u"):
        assert float(np.max(np.abs(dev[key].cpu().numpy() - host[key]))) <= 1e-14


def test_single_modes_and_launch_independence(q):
    import torch
    dims = (40, 6, 5)
    N = int(np.prod(dims))
    x = np.arange(N) % dims[0]
    y = (np.arange(N) // dims[0]) % dims[1]
    z = np.arange(N) // (dims[0] * dims[1])
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    # one cosine / one sine mode each, with offset and scale
    for k, A, B in (((3, 0, 0), 1.0, 0.0), ((0, -2, 1), 0.0, 1.0), ((-5, 1, -2), 0.3, -0.7)):
        q.qlbm_fourier_field(dims, np.array([k]), [A], [B], 2.0, 0.5, out)
        ph = 2 * np.pi * (k[0] * x / dims[0] + k[1] * y / dims[1] + k[2] * z / dims[2])
        exp = 0.5 + 2.0 * (A * np.cos(ph) + B * np.sin(ph))
        assert float(np.max(np.abs(out.cpu().numpy() - exp))) <= 1e-14, k
    # no modes: the offset
    q.qlbm_fourier_field(dims, np.zeros((0, 3)), [], [], 1.0, 0.25, out)
    assert torch.all(out == 0.25)
    # the same call twice, and on another stream: bit-identical
    f = fields.ModeField(3, dims, 4, 100, 4)
    q.qlbm_fourier_field(dims, f.k, f.A, f.B, 1.0, 0.0, out)
    a = out.clone()
    s = torch.cuda.Stream()
    q.qlbm_fourier_field(dims, f.k, f.A, f.B, 1.0, 0.0, out, s.cuda_stream)
    s.synchronize()
    assert torch.equal(a, out)


def test_bad_arguments_are_refused(q):
    import torch
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    dims = (4, 4, 4)
    too_many = np.zeros((q.QLBM_FOURIER_MAX_MODES + 1, 3), np.int64)
    big_k = np.array([[q.QLBM_FOURIER_MAX_K + 1, 0, 0]])
    for k, n, d in ((too_many, q.QLBM_FOURIER_MAX_MODES + 1, dims), (big_k, 1, dims), (np.zeros((1, 3)), 1, (4, 0, 4))):
        with pytest.raises(q.QLBMError) as e:
            q.qlbm_fourier_field(d, k, np.ones(n), np.ones(n), 1.0, 0.0, out)
        assert e.value.code == q.QLBM_ERR_INVALID_ARG
        assert "qlbm_fourier_field" in q.qlbm_last_error(None)
    with pytest.raises(ValueError):
        q.qlbm_fourier_field((8, 8, 8), np.zeros((1, 3)), [1.0], [0.0], 1.0, 0.0, out)   # out too short
