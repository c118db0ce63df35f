"""The row-pipelined FP16 step (each block updates several consecutive rows
and copies the next row's vectors into shared memory while the current row
computes).  Lattices here are sized so that blocks take more than one row and
the last block of the grid a ragged remainder, in both AA parities and with
the magnetic-field rotation; the state must equal, bit for bit, that of the
fused step-with-FD-output kernel (one site per thread, same collision), and
follow the FP64 oracle within the FP16 storage bound."""
import numpy as np
import pytest

from paper_1309_1656_gb300 import fields

pytestmark = pytest.mark.gpu

MIN_BLOCKS_FP16 = {2: 6, 3: 4}     # resident step blocks per SM (launch bounds)
ROWS_MAX = {2: 8, 3: 4}


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1309_1656_gb300 import qlbm
    return qlbm


def block_width(nx):
    if nx <= 128:
        return (nx + 31) // 32 * 32
    best, idle = 128, (128 - nx % 128) % 128
    for bx in (96, 64):
        i = (bx - nx % bx) % bx
        if i < idle:
            best, idle = bx, i
    return best


def rows_per_block(d, dims):
    """The launcher's rule: ROWS_MAX, or fewer to keep four waves."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nx, ny, nz = dims
    nxb = -(-nx // block_width(nx))
    blocks = nxb * ny * nz
    return max(1, min(ROWS_MAX[d], blocks // (4 * MIN_BLOCKS_FP16[d] * sms)))


def shapes():
    """(d, nx, rows per block wanted, ragged remainder): the row count is
    derived from the device's SM count so that the rule picks exactly that
    many rows per block."""
    return [(2, 32, 8, 3), (3, 32, 4, 1), (3, 150, 2, 1)]


def dims_for(d, nx, r, extra, sms=None):
    if sms is None:
        import torch
        sms = torch.cuda.get_device_properties(0).multi_processor_count
    wave4 = 4 * MIN_BLOCKS_FP16[d] * sms
    nxb = -(-nx // block_width(nx))
    rows_min = -(-wave4 * r // nxb)       # fewest rows giving r rows per block
    if d == 2:
        return (nx, rows_min + (extra - rows_min) % r, 1)
    nz = 7
    ny = -(-rows_min // nz)
    while (ny * nz) % r != extra % r:
        ny += 1
    return (nx, ny, nz)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("shape", shapes(), ids=lambda s: "d%d-nx%d-r%d" % s[:3])
@pytest.mark.parametrize("field", [False, True])
def test_rows_step_equals_site_kernel(q, shape, field):
    d, nx, r, extra = shape
    dims = dims_for(d, nx, r, extra)
    assert rows_per_block(d, dims) == r
    assert (dims[1] * dims[2]) % r != 0
    fl = fields.random_fields(d, dims, seed=31, umax=0.1)
    with q.Lattice(d, dims, 0.7, 1.0, precision="fp16dev") as a, \
            q.Lattice(d, dims, 0.7, 1.0, precision="fp16dev") as b:
        for lat in (a, b):
            if field:
                lat.set_magnetic_field(0.3, (0.4, -0.25, 0.9))
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            lat.step(3)
        assert np.array_equal(a.get_state(), b.get_state())
        for _ in range(2):      # an even and an odd step
            a.step(1)
            out = b.step_fd_output()
            assert out[4] == 0
            assert np.array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("shape", shapes(), ids=lambda s: "d%d-nx%d-r%d" % s[:3])
def test_rows_step_vs_oracle(q, oracle_mod, shape):
    # bound as for the two-step sampled checks, over n steps: each step
    # rounds every stored value once to half precision (u_s = 2^-11) and the
    # rest population collects the float roundings (u_a = 2^-24) of a b-term
    # sum plus two operations, on deviations of size D:
    #   n ((b + 2) u_a + u_s) D / max|W|, normwise relative
    d, nx, r, extra = shape
    dims = dims_for(d, nx, r, extra)
    n, tau, beta0 = 5, 0.7, 1.0
    fl = fields.random_fields(d, dims, seed=32, umax=0.1)
    with q.Lattice(d, dims, tau, beta0, precision="fp16dev") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(n)
        got = lat.get_state()
    st = oracle_mod.init_equilibrium(d, dims, beta0, fl["rho4"], fl["u"], fl["eps"])
    exp = oracle_mod.run(d, dims, tau, beta0, n, st)
    c = oracle_mod.constants(d, beta0)
    dev = exp.copy()
    dev[:, 0, :] -= c["w"][:, None]
    tol = n * ((c["b"] + 2) * 2.0 ** -24 + 2.0 ** -11) * np.max(np.abs(dev)) / np.max(np.abs(exp))
    assert rel(got, exp) < tol
