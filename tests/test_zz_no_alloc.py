"""The allocation-free entry point qlbm_conserved_static.

It serves callers that cannot allocate device memory where they need the
conserved sums (code under another component's memory manager, or loops
that cannot afford cudaMalloc/cudaFree).  This test calls it through the C
ABI on caller-owned device buffers and checks it against qlbm_conserved,
which computes the same averages from the handle's own buffer, on two
calls in a row sharing the library's fixed scratch array, and against the
FP64 oracle on host-generated states, including lattices larger than one
pass of the fixed scratch and a call on a non-default stream.  The file name
makes pytest collect it last; it also runs alone in a fresh process.
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
    import __graft_entry__
    from paper_1309_1656_gb300 import _build
    if not _build.up_to_date():
        __graft_entry__.build()
    from paper_1309_1656_gb300 import qlbm
    return qlbm


@pytest.mark.parametrize("d,dims", [(2, (130, 37, 1)), (3, (33, 20, 9))])
def test_conserved_static_matches_conserved(q, oracle_mod, d, dims):
    import torch
    b = 9 if d == 2 else 19
    N = int(np.prod(dims))
    beta0 = 1.2
    fl = fields.random_fields(d, dims, seed=31)
    with q.Lattice(d, dims, 0.7, beta0, precision="fp64") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(3)
        state = torch.zeros((b, 4, N), dtype=torch.float64, device="cuda")
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        for call in range(2):
            q.qlbm_get_state(lat.h, state)
            ref = lat.conserved()
            q.qlbm_conserved_static(d, dims, beta0, state, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            scale = np.max(np.abs(ref))
            assert np.all(np.isfinite(got)), call
            assert np.max(np.abs(got - ref)) <= 1e-12 * scale, (call, got, ref)
            lat.step(2)  # the second call sees a different state
    # and against the oracle on a host-generated state
    st = fields.random_populations(d, dims, seed=33)
    state = torch.from_numpy(st).cuda()
    q.qlbm_conserved_static(d, dims, beta0, state, out)
    torch.cuda.synchronize()
    ref = oracle_mod.conserved(d, dims, beta0, st)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("d,dims", [(2, (600, 500, 1)), (3, (70, 66, 61))])
def test_conserved_static_large_lattice_vs_oracle(q, oracle_mod, d, dims):
    # more sites than the fixed scratch's blocks cover in one pass (1024
    # blocks of 256 threads), so the grid-stride loop runs more than once;
    # the state is generated on the host and the same array goes to the
    # oracle; one call on a non-default stream, one on the default stream
    import torch
    N = int(np.prod(dims))
    assert N > q.QLBM_STATIC_SCRATCH_BLOCKS * 256
    beta0 = 0.9
    st = fields.random_populations(d, dims, seed=32 + d)
    ref = oracle_mod.conserved(d, dims, beta0, st)
    state = torch.from_numpy(st).cuda()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    for stream in (s.cuda_stream, None):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        q.qlbm_conserved_static(d, dims, beta0, state, out, stream)
        if stream is not None:
            s.synchronize()
        else:
            torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (stream, got, ref)


def test_conserved_static_rejects_bad_sizes(q):
    import torch
    state = torch.zeros((9, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    for dims in ((2, 2, 2), (0, 2, 1), (1 << 20, 1 << 20, 1)):
        with pytest.raises(q.QLBMError) as e:
            q.qlbm_conserved_static(2, dims, 1.0, state, out)
        assert e.value.code == q.QLBM_ERR_INVALID_ARG
        assert "qlbm_conserved_static" in q.qlbm_last_error(None)
