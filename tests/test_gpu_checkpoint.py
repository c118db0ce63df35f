"""Checkpoint and restart across handles.

k steps, save, a new handle, load, N - k more steps must give exactly the
state of N uninterrupted steps, in every storage precision and from either
AA parity at the save (k odd leaves the buffer in the swapped order).  The
image is the populations in the storage precision (qlbm_save_checkpoint /
qlbm_load_checkpoint), through host and device buffers.  The canonical
double layout (get_state / set_state) is exact for FP64, FP64_DF and
FP16-deviation storage; for FP32 storage it is exact except for trace
deviations below 2^-29 in magnitude (changed by at most 2^-54), and for
double-float storage a value moves by at most 2^-48 relative."""
import numpy as np
import pytest

from paper_1309_1656_gb300 import fields

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "fp64df", "df64", "fp32", "fp16dev"]


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1309_1656_gb300 import qlbm
    return qlbm


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("d,dims", [(2, (40, 30, 1)), (3, (18, 14, 10))])
def test_restart_from_checkpoint_is_bit_exact(q, d, dims, prec, k):
    import torch
    total, tau = 9, 0.75
    fl = fields.random_fields(d, dims, seed=71 + d)
    with q.Lattice(d, dims, tau, 1.0, precision=prec) as a:
        a.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        a.step(total)
        ref = a.get_state()
    with q.Lattice(d, dims, tau, 1.0, precision=prec) as b:
        b.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        b.step(k)
        img = b.save_checkpoint()
        dimg = torch.empty(q.qlbm_checkpoint_bytes(b.h), dtype=torch.uint8, device="cuda")
        q.qlbm_save_checkpoint(b.h, dimg)
        assert np.array_equal(dimg.cpu().numpy(), img)
        at_k = b.get_state()
    for src in (img, dimg):
        with q.Lattice(d, dims, tau, 1.0, precision=prec) as c:
            if isinstance(src, np.ndarray):
                c.load_checkpoint(src)
            else:
                q.qlbm_load_checkpoint(c.h, src)
            assert q.qlbm_time(c.h) == 0
            assert np.array_equal(c.get_state(), at_k)
            c.step(total - k)
            got = c.get_state()
        assert np.array_equal(got, ref), prec


def test_checkpoint_of_another_geometry_is_refused(q):
    with q.Lattice(2, (12, 10, 1), 0.8, 1.0, precision="fp32") as a, \
            q.Lattice(2, (12, 11, 1), 0.8, 1.0, precision="fp32") as b:
        img = np.zeros(q.qlbm_checkpoint_bytes(a.h), np.uint8)
        assert q.qlbm_checkpoint_bytes(b.h) > img.nbytes
        with pytest.raises(ValueError):
            b.load_checkpoint(img)


@pytest.mark.parametrize("prec", ["fp64", "fp64df", "fp16dev"])
@pytest.mark.parametrize("d,dims", [(2, (40, 30, 1)), (3, (18, 14, 10))])
def test_canonical_round_trip_is_exact(q, d, dims, prec):
    st = fields.random_populations(d, dims, seed=81)
    with q.Lattice(d, dims, 0.8, 1.0, precision=prec) as a, q.Lattice(d, dims, 0.8, 1.0, precision=prec) as b:
        a.set_state(st)
        a.step(3)                       # arbitrary stored bits, swapped parity
        img_a = a.save_checkpoint()
        b.set_state(a.get_state())
        assert np.array_equal(b.save_checkpoint(), img_a)


@pytest.mark.parametrize("d,dims", [(2, (40, 30, 1)), (3, (18, 14, 10))])
def test_canonical_round_trip_fp32_bound(q, oracle_mod, d, dims):
    # stored trace deviations d_i = f_i - w_i of at least 2^-29 survive the
    # trip get_state -> set_state exactly; smaller nonzero ones (planted
    # here) move by at most 2^-54; spin components are always exact.  The
    # stored values are read from the checkpoint images (float32 [b][N][4]).
    st = fields.random_populations(d, dims, seed=82)
    w = oracle_mod.constants(d, 1.0)["w"]
    b_ = len(w)
    N = int(np.prod(dims))
    rng = np.random.default_rng(3)
    tiny = rng.random((b_, N)) < 0.05
    st[:, 0][tiny] = (w[:, None] + rng.choice([-1, 1], (b_, N)) * 2.0 ** rng.uniform(-60, -29, (b_, N)))[tiny]
    with q.Lattice(d, dims, 0.8, 1.0, precision="fp32") as a, q.Lattice(d, dims, 0.8, 1.0, precision="fp32") as b:
        a.set_state(st)
        img_a = a.save_checkpoint().view(np.float32).reshape(b_, N, 4)
        b.set_state(a.get_state())
        img_b = b.save_checkpoint().view(np.float32).reshape(b_, N, 4)
    assert np.array_equal(img_b[:, :, 1:], img_a[:, :, 1:])
    da, db = img_a[:, :, 0].astype(np.float64), img_b[:, :, 0].astype(np.float64)
    big = np.abs(da) >= 2.0 ** -29
    assert np.array_equal(db[big], da[big])
    assert np.max(np.abs(db - da)) <= 2.0 ** -54
    assert (~big & (da != 0)).sum() > 0


def test_canonical_round_trip_df64_bound(q):
    # a double-float pair holds 48 significant bits, a double 53 (with the
    # pair's two parts possibly far apart): the trip moves a value by at most
    # 2^-48 relative
    d, dims = 3, (18, 14, 10)
    st = fields.random_populations(d, dims, seed=83)
    with q.Lattice(d, dims, 0.8, 1.0, precision="df64") as a, q.Lattice(d, dims, 0.8, 1.0, precision="df64") as b:
        a.set_state(st)
        a.step(5)
        s1 = a.get_state()
        b.set_state(s1)
        s2 = b.get_state()
    assert np.all(np.abs(s2 - s1) <= 2.0 ** -48 * np.abs(s1))
