"""The D3Q19 192^3 reverse-mode workload at full size: gradient of the total
spin magnetisation s_z in the central 32^3 box after 2000 FP32 steps with
respect to the initial spin field and tau (Eq. WeqAlgo initial state,
Fourier-mode fields, tau = 0.7, beta0 = 1), through the torch.autograd
interface with square-root checkpointing (45 checkpoints + 44 segment
states), checked by central finite differences (h = 1e-4) on 16 seeded
directions of the spin field and on tau.

The finite differences use double-float forward runs (within 1e-12 of FP64
per step, ~3 s per run here) for all 16 directions, and true FP64 runs for
two of them and for tau; the FP64 and double-float differences must agree
to far below the tolerance.  Runs about 3 minutes and holds ~200 GB of
device memory."""
import numpy as np
import pytest

from paper_1309_1656_gb300 import fields

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

L, T, TAU, BETA0, H = 192, 2000, 0.7, 1.0, 1e-4
BOX = slice(80, 112)


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 230e9:
        pytest.skip("needs ~215 GB of free device memory (89 FP32 states of 2.15 GB)")
    from paper_1309_1656_gb300 import qlbm
    return qlbm


def test_d3q19_192_spin_magnetisation_gradient(q):
    import torch
    from paper_1309_1656_gb300.autograd import rollout
    dims = (L, L, L)
    N = L ** 3
    fl = fields.modes(3, dims, seed=7)
    box = np.zeros((L, L, L), bool)        # [z][y][x], x fastest
    box[BOX, BOX, BOX] = True
    box = box.ravel()
    mask = torch.from_numpy(box).cuda()

    rho4 = torch.from_numpy(fl["rho4"]).cuda().requires_grad_(True)
    u = torch.from_numpy(fl["u"]).cuda()
    tau_t = torch.tensor(TAU, dtype=torch.float64, device="cuda", requires_grad=True)
    with q.Lattice(3, dims, TAU, BETA0, precision="fp32") as lat:
        state = rollout(lat, rho4, u, None, tau_t, T)
        J0 = state[:, 3, :][:, mask].sum()
        J0.backward()
        del state
    g_spin = rho4.grad[1:].cpu().numpy()
    g_tau = float(tau_t.grad)
    del rho4
    torch.cuda.empty_cache()

    m_rho4 = torch.empty((4, N), dtype=torch.float64, device="cuda")
    m_u = torch.empty((3, N), dtype=torch.float64, device="cuda")
    m_eps = torch.empty(N, dtype=torch.float64, device="cuda")

    def J(r4, tau, prec):
        with q.Lattice(3, dims, tau, BETA0, precision=prec) as lt:
            lt.init_equilibrium(r4, fl["u"])
            lt.step(T)
            q.qlbm_moments(lt.h, m_rho4, m_u, m_eps)
            return float(m_rho4[3][mask].sum())

    rng = np.random.default_rng(192)
    rows = []
    for k in range(16):
        dv = rng.normal(size=(3, N))
        r_p = fl["rho4"].copy()
        r_m = fl["rho4"].copy()
        r_p[1:] += H * dv
        r_m[1:] -= H * dv
        ad = float(np.sum(g_spin * dv))
        fdd = (J(r_p, TAU, "df64") - J(r_m, TAU, "df64")) / (2 * H)
        fd64 = (J(r_p, TAU, "fp64") - J(r_m, TAU, "fp64")) / (2 * H) if k < 2 else None
        rows.append((ad, fdd, fd64))
    fdtd = (J(fl["rho4"], TAU + H, "df64") - J(fl["rho4"], TAU - H, "df64")) / (2 * H)
    fdt64 = (J(fl["rho4"], TAU + H, "fp64") - J(fl["rho4"], TAU - H, "fp64")) / (2 * H)

    for k, (ad, fdd, fd64) in enumerate(rows):
        print("dir %2d  adjoint %.10e  fd(df64) %.10e (rel %.2e)%s" % (
            k, ad, fdd, abs(ad - fdd) / abs(fdd),
            "" if fd64 is None else "  fd(fp64) %.10e" % fd64))
    print("tau     adjoint %.10e  fd(df64) %.10e  fd(fp64) %.10e" % (g_tau, fdtd, fdt64))

    # The reverse mode's own error against FP64-class differences: the FP32
    # trajectory and cotangents (measured ~3e-6 relative).
    for ad, fdd, fd64 in rows:
        assert ad == pytest.approx(fdd, rel=1e-4)
        if fd64 is not None:
            assert fdd == pytest.approx(fd64, rel=1e-6)
    assert g_tau == pytest.approx(fdtd, rel=1e-4)
    assert fdtd == pytest.approx(fdt64, rel=1e-6)
