"""GPU parity of the reverse mode (adjoint step, checkpointed rollout, init
adjoint, autograd) against the FP64 oracle's own adjoint (written in matrix
form, independently of the kernels' Pauli form) and against central finite
differences of FP64 forward runs."""
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


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


SHAPES = [(2, (37, 5, 1)), (3, (9, 7, 5))]


@pytest.mark.parametrize("d,dims", SHAPES)
@pytest.mark.parametrize("pre_steps", [0, 1])
def test_step_adjoint_fp64_vs_oracle(q, oracle_mod, d, dims, pre_steps):
    tau, beta0 = 0.7, 1.1
    st = fields.random_populations(d, dims, seed=40 + d)
    rng = np.random.default_rng(3)
    lam_next = rng.normal(size=st.shape)
    with q.Lattice(d, dims, tau, beta0, precision="fp64") as lat:
        lat.set_state(st)
        lat.step(pre_steps)          # pre_steps = 1 leaves the AA buffer swapped
        w = lat.get_state()
        lam, g = lat.step_adjoint(lam_next)
        assert np.array_equal(lat.get_state(), w)   # state untouched
    lam_o, g_o = oracle_mod.adjoint_step(d, dims, tau, beta0, w, lam_next)
    assert rel(lam, lam_o) < 1e-12
    assert g == pytest.approx(g_o, rel=1e-11)


@pytest.mark.parametrize("d,dims", SHAPES)
@pytest.mark.parametrize("nsteps,interval", [(7, 3), (7, 0), (7, 1), (8, 8)])
def test_rollout_adjoint_fp64_vs_oracle(q, oracle_mod, d, dims, nsteps, interval):
    tau, beta0 = 0.8, 1.0
    st = fields.random_populations(d, dims, seed=50 + d)
    lam_T = np.random.default_rng(4).normal(size=st.shape)
    with q.Lattice(d, dims, tau, beta0, precision="fp64") as lat:
        lat.set_state(st)
        lat.rollout(nsteps, interval)
        end = lat.get_state()
        lam0, g = lat.rollout_adjoint(lam_T)
        assert np.array_equal(lat.get_state(), end)
    traj = [st]
    for _ in range(nsteps):
        traj.append(oracle_mod.run(d, dims, tau, beta0, 1, traj[-1]))
    assert rel(end, traj[-1]) < 1e-12 * nsteps
    lam, g_o = lam_T, 0.0
    for k in reversed(range(nsteps)):
        lam, gk = oracle_mod.adjoint_step(d, dims, tau, beta0, traj[k], lam)
        g_o += gk
    assert rel(lam0, lam) < 1e-11 * nsteps
    assert g == pytest.approx(g_o, rel=1e-10)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev"])
def test_checkpoint_interval_does_not_change_the_result(q, prec):
    # Segment states are recomputed with the two-buffer kernel; they must be
    # bit-identical to the in-place forward states, so every interval gives
    # the same cotangent.
    d, dims = 3, (12, 6, 5)
    fl = fields.random_fields(d, dims, seed=9)
    lam_T = np.random.default_rng(8).normal(size=(19, 4, int(np.prod(dims))))
    res = []
    with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.step(13)
        plain_end = lat.get_state()
    for interval in (0, 1, 2, 5, 13):
        with q.Lattice(d, dims, 0.7, 1.0, precision=prec) as lat:
            lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
            lat.rollout(13, interval)
            # a small rollout keeps every state automatically
            assert q.qlbm_rollout_interval(lat.h) == (interval or 1)
            assert np.array_equal(lat.get_state(), plain_end)
            res.append(lat.rollout_adjoint(lam_T))
    for lam, g in res[1:]:
        assert np.array_equal(lam, res[0][0])
        assert g == res[0][1]


@pytest.mark.parametrize("d,dims", [(2, (40, 24, 1)), (3, (16, 12, 10))])
def test_rollout_adjoint_fp32_vs_oracle(q, oracle_mod, d, dims):
    tau, beta0, nsteps = 0.7, 1.0, 20
    fl = fields.modes(d, dims, seed=12, amp=0.05, umax=0.1)
    lam_T = np.random.default_rng(6).normal(size=(9 if d == 2 else 19, 4, int(np.prod(dims))))
    with q.Lattice(d, dims, tau, beta0, precision="fp32") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.rollout(nsteps, 0)
        lam0, g = lat.rollout_adjoint(lam_T)
    st = oracle_mod.init_equilibrium(d, dims, beta0, fl["rho4"], fl["u"], fl["eps"])
    traj = [st]
    for _ in range(nsteps):
        traj.append(oracle_mod.run(d, dims, tau, beta0, 1, traj[-1]))
    lam, g_o = lam_T, 0.0
    for k in reversed(range(nsteps)):
        lam, gk = oracle_mod.adjoint_step(d, dims, tau, beta0, traj[k], lam)
        g_o += gk
    assert rel(lam0, lam) < 1e-5
    assert g == pytest.approx(g_o, rel=1e-4)


@pytest.mark.parametrize("d,dims", [(2, (40, 24, 1)), (3, (16, 12, 10))])
def test_rollout_adjoint_fp16dev_vs_oracle(q, oracle_mod, d, dims):
    # FP16-deviation storage: the reverse sweep runs on the half-precision
    # trajectory (float cotangents), so it differs from the oracle's exact
    # adjoint by the trajectory's own error -- half precision's 2^-11 on
    # deviations of ~5 % -- carried through the collision Jacobian over 20
    # steps: a few 1e-4, bounded here at 3e-3
    tau, beta0, nsteps = 0.7, 1.0, 20
    fl = fields.modes(d, dims, seed=12, amp=0.05, umax=0.1)
    lam_T = np.random.default_rng(6).normal(size=(9 if d == 2 else 19, 4, int(np.prod(dims))))
    with q.Lattice(d, dims, tau, beta0, precision="fp16dev") as lat:
        lat.init_equilibrium(fl["rho4"], fl["u"], fl["eps"])
        lat.rollout(nsteps, 0)
        lam0, g = lat.rollout_adjoint(lam_T)
    st = oracle_mod.init_equilibrium(d, dims, beta0, fl["rho4"], fl["u"], fl["eps"])
    traj = [st]
    for _ in range(nsteps):
        traj.append(oracle_mod.run(d, dims, tau, beta0, 1, traj[-1]))
    lam, g_o = lam_T, 0.0
    for k in reversed(range(nsteps)):
        lam, gk = oracle_mod.adjoint_step(d, dims, tau, beta0, traj[k], lam)
        g_o += gk
    print("fp16dev adjoint: lambda %.3e  dJ/dtau %.3e" % (rel(lam0, lam), abs(g - g_o) / abs(g_o)))
    assert rel(lam0, lam) < 3e-3
    assert g == pytest.approx(g_o, rel=3e-3)


@pytest.mark.parametrize("d,dims", [(2, (7, 5, 1)), (3, (4, 3, 3))])
def test_init_adjoint_vs_finite_differences(q, oracle_mod, d, dims):
    beta0 = 1.0
    N = int(np.prod(dims))
    b = 9 if d == 2 else 19
    fl = fields.random_fields(d, dims, seed=14)
    c = np.random.default_rng(2).normal(size=(b, 4, N))
    J = lambda r4, u, e: float(np.sum(c * oracle_mod.init_equilibrium(d, dims, beta0, r4, u, e)))
    with q.Lattice(d, dims, 0.7, beta0) as lat:
        g_r = np.zeros((4, N))
        g_u = np.zeros((d, N))
        g_e = np.zeros(N)
        q.qlbm_init_equilibrium_adjoint(lat.h, fl["rho4"], fl["u"], fl["eps"], c, g_r, g_u, g_e)
    rng = np.random.default_rng(5)
    h = 1e-6
    for name, grad in (("rho4", g_r), ("u", g_u), ("eps", g_e)):
        for _ in range(3):
            dv = rng.normal(size=grad.shape)
            args_p = {k: fl[k].copy() for k in ("rho4", "u", "eps")}
            args_m = {k: fl[k].copy() for k in ("rho4", "u", "eps")}
            args_p[name] = args_p[name] + h * dv
            args_m[name] = args_m[name] - h * dv
            fd = (J(args_p["rho4"], args_p["u"], args_p["eps"]) -
                  J(args_m["rho4"], args_m["u"], args_m["eps"])) / (2 * h)
            assert float(np.sum(grad * dv)) == pytest.approx(fd, rel=1e-7, abs=1e-9), name


def test_autograd_spin_magnetisation_gradient(q):
    # The D3Q19 adjoint workload at reduced size: gradient of the total spin
    # magnetisation s_z in a central box after T FP32 steps with respect to
    # the initial spin field and tau, checked by central differences of
    # FP64 forward runs (h = 1e-4) on seeded directions.
    import torch
    from paper_1309_1656_gb300.autograd import rollout
    d, L, T, tau, beta0 = 3, 24, 40, 0.7, 1.0
    dims = (L, L, L)
    N = L ** 3
    fl = fields.modes(3, dims, seed=4)
    box = np.zeros((L, L, L), bool)
    box[8:16, 8:16, 8:16] = True
    mask = torch.from_numpy(box.ravel()).cuda()
    rho4 = torch.from_numpy(fl["rho4"]).cuda().requires_grad_(True)
    u = torch.from_numpy(fl["u"]).cuda()
    tau_t = torch.tensor(tau, dtype=torch.float64, device="cuda", requires_grad=True)
    with q.Lattice(d, dims, tau, beta0, precision="fp32") as lat:
        state = rollout(lat, rho4, u, None, tau_t, T)
        Jv = state[:, 3, :][:, mask].sum()
        Jv.backward()
    g_spin = rho4.grad[1:].cpu().numpy()
    g_tau = float(tau_t.grad)

    def J64(r4, t):
        with q.Lattice(d, dims, t, beta0, precision="fp64") as l64:
            l64.init_equilibrium(r4, fl["u"])
            l64.step(T)
            st = l64.get_state()
        return float(st[:, 3, box.ravel()].sum())

    rng = np.random.default_rng(16)
    h = 1e-4
    for _ in range(4):
        dv = np.zeros_like(fl["rho4"])
        dv[1:] = rng.normal(size=(3, N))
        fd = (J64(fl["rho4"] + h * dv, tau) - J64(fl["rho4"] - h * dv, tau)) / (2 * h)
        ad = float(np.sum(g_spin * dv[1:]))
        assert ad == pytest.approx(fd, rel=1e-4, abs=1e-6)
    fdt = (J64(fl["rho4"], tau + h) - J64(fl["rho4"], tau - h)) / (2 * h)
    assert g_tau == pytest.approx(fdt, rel=1e-3, abs=1e-6)


def test_autograd_momentum_flux_gradient(q, oracle_mod):
    # observable: the momentum flux Pi_xy = sum_i e_ix e_iy tr W_i summed over
    # a box after T FP32 steps; gradient with respect to the initial density,
    # velocity and internal-energy fields and tau, against central
    # differences of FP64 forward runs (h = 1e-5)
    import torch
    from paper_1309_1656_gb300.autograd import rollout
    d, dims, T, tau, beta0 = 2, (40, 36, 1), 30, 0.75, 1.0
    N = int(np.prod(dims))
    fl = fields.random_fields(d, dims, seed=31)
    c = oracle_mod.constants(d, beta0)
    xi = c["xi"]
    idx = c["idx"]
    wxy = torch.tensor([xi * xi * i[0] * i[1] for i in idx], dtype=torch.float64, device="cuda")
    box = np.zeros((dims[1], dims[0]), bool)
    box[10:26, 12:30] = True
    box = box.ravel()
    mask = torch.from_numpy(box).cuda()
    rho4 = torch.from_numpy(fl["rho4"]).cuda().requires_grad_(True)
    u = torch.from_numpy(fl["u"]).cuda().requires_grad_(True)
    eps = torch.from_numpy(fl["eps"]).cuda().requires_grad_(True)
    tau_t = torch.tensor(tau, dtype=torch.float64, device="cuda", requires_grad=True)
    with q.Lattice(d, dims, tau, beta0, precision="fp32") as lat:
        state = rollout(lat, rho4, u, eps, tau_t, T)
        J = (wxy[:, None] * state[:, 0, :])[:, mask].sum()
        J.backward()
    grads = {"rho4": rho4.grad.cpu().numpy(), "u": u.grad.cpu().numpy(), "eps": eps.grad.cpu().numpy()}
    g_tau = float(tau_t.grad)
    w_np = wxy.cpu().numpy()

    def J64(r4, uu, ee, t):
        with q.Lattice(d, dims, t, beta0, precision="fp64") as l64:
            l64.init_equilibrium(r4, uu, ee)
            l64.step(T)
            st = l64.get_state()
        return float((w_np[:, None] * st[:, 0, :])[:, box].sum())

    rng = np.random.default_rng(77)
    h = 1e-5
    base = {k: fl[k] for k in ("rho4", "u", "eps")}
    for name in ("rho4", "u", "eps"):
        dv = rng.normal(size=base[name].shape)
        p = dict(base)
        m = dict(base)
        p[name] = base[name] + h * dv
        m[name] = base[name] - h * dv
        fd = (J64(p["rho4"], p["u"], p["eps"], tau) - J64(m["rho4"], m["u"], m["eps"], tau)) / (2 * h)
        ad = float(np.sum(grads[name] * dv))
        assert ad == pytest.approx(fd, rel=2e-4, abs=1e-7), name
    fdt = (J64(base["rho4"], base["u"], base["eps"], tau + h) -
           J64(base["rho4"], base["u"], base["eps"], tau - h)) / (2 * h)
    assert g_tau == pytest.approx(fdt, rel=2e-4, abs=1e-7)


def test_autograd_refuses_a_rollout_it_did_not_record(q):
    # two forward passes on one handle, then backward of the first: the
    # handle holds only the second rollout's checkpoints, so backward must
    # refuse instead of pairing the first graph's inputs with them; the
    # second graph's backward still works
    import torch
    from paper_1309_1656_gb300.autograd import rollout
    d, dims, T, tau = 2, (20, 16, 1), 6, 0.8
    fl = fields.random_fields(d, dims, seed=41)
    r1 = torch.from_numpy(fl["rho4"]).cuda().requires_grad_(True)
    r2 = torch.from_numpy(fl["rho4"] * 1.01).cuda().requires_grad_(True)
    u = torch.from_numpy(fl["u"]).cuda()
    with q.Lattice(d, dims, tau, 1.0, precision="fp64") as lat:
        s1 = rollout(lat, r1, u, None, tau, T)
        id1 = q.qlbm_rollout_id(lat.h)
        s2 = rollout(lat, r2, u, None, tau, T)
        assert q.qlbm_rollout_id(lat.h) == id1 + 1
        with pytest.raises(RuntimeError, match="rollout"):
            s1[:, 3].sum().backward()
        s2[:, 3].sum().backward()
        assert r2.grad is not None and torch.isfinite(r2.grad).all()
        lat.step(1)
        assert q.qlbm_rollout_id(lat.h) == -1
