"""torch.autograd interface of the checkpointed rollout and its adjoint.

A handle records one rollout at a time: backward() of a graph whose rollout
is no longer the handle's last one (checked through qlbm_rollout_id) raises
RuntimeError instead of pairing its saved inputs with another pass's
checkpoints.

``rollout(lat, rho4, u, eps, tau, nsteps)`` initialises the handle's state
from the fields (Eq. WeqAlgo), advances it nsteps with square-root
checkpointing (``qlbm_rollout``) and returns the final state as a CUDA
float64 tensor [b][4][N].  Its backward pass runs ``qlbm_rollout_adjoint``
(segment recomputation + reverse steps, in the library's kernels) and
``qlbm_init_equilibrium_adjoint``, giving gradients with respect to rho4
(density and spin field), u, eps and tau.  This module only marshals
tensors between torch's autograd and the C ABI.
"""
import torch

from . import qlbm


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho4, u, eps, tau, lat, nsteps, interval):
        if abs(float(tau) - lat.tau) > 1e-15 * max(1.0, lat.tau):
            raise ValueError("tau must equal the handle's tau (%g)" % lat.tau)
        qlbm.qlbm_init_equilibrium(lat.h, rho4, u, eps)
        qlbm.qlbm_rollout(lat.h, nsteps, interval)
        state = torch.empty((lat.b, 4, lat.N), dtype=torch.float64, device=rho4.device)
        qlbm.qlbm_get_state(lat.h, state)
        ctx.lat = lat
        ctx.rollout_id = qlbm.qlbm_rollout_id(lat.h)
        ctx.has_eps = eps is not None
        ctx.save_for_backward(rho4, u, eps if eps is not None else rho4.new_empty(0))
        return state

    @staticmethod
    def backward(ctx, gstate):
        lat = ctx.lat
        # the handle keeps only its last rollout: refuse to sweep over
        # another forward pass's checkpoints
        if qlbm.qlbm_rollout_id(lat.h) != ctx.rollout_id:
            raise RuntimeError("the handle's recorded rollout is no longer the one this graph's forward pass "
                               "made (another rollout, step, init or set_state came in between); run the "
                               "forward pass again before backward")
        rho4, u, eps = ctx.saved_tensors
        eps = eps if ctx.has_eps else None
        lam0 = torch.empty_like(gstate)
        dtau = qlbm.qlbm_rollout_adjoint(lat.h, gstate.contiguous(), lam0)
        g_rho4 = torch.empty_like(rho4)
        g_u = torch.empty_like(u)
        g_eps = torch.empty_like(eps) if eps is not None else None
        qlbm.qlbm_init_equilibrium_adjoint(lat.h, rho4, u, eps, lam0, g_rho4, g_u, g_eps)
        g_tau = torch.tensor(dtau, dtype=torch.float64, device=rho4.device)
        return g_rho4, g_u, g_eps, g_tau, None, None, None


def rollout(lat, rho4, u, eps, tau, nsteps, interval=0):
    """Differentiable rollout on the handle ``lat`` (a qlbm.Lattice)."""
    if not torch.is_tensor(tau):
        tau = torch.tensor(float(tau), dtype=torch.float64, device=rho4.device)
    return _Rollout.apply(rho4, u, eps, tau, lat, int(nsteps), int(interval))
