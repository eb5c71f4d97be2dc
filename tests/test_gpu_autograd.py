"""The rollout as a torch autograd operation (DloRollout): its gradients are exactly those of
dlo_backward on the same recorded rollout, and a few gradient steps on the gripper actions
lower a trajectory-optimisation loss (mean squared distance of the final vertices to a
target curve)."""
import numpy as np
import pytest
import torch

from paper_2606_04206_gb300 import dlo, inputs
from gpu_util import sim_for, actions_dev

pytestmark = pytest.mark.gpu


def test_autograd_rollout_matches_dlo_backward():
    p = inputs.small_case("trajopt", n_rods=4, n=32, frames=6)
    sim = sim_for(p)
    x0, v0, th0 = (t.clone().requires_grad_(True) for t in sim.tensors_from_problem())
    acts = actions_dev(p).requires_grad_(True)
    mat = sim.material_tensor().requires_grad_(True)
    target = torch.zeros_like(x0)
    target[:, :3] = torch.as_tensor(p.target, dtype=torch.float32, device=x0.device)
    x, v, th = dlo.rollout(sim, x0, v0, th0, acts, mat)
    loss = ((x - target)[:, :3] ** 2).sum(1).mean() + 1e-3 * (v[:, :3] ** 2).sum() + 1e-3 * (th ** 2).sum()
    loss.backward()
    # the same cotangents through the C ABI directly
    gx = torch.zeros_like(x)
    gx[:, :3] = 2.0 * (x.detach() - target)[:, :3] / x.shape[0]
    gv = torch.zeros_like(v)
    gv[:, :3] = 2e-3 * v.detach()[:, :3]
    gth = 2e-3 * th.detach()
    sim.set_state(x0.detach(), v0.detach(), th0.detach())
    sim.begin_rollout(p.frames)
    sim.step(acts.detach(), p.frames)
    ref = sim.backward(gx, gv, gth)
    for name, t in (("x0", x0), ("v0", v0), ("theta0", th0), ("actions", acts), ("material", mat)):
        assert t.grad is not None, name
        torch.testing.assert_close(t.grad, ref[name], rtol=1e-5, atol=1e-12, msg=name)


def test_steps_along_the_negative_action_gradient_lower_the_loss():
    p = inputs.small_case("trajopt", n_rods=4, n=32, frames=20)
    sim = sim_for(p)
    x0, v0, th0 = sim.tensors_from_problem()
    target = torch.zeros_like(x0)
    target[:, :3] = torch.as_tensor(p.target, dtype=torch.float32, device=x0.device)
    acts = actions_dev(p).requires_grad_(True)
    losses = []
    for _ in range(3):
        acts.grad = None
        x, _, _ = dlo.rollout(sim, x0, v0, th0, acts)
        loss = ((x - target)[:, :3] ** 2).sum(1).mean()
        loss.backward()
        losses.append(float(loss.detach()))
        with torch.no_grad():   # 20 um total gripper displacement along the descent direction
            acts -= 2e-5 * acts.grad / acts.grad.norm()
    assert np.isfinite(losses).all() and losses[2] < losses[1] < losses[0], losses
