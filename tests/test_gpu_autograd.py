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


def changed_material(p):
    """The workload's material with every rod's moduli, yield curvature and damping changed;
    the first rod made stiff enough to need more substeps than it had."""
    m = np.stack([np.asarray(getattr(p, k), np.float64) for k in dlo.MATERIAL_KEYS], 1)
    m[:, 0] *= 2.0
    m[:, 1] *= 3.0
    m[:, 2] *= 0.5
    m[:, 3] = np.where(p.plastic, 0.7 * m[:, 3], m[:, 3])
    m[:, 4] = 2.5
    m[0, :3] = [1e8, 1e8, 4e7]
    return inputs.f32(m)


def with_material(p, m):
    import copy
    q = copy.deepcopy(p)
    for k, col in zip(dlo.MATERIAL_KEYS, m.T):
        setattr(q, k, inputs.f32(col))
    return q


def test_set_material_equals_a_context_created_with_it():
    """dlo_set_material: the same rollout, bit for bit, as a context created with the new
    material, including each rod's recomputed substep count; a change of a create-time
    quantity (the density) is refused and names the rod."""
    p = inputs.small_case("trajopt", n_rods=3, n=24, frames=5)
    m = changed_material(p)
    sim, fresh = sim_for(p), sim_for(with_material(p, m))
    n0 = sim.query(dlo.Q_SUBSTEPS)
    sim.set_material(m)
    assert np.array_equal(sim.query(dlo.Q_SUBSTEPS), fresh.query(dlo.Q_SUBSTEPS))
    assert fresh.query(dlo.Q_SUBSTEPS)[0] > n0[0]
    out = []
    for s in (sim, fresh):
        s.reset()
        s.step(actions_dev(p), 5)
        out.append(s.get_state()[0].cpu().numpy())
    assert np.array_equal(out[0], out[1])
    bad = (dlo.Material * 3)()
    lib = sim.lib
    mats = sim._materials(m)
    for b in range(3):
        bad[b] = mats[b]
    bad[2].density = 1200.0
    st = lib.dlo_set_material(sim.ctx, bad)
    assert st == 1 and "rod 2" in lib.dlo_last_error(sim.ctx).decode()


def test_rollout_applies_its_material_argument():
    """DloRollout.forward sets the material it is given: the rollout and its gradients equal
    those of a context created with that material."""
    p = inputs.small_case("trajopt", n_rods=3, n=24, frames=5)
    m = changed_material(p)
    res = []
    for prob, mat in ((p, m), (with_material(p, m), None)):
        sim = sim_for(prob)
        x0, v0, th0 = sim.tensors_from_problem()
        acts = actions_dev(p).requires_grad_(True)
        mt = (sim.material_tensor() if mat is None else torch.as_tensor(mat, dtype=torch.float32, device="cuda"))
        mt.requires_grad_(True)
        x, _, _ = dlo.rollout(sim, x0, v0, th0, acts, mt)
        (x[:, :3] ** 2).sum().backward()
        res.append((x.detach().cpu().numpy(), acts.grad.cpu().numpy(), mt.grad.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0])          # the forward is bitwise reproducible
    for a, b in zip(res[0][1:], res[1][1:]):             # the backward adds some cotangents with
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())   # float atomics


def test_backward_of_a_superseded_rollout_raises():
    """Two rollouts on one context before the first loss's backward: the context's record is
    the second rollout's, so the first backward must refuse rather than return its gradients."""
    p = inputs.small_case("trajopt", n_rods=2, n=16, frames=3)
    sim = sim_for(p)
    x0, v0, th0 = sim.tensors_from_problem()
    acts = actions_dev(p).requires_grad_(True)
    x1, _, _ = dlo.rollout(sim, x0, v0, th0, acts)
    x2, _, _ = dlo.rollout(sim, x0, v0, th0, acts)
    with pytest.raises(RuntimeError, match="another rollout"):
        x1.sum().backward()
    x2.sum().backward()
    assert acts.grad is not None and bool(torch.isfinite(acts.grad).all())
