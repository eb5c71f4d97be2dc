"""The device silhouette loss (dlo_loss_silhouette) against its FP64 definition
(oracle/silhouette.py, pinned in tests/test_oracle_silhouette.py): soft renders, per-rod loss
and position gradient with two cameras, and the system-identification gradient with respect
to the material through a recorded rollout."""
import math

import numpy as np
import pytest
import torch

from oracle import OracleSim
from oracle.silhouette import camera, render, silhouette_loss
from paper_2606_04206_gb300 import inputs
from gpu_util import sim_for, actions_dev, grad_agreement

pytestmark = pytest.mark.gpu

H, W, TAU = 48, 64, 0.6


def cameras():
    down = camera(60.0, 60.0, W / 2, H / 2, np.diag([1.0, -1.0, -1.0]), [0.0, 0.0, 1.3])
    a = math.radians(50.0)          # tilted about x: looks down at 50 degrees from the side
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, -math.sin(a), -math.cos(a)], [0.0, math.cos(a), -math.sin(a)]])
    eye = np.array([0.0, -1.1 * math.cos(a), 1.1 * math.sin(a)]) * 1.2
    side = camera(70.0, 70.0, W / 2, H / 2, Rx, -Rx @ eye)
    return np.stack([down, side])


def target_masks(p, shift, cams):
    """Binary masks of the rods moved by `shift` (the oracle's renders, thresholded at 0.5)."""
    out = np.zeros((p.batch, len(cams), H, W), np.uint8)
    for b in range(p.batch):
        xb = torch.tensor(p.x0[p.vert_off[b]:p.vert_off[b + 1]] + shift, dtype=torch.float64)
        for c in range(len(cams)):
            out[b, c] = (render(xb, cams[c], H, W, TAU, float(p.radius[b]), bool(p.closed[b])) > 0.5).numpy()
    return out


def test_silhouette_renders_values_and_gradients():
    p = inputs.small_case("trajopt", n_rods=3, n=24, frames=6)
    sim = sim_for(p)
    sim.reset()
    sim.step(actions_dev(p), 6)
    x, _, _ = sim.get_state()
    cams = cameras()
    masks = target_masks(p, np.array([0.02, -0.01, 0.0]), cams)
    g = torch.tensor([1.0, 0.5, 2.0], device="cuda")
    q, gx, img = sim.silhouette(x, torch.tensor(cams, dtype=torch.float32, device="cuda"),
                                torch.tensor(masks, device="cuda"), TAU, g, render=True)
    xs = x[:, :3].double().cpu()
    for b in range(p.batch):
        v0, v1 = p.vert_off[b], p.vert_off[b + 1]
        xb = xs[v0:v1].clone().requires_grad_(True)
        r = float(p.radius[b])
        L = silhouette_loss(xb, cams, masks[b], TAU, r)
        gb, = torch.autograd.grad(L, [xb])
        L = float(L.detach())
        assert abs(float(q[b]) - L) <= 1e-4 * L + 1e-7, (b, float(q[b]), L)
        rel, cos = grad_agreement(gx[v0:v1, :3].double().cpu().numpy(), float(g[b]) * gb.numpy())
        assert rel <= 1e-3 and cos >= 0.999, (b, rel, cos)
        for c in range(len(cams)):
            o = render(xb.detach(), cams[c], H, W, TAU, r)
            assert np.abs(img[b, c].double().cpu().numpy() - o.numpy()).max() <= 2e-5
            assert o.max() > 0.5                                     # the rod is in view
    assert not gx[:, 3].any()


def test_system_identification_gradient_through_the_rollout():
    """d/d(material, actions) of the silhouette loss of the final state of a recorded
    rollout: dlo_loss_silhouette's dL/dx_T fed to dlo_backward, against FP64 autograd
    through the oracle rollout and the oracle's silhouette."""
    frames = 3
    p = inputs.small_case("trajopt", n_rods=3, n=24, frames=frames)
    cams = cameras()
    masks = target_masks(p, np.array([0.0, 0.015, 0.0]), cams)
    sim = sim_for(p)
    sim.reset()
    sim.begin_rollout(frames)
    sim.step(actions_dev(p), frames)
    x, _, _ = sim.get_state()
    _, gx, _ = sim.silhouette(x, torch.tensor(cams, dtype=torch.float32, device="cuda"),
                              torch.tensor(masks, device="cuda"), TAU)
    got = sim.backward(dL_dx=gx, want=("actions", "material"))

    mats = {k: torch.tensor(np.asarray(getattr(p, k), np.float64), requires_grad=True)
            for k in ("K", "E", "G", "yield_curv", "damping")}
    act = torch.tensor(np.asarray(p.actions[:frames], np.float64), requires_grad=True)
    o = OracleSim(p, params=mats)
    o.set_state(torch.tensor(p.x0), torch.tensor(p.v0), torch.tensor(p.theta0), torch.tensor(p.omega0))
    o.step(act, frames, diff=True)
    xT = o.get_state(as_numpy=False)["x"]
    loss = 0.0
    for b in range(p.batch):
        xb = xT[p.vert_off[b]:p.vert_off[b + 1]]
        loss = loss + silhouette_loss(xb, cams, masks[b], TAU, float(p.radius[b]))
    names = ("K", "E", "G", "yield_curv", "damping")
    grads = torch.autograd.grad(loss, [act] + [mats[k] for k in names], allow_unused=True)
    ref_act = grads[0].numpy()
    pv = np.stack([np.asarray(getattr(p, k), np.float64) for k in names], 1)
    ref_mat = np.stack([(gk.numpy() if gk is not None else np.zeros(p.batch)) for gk in grads[1:]], 1) * pv
    dev_mat = got["material"].double().cpu().numpy() * pv
    for name, a, b in (("actions", got["actions"].double().cpu().numpy(), ref_act), ("material", dev_mat, ref_mat)):
        rel, cos = grad_agreement(a, b)
        assert rel <= 1e-3 and cos >= 0.999, (name, rel, cos)
