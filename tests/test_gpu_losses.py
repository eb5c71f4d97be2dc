"""The device task losses (dlo_loss) against their FP64 definitions (oracle/losses.py,
pinned in tests/test_oracle_losses.py): per-rod values and the gradient of sum_b g_b Q_b with
respect to the vertex positions, on open rods (trajopt) and closed knotted bands
(selfcontact) after a few frames of motion."""
import numpy as np
import pytest
import torch

from oracle import losses as L
from paper_2606_04206_gb300 import dlo, inputs
from gpu_util import sim_for, actions_dev, grad_agreement

pytestmark = pytest.mark.gpu


def setup(kind, n_rods, n):
    p = inputs.small_case(kind, n_rods=n_rods, n=n, frames=8)
    sim = sim_for(p)
    sim.reset()
    sim.step(actions_dev(p), 8)
    x, _, _ = sim.get_state()
    g = torch.as_tensor(np.random.default_rng(3).uniform(0.5, 2.0, p.batch), dtype=torch.float32, device=x.device)
    return p, sim, x, g


def per_rod(p, x, fn):
    """Oracle value and gradient of fn for every rod (float64 autograd)."""
    xs = x[:, :3].double().cpu()
    q, gx = [], np.zeros((xs.shape[0], 3))
    for b in range(p.batch):
        v0, v1 = p.vert_off[b], p.vert_off[b + 1]
        xb = xs[v0:v1].clone().requires_grad_(True)
        val = fn(b, xb)
        gb, = torch.autograd.grad(val, [xb])
        q.append(float(val.detach()))
        gx[v0:v1] = gb.numpy()
    return np.array(q), gx


def check(q_dev, g_dev, q_ref, g_ref, g, p, q_tol):
    q_dev = q_dev.double().cpu().numpy()
    assert np.abs(q_dev - q_ref).max() <= q_tol * (1.0 + np.abs(q_ref).max()), (q_dev, q_ref)
    gw = g.double().cpu().numpy()
    ref = g_ref * np.repeat(gw, np.diff(p.vert_off))[:, None]
    assert not g_dev[:, 3].any()
    if np.abs(ref).max() < 1e-9:          # an analytically zero gradient (a loop's winding number)
        assert not g_dev.any()
        return
    rel, cos = grad_agreement(g_dev[:, :3].double().cpu().numpy(), ref)
    assert rel <= 1e-3 and cos >= 0.999, (rel, cos)


@pytest.mark.parametrize("kind,n", [("trajopt", 64), ("selfcontact", 60)])
def test_target_and_chamfer(kind, n):
    p, sim, x, g = setup(kind, 4, n)
    rng = np.random.default_rng(4)
    tg = torch.zeros_like(x)
    tg[:, :3] = x[:, :3] + torch.as_tensor(rng.normal(scale=0.01, size=(x.shape[0], 3)), dtype=torch.float32,
                                            device=x.device)
    q, gx = sim.loss(dlo.LOSS_TARGET, x, tg, g)
    tgd = tg[:, :3].double().cpu()
    q_ref, g_ref = per_rod(p, x, lambda b, xb: L.target_mse(xb, tgd[p.vert_off[b]:p.vert_off[b + 1]]))
    check(q, gx, q_ref, g_ref, g, p, 1e-5)
    m = 37
    pts = torch.zeros(p.batch, m, 4, device=x.device)
    for b in range(p.batch):
        xb = x[p.vert_off[b]:p.vert_off[b + 1], :3]
        c = xb.mean(0)
        pts[b, :, :3] = c + torch.as_tensor(rng.normal(scale=0.2, size=(m, 3)), dtype=torch.float32, device=x.device)
    q, gx = sim.loss(dlo.LOSS_CHAMFER, x, pts, g)
    ptd = pts[:, :, :3].double().cpu()
    q_ref, g_ref = per_rod(p, x, lambda b, xb: L.chamfer(xb, ptd[b]))
    check(q, gx, q_ref, g_ref, g, p, 1e-5)


@pytest.mark.parametrize("kind,n", [("trajopt", 64), ("selfcontact", 60)])
def test_winding_number(kind, n):
    p, sim, x, g = setup(kind, 4, n)
    post = torch.zeros(p.batch, 4, device=x.device)
    for b in range(p.batch):
        post[b, :2] = x[p.vert_off[b]:p.vert_off[b + 1], :2].mean(0)
    q, gx = sim.loss(dlo.LOSS_WINDING, x, post, g)
    pd = post.double().cpu()
    q_ref, g_ref = per_rod(p, x, lambda b, xb: L.winding(xb, pd[b, :2], closed=bool(p.closed[b])))
    check(q, gx, q_ref, g_ref, g, p, 1e-5)
    if kind == "selfcontact":   # a closed band winds an integer number of times
        assert np.allclose(q.double().cpu().numpy(), np.round(q_ref), atol=1e-4)


@pytest.mark.parametrize("kind,n", [("trajopt", 48), ("selfcontact", 48)])
def test_crossing_sum(kind, n):
    p, sim, x, g = setup(kind, 3, n)
    q, gx = sim.loss(dlo.LOSS_CROSSING, x, None, g)
    q_ref, g_ref = per_rod(p, x, lambda b, xb: L.crossing(xb, closed=bool(p.closed[b])))
    if kind == "selfcontact":
        assert np.abs(q_ref).max() > 0.5     # knotted bands have large writhe
    check(q, gx, q_ref, g_ref, g, p, 2e-4)
