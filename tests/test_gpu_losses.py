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


def rest_edges(p):
    return np.array([np.linalg.norm(np.diff(p.x_rest[a:b], axis=0), axis=1).mean()
                     for a, b in zip(p.vert_off[:-1], p.vert_off[1:])])


@pytest.mark.parametrize("kind,n", [("trajopt", 64), ("selfcontact", 60), ("cmaes", 64)])
def test_mindist_and_repulsion(kind, n):
    p, sim, x, g = setup(kind, 4, n)
    obj = torch.zeros(p.batch, 4, device=x.device)
    rng = np.random.default_rng(5)
    for b in range(p.batch):
        obj[b, :3] = x[p.vert_off[b]:p.vert_off[b + 1], :3].mean(0) + torch.as_tensor(
            rng.normal(scale=0.05, size=3), dtype=torch.float32, device=x.device)
    q, gx = sim.loss(dlo.LOSS_MINDIST, x, obj, g)
    od = obj.double().cpu()
    q_ref, g_ref = per_rod(p, x, lambda b, xb: L.mindist(xb, od[b]))
    check(q, gx, q_ref, g_ref, g, p, 1e-6)
    # delta three rest edges (wider than the task's two, so that every shape has pairs inside)
    prm = torch.zeros(p.batch, 4, device=x.device)
    prm[:, 0] = torch.as_tensor(3.0 * rest_edges(p), dtype=torch.float32, device=x.device)
    prm[:, 1] = 2.0
    q, gx = sim.loss(dlo.LOSS_REPULSION, x, prm, g)
    pd = prm.double().cpu()
    q_ref, g_ref = per_rod(p, x, lambda b, xb: L.repulsion(xb, float(pd[b, 0]), 2, closed=bool(p.closed[b])))
    assert (q_ref > 0).any()
    check(q, gx, q_ref, g_ref, g, p, 1e-4)


def test_task_loss_gradient_through_the_rollout():
    """dlo_loss's dL/dx_T fed to dlo_backward: the gradient of a task loss (Chamfer distance
    to a point set plus a tenth of the crossing sum) with respect to the actions and the
    initial positions, against FP64 autograd of the same loss through the oracle rollout."""
    from oracle import OracleSim
    frames = 3
    p = inputs.small_case("trajopt", n_rods=3, n=24, frames=frames)
    sim = sim_for(p)
    rng = np.random.default_rng(6)
    m = 16
    pts = np.zeros((p.batch, m, 4), np.float32)
    for b in range(p.batch):
        pts[b, :, :3] = p.x0[p.vert_off[b]:p.vert_off[b + 1]].mean(0) + rng.normal(scale=0.2, size=(m, 3))
    dev_pts = torch.as_tensor(pts, device="cuda")
    sim.reset()
    sim.begin_rollout(frames)
    sim.step(actions_dev(p), frames)
    x, _, _ = sim.get_state()
    _, g1 = sim.loss(dlo.LOSS_CHAMFER, x, dev_pts)
    gw = torch.full((p.batch,), 0.1, device="cuda")
    _, g2 = sim.loss(dlo.LOSS_CROSSING, x, None, gw)
    got = sim.backward(dL_dx=g1 + g2, want=("actions", "x0"))

    act = torch.tensor(np.asarray(p.actions[:frames], np.float64), requires_grad=True)
    x0 = torch.tensor(np.asarray(p.x0, np.float64), requires_grad=True)
    o = OracleSim(p)
    o.set_state(x0, torch.tensor(p.v0), torch.tensor(p.theta0), torch.tensor(p.omega0))
    o.step(act, frames, diff=True)
    xT = o.get_state(as_numpy=False)["x"]
    loss = 0.0
    for b in range(p.batch):
        xb = xT[p.vert_off[b]:p.vert_off[b + 1]]
        loss = loss + L.chamfer(xb, torch.tensor(pts[b, :, :3], dtype=torch.float64)) + 0.1 * L.crossing(xb)
    ga, gx0 = torch.autograd.grad(loss, [act, x0])
    for name, dev_g, ref in (("actions", got["actions"], ga), ("x0", got["x0"][:, :3], gx0)):
        rel, cos = grad_agreement(dev_g.double().cpu().numpy(), ref.numpy())
        assert rel <= 1e-3 and cos >= 0.999, (name, rel, cos)


def test_population_scores_after_forward_rollouts():
    """A small CMA-ES generation: candidates stepped forward (self-contact on) and scored by
    crossing sum and repulsion, against the oracle's rollout and the FP64 definitions."""
    from oracle import OracleSim
    frames = 3
    p = inputs.small_case("cmaes", n_rods=3, n=48, frames=frames)
    sim = sim_for(p)
    sim.reset()
    sim.step(actions_dev(p), frames)
    x, _, _ = sim.get_state()
    prm = torch.zeros(p.batch, 4, device="cuda")
    prm[:, 0] = torch.as_tensor(2.0 * rest_edges(p), dtype=torch.float32, device="cuda")
    prm[:, 1] = 2.0
    qc, _ = sim.loss(dlo.LOSS_CROSSING, x, None, grad=False)
    qr, _ = sim.loss(dlo.LOSS_REPULSION, x, prm, grad=False)
    o = OracleSim(p)
    o.set_state(p.x0, p.v0, p.theta0, p.omega0)
    o.step(p.actions, frames)
    xo = torch.as_tensor(o.get_state()["x"])
    for b in range(p.batch):
        xb = xo[p.vert_off[b]:p.vert_off[b + 1]]
        c_ref = float(L.crossing(xb))
        r_ref = float(L.repulsion(xb, float(prm[b, 0]), 2))
        assert abs(c_ref) > 1.0                               # the rope is knotted
        assert abs(float(qc[b]) - c_ref) <= 1e-4, (b, float(qc[b]), c_ref)
        assert abs(float(qr[b]) - r_ref) <= 1e-3 * max(r_ref, 1e-9) + 1e-10, (b, float(qr[b]), r_ref)
