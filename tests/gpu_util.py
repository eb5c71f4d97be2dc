"""Shared helpers of the GPU tests: build/load the library, run the oracle beside it."""
import numpy as np
import torch

from oracle import OracleSim


def sim_for(prob, **opt):
    from paper_2606_04206_gb300 import build, dlo
    build.build()
    return dlo.DloSim(prob, **opt)


def oracle_from_device_state(prob, sim):
    """An oracle loaded with the device's current (float32) state, every internal array included."""
    o = OracleSim(prob)
    o.set_full_state(sim.full_state_numpy())
    return o


def actions_dev(prob, f0=0, f1=None):
    f1 = prob.frames if f1 is None else f1
    return torch.as_tensor(np.ascontiguousarray(prob.actions[f0:f1], np.float32), device="cuda")


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def oracle_gradients(prob, frames, wx, wv, wth, dtype=None):
    """Autograd gradients of L = sum(wx * x_T) + sum(wv * (v_T, twist rate)) + sum(wth * theta_T)
    through the FP64 oracle rollout, with respect to the initial state, the actions and the
    per-rod material (K, E, G, yield curvature, damping).  dtype=torch.float32 runs the same
    definitions in float32, which measures how well float32 arithmetic can resolve a gradient."""
    import torch as T
    p = prob
    dt = T.float64 if dtype is None else dtype
    leaf = lambda a: T.tensor(np.asarray(a, np.float64), dtype=dt, requires_grad=True)
    leaves = dict(x0=leaf(p.x0), v0=leaf(p.v0), th0=leaf(p.theta0), om0=leaf(p.omega0), act=leaf(p.actions[:frames]))
    mats = {k: leaf(getattr(p, k)) for k in ("K", "E", "G", "yield_curv", "damping")}
    sim = OracleSim(p, params=mats, dtype=dt)
    sim.set_state(leaves["x0"], leaves["v0"], leaves["th0"], leaves["om0"])
    sim.step(leaves["act"], frames, diff=True)
    st = sim.get_state(as_numpy=False)
    om_w = np.zeros(int(p.edge_off[-1]))
    vo, eo = p.vert_off, p.edge_off
    for b in range(p.batch):
        ne = eo[b + 1] - eo[b]
        om_w[eo[b]:eo[b + 1]] = wv[vo[b]:vo[b] + ne, 3]
    w = lambda a: T.tensor(a, dtype=dt)
    L = ((st["x"] * w(wx[:, :3])).sum() + (st["v"] * w(wv[:, :3])).sum()
         + (st["omega"] * w(om_w)).sum() + (st["theta"] * w(wth)).sum())
    names = ["x0", "v0", "th0", "om0", "act"] + list(mats)
    inputs_ = [leaves[n] for n in names[:5]] + [mats[n] for n in names[5:]]
    g = T.autograd.grad(L, inputs_, allow_unused=True)
    out = {n: (gi.double().numpy() if gi is not None else np.zeros(tuple(x.shape))) for n, gi, x in zip(names, g, inputs_)}
    out["material"] = np.stack([out[k] for k in ("K", "E", "G", "yield_curv", "damping")], 1)
    return out, float(L.detach())


def device_gradients(sim, prob, frames, wx, wv, wth, substeps=0):
    """The C-ABI backward for the same loss; returns numpy arrays in the oracle's layout."""
    import torch as T
    dev = sim.device
    sim.reset()
    sim.begin_rollout(frames)
    sim.step(T.as_tensor(np.ascontiguousarray(prob.actions[:frames], np.float32), device=dev), frames, substeps)
    g = sim.backward(T.as_tensor(wx, dtype=T.float32, device=dev), T.as_tensor(wv, dtype=T.float32, device=dev),
                     T.as_tensor(wth, dtype=T.float32, device=dev))
    g = {k: v.double().cpu().numpy() for k, v in g.items()}
    vo, eo = prob.vert_off, prob.edge_off
    om = np.zeros(int(eo[-1]))
    for b in range(prob.batch):
        ne = eo[b + 1] - eo[b]
        om[eo[b]:eo[b + 1]] = g["v0"][vo[b]:vo[b] + ne, 3]
    return dict(x0=g["x0"][:, :3], v0=g["v0"][:, :3], om0=om, th0=g["theta0"], act=g["actions"],
                material=g["material"])


def grad_agreement(a, b):
    a, b = np.ravel(a), np.ravel(b)
    nb = np.linalg.norm(b)
    if nb == 0:
        return (0.0 if np.linalg.norm(a) == 0 else np.inf), 1.0
    rel = np.linalg.norm(a - b) / nb
    cos = float(a @ b / (np.linalg.norm(a) * nb + 1e-300))
    return rel, cos


def rod_state(st, prob, b):
    """One rod's slice of a full device state (as returned by DloSim.full_state_numpy), in the
    layout OracleSim.set_full_state expects for prob.subset([b])."""
    vo, eo = prob.vert_off, prob.edge_off
    v0, v1, e0, e1 = vo[b], vo[b + 1], eo[b], eo[b + 1]
    return dict(x=st["x"][v0:v1], v=st["v"][v0:v1], theta=st["theta"][e0:e1], omega=st["omega"][e0:e1],
                d1b=st["d1b"][e0:e1], tb=st["tb"][e0:e1], kbar=st["kbar"][v0:v1], mprev=st["mprev"][v0:v1],
                mbar=st["mbar"][v0:v1], gp=st["gp"][b:b + 1], gR=st["gR"][b:b + 1])
