"""Gradients over the differentiation configuration's horizon: 500 frames, checkpoints every
50 frames, so the device adjoint replays each 50-frame segment from its checkpoint (Sec. 3.3).

Two rods of the differentiation workload (64 vertices, 1 m, ground contact, two grippers): an
elastic rope and a plastic wire.  Their device gradients are compared with
  * the FP64 oracle's reverse-mode gradients of the same 500-frame rollout, per group, at
    relative L2 error <= 1e-3 and cosine >= 0.999 (actions, initial state, the scale-free
    material sensitivities p dL/dp);
  * FP64 central differences (h = 1e-6 of the coordinate's scale) of the configuration's loss,
    the mean squared distance of the final vertices to the seeded target curve, on at least
    16 of 40 sampled coordinates (actions, initial positions and velocities, E, yield
    curvature).  A coordinate whose +h and -h oracle runs take different branches anywhere (a
    rigid contact switching, a hinge yielding or not, a strain-limit projection switching) is
    not differentiable across the interval: it is reported and set aside.  Over 500 frames
    that is most coordinates of the plastic wire, whose bent hinges sit on the yield surface.
"""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest
import torch

from paper_2606_04206_gb300 import inputs
from paper_2606_04206_gb300.dlo import Q_CONFIG
from gpu_util import sim_for, oracle_gradients, device_gradients, grad_agreement
import oracle_fd

pytestmark = pytest.mark.gpu

FRAMES, K = 500, 50
GROUPS = ("x0", "v0", "om0", "th0", "act", "material")


def workload():
    p = inputs.diff(n_rods=4, frames=FRAMES, seed=2000, n=64)
    return p.subset([0, 2])          # rod 0 elastic rope, rod 2 plastic wire


def log_sens(prob, g):
    pv = np.stack([np.asarray(getattr(prob, k), np.float64) for k in ("K", "E", "G", "yield_curv", "damping")], 1)
    return g * pv


def test_500_frames_with_segment_replay_against_oracle_and_central_differences():
    p = workload()
    assert p.plastic.tolist() == [False, True]
    rng = np.random.default_rng(11)
    # FD coordinates: drawn now, evaluated by worker processes (spawned: independent of the
    # CUDA context of this process) while the device and the oracle's autograd run here
    draws = []
    for _ in range(40):
        kind = rng.choice(["act"] * 8 + ["x0"] * 3 + ["v0", "E", "E", "yield_curv", "yield_curv"])
        b = int(rng.integers(2))
        if kind == "act":
            draws.append(("act", (int(rng.integers(FRAMES)), b, int(rng.integers(2)), int(rng.integers(6))), b))
        elif kind in ("x0", "v0"):
            v = int(p.vert_off[b] + rng.integers(64))
            draws.append((kind, (v, int(rng.integers(3))), b))
        else:
            r = b if kind == "E" else 1          # yield curvature: the plastic wire only
            draws.append((kind, r, r))
    n_total = int(p.vert_off[-1])

    def job(name, idx, b):
        sub = p.subset([b])
        base = {"act": p.actions, "x0": p.x0, "v0": p.v0, "E": p.E, "yield_curv": p.yield_curv}[name]
        val = float(np.asarray(base)[idx])
        scale = max(abs(val), 1e-3 if name in ("act", "x0", "v0") else 1.0)
        h = 1e-6 * scale
        if name == "act":
            sidx = (idx[0], 0, idx[2], idx[3])
        elif name in ("x0", "v0"):
            sidx = (idx[0] - int(p.vert_off[b]), idx[1])
        else:
            sidx = 0
        return (sub, FRAMES, n_total, name, sidx, h)

    ctx = mp.get_context("spawn")
    pool = ProcessPoolExecutor(max_workers=max(2, min(16, os.cpu_count() or 2)), mp_context=ctx)
    futs = [pool.submit(oracle_fd.central_difference, job(*d)) for d in draws]
    try:
        check_device(p, futs, draws)
    finally:
        pool.shutdown(wait=False, cancel_futures=True)


def check_device(p, futs, draws):
    # device: one recorded 500-frame rollout, checkpoints every 50 frames
    sim = sim_for(p, checkpoint_every=K)
    rng_w = np.random.default_rng(5)
    V, E = int(p.vert_off[-1]), int(p.edge_off[-1])
    wx = np.zeros((V, 4))
    wx[:, :3] = rng_w.normal(size=(V, 3))
    wv = np.zeros((V, 4))
    wv[:, :3] = rng_w.normal(size=(V, 3)) * 1e-2
    wth = rng_w.normal(size=E) * 1e-2
    got = device_gradients(sim, p, FRAMES, wx, wv, wth)
    assert int(sim.query(Q_CONFIG)[1]) == K
    # the configuration's loss on the same recorded rollout: dL/dx_T = 2 (x_T - target) / N
    xT = sim.get_state()[0]
    tgt = torch.zeros_like(xT)
    tgt[:, :3] = torch.as_tensor(p.target, dtype=torch.float32, device=xT.device)
    gl = sim.backward(dL_dx=(2.0 / V) * (xT - tgt), want=("actions", "material", "x0", "v0"))
    gl = {k: v.double().cpu().numpy() for k, v in gl.items()}

    # oracle reverse mode over the same 500 frames
    ref, _ = oracle_gradients(p, FRAMES, wx, wv, wth)
    got["material"], ref["material"] = log_sens(p, got["material"]), log_sens(p, ref["material"])
    report = {k: grad_agreement(got[k], ref[k]) for k in GROUPS}
    print("500 frames, K = 50: gradient agreement (rel L2, cosine):",
          {k: (f"{r:.2e}", f"{c:.6f}") for k, (r, c) in report.items()})
    bad = {k: v for k, v in report.items() if not (v[0] <= 1e-3 and v[1] >= 0.999)}
    assert not bad, report

    # central differences; coordinates whose runs cross a branch are set aside
    scale_act = np.abs(gl["actions"]).max()
    ok, flagged = [], []
    for f, (name, idx, b) in zip(futs, draws):
        fd, same = f.result()
        if name == "act":
            g = gl["actions"][idx]
        elif name in ("x0", "v0"):
            g = gl[name][idx]
        else:
            g = gl["material"][idx, {"E": 1, "yield_curv": 3}[name]]
        (ok if same else flagged).append((name, idx, g, fd))
    print(f"central differences: {len(ok)} coordinates compared, {len(flagged)} flagged (branch flip between "
          f"+h and -h): {[(n, i) for n, i, _, _ in flagged]}")
    for name, idx, g, fd in ok:
        print("central difference", name, idx, "device %.6e fd %.6e" % (g, fd))
    assert len(ok) >= 16
    for name, idx, g, fd in ok:
        assert g == pytest.approx(fd, rel=1e-3, abs=1e-5 * scale_act), (name, idx, g, fd)
