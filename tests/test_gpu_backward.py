"""The device adjoint (dlo_backward) against the FP64 oracle's reverse-mode gradients and
against FP64 central differences.  Tolerance: relative L2 error <= 1e-3 and cosine >= 0.999
for the gradients with respect to the actions, the initial positions, velocities, twist
rates and twist angles, and the material parameters; the latter are compared as the
scale-free sensitivities p * dL/dp (K, E, G, yield curvature, damping), since their raw
gradients span many orders of magnitude."""
import numpy as np
import pytest
import torch

from oracle import OracleSim
from paper_2606_04206_gb300 import inputs
from gpu_util import sim_for, oracle_gradients, device_gradients, grad_agreement

pytestmark = pytest.mark.gpu

GROUPS = ("x0", "v0", "om0", "th0", "act", "material")


def weights(prob, seed=0):
    rng = np.random.default_rng(seed)
    V, E = int(prob.vert_off[-1]), int(prob.edge_off[-1])
    wx = np.zeros((V, 4))
    wx[:, :3] = rng.normal(size=(V, 3))
    wv = np.zeros((V, 4))
    wv[:, :3] = rng.normal(size=(V, 3)) * 1e-2
    wv[:, 3] = rng.normal(size=V) * 1e-3
    wth = rng.normal(size=E) * 1e-2
    return wx, wv, wth


TOL = {}


def log_sens(prob, g):
    pv = np.stack([np.asarray(getattr(prob, k), np.float64) for k in ("K", "E", "G", "yield_curv", "damping")], 1)
    return g * pv


def check(prob, frames, seed=0, tol=None, **opt):
    wx, wv, wth = weights(prob, seed)
    ref, _ = oracle_gradients(prob, frames, wx, wv, wth)
    tol = TOL if tol is None else tol
    sim = sim_for(prob, **opt)
    got = device_gradients(sim, prob, frames, wx, wv, wth)
    got["material"], ref["material"] = log_sens(prob, got["material"]), log_sens(prob, ref["material"])
    report = {}
    for k in GROUPS:
        rel, cos = grad_agreement(got[k], ref[k])
        report[k] = (rel, cos)
    print("gradient agreement (rel L2, cosine):", {k: (f"{r:.2e}", f"{c:.6f}") for k, (r, c) in report.items()})
    bad = {k: v for k, v in report.items() if not (v[0] <= tol.get(k, 1e-3) and v[1] >= 0.999)}
    assert not bad, report
    return report


@pytest.mark.parametrize("kind", ["trajopt", "diff", "batching"])
def test_backward_matches_oracle_autograd(kind):
    p = inputs.small_case(kind, n_rods=3, n=12, frames=3)
    check(p, 3)


def test_backward_with_creep_below_full_return():
    """Bending creep with r_c = 0.3 (App. A.1: the rest curvature moves toward the current one
    by r_c of the excess over the yield surface): plastic wires bent past yield.

    These rods are stiff (E up to 3e7 Pa, K = E), so their strains sit near float32's
    resolution and the scale-free material sensitivities are poorly conditioned in float32:
    the same definitions evaluated in float32 (the oracle at dtype float32) miss the FP64
    values by ~1e-2.  The material bar is therefore max(1e-3, 2 x that float32 error),
    measured here on the same inputs; every other gradient keeps the 1e-3 bar."""
    p = inputs.small_case("batching", n_rods=3, n=24, frames=4)
    p.creep_rate[:] = 0.3
    p.yield_curv[:] = inputs.f32(np.full(3, 1.0))
    wx, wv, wth = weights(p, 0)
    ref, _ = oracle_gradients(p, 4, wx, wv, wth)
    f32, _ = oracle_gradients(p, 4, wx, wv, wth, dtype=torch.float32)
    floor, _ = grad_agreement(log_sens(p, f32["material"]), log_sens(p, ref["material"]))
    print("float32 floor of the material sensitivities:", floor)
    check(p, 4, tol={"material": max(1e-3, 2.0 * floor)})


def test_backward_with_self_contact_and_loops():
    p = inputs.small_case("selfcontact", n_rods=2, n=30, frames=2)
    check(p, 2)


def test_backward_coil_in_self_contact():
    import test_gpu_forward as T
    p = T.coils(n_rods=2, frames=2, n=32)
    check(p, 2)


def test_backward_matches_central_differences_sampled():
    """Sixteen sampled coordinates (actions, E, yield curvature, initial positions) of a
    longer rollout: device adjoint against FP64 central differences of the oracle, h = 1e-6
    relative to the coordinate's scale."""
    p = inputs.small_case("diff", n_rods=2, n=16, frames=10)
    wx, wv, wth = weights(p, 3)
    sim = sim_for(p)
    got = device_gradients(sim, p, 10, wx, wv, wth)

    om_w = np.zeros(int(p.edge_off[-1]))
    for b in range(p.batch):
        ne = p.edge_off[b + 1] - p.edge_off[b]
        om_w[p.edge_off[b]:p.edge_off[b + 1]] = wv[p.vert_off[b]:p.vert_off[b] + ne, 3]

    def loss(pp):
        o = OracleSim(pp)
        o.set_state(pp.x0, pp.v0, pp.theta0, pp.omega0)
        o.step(pp.actions, 10)
        st = o.get_state()
        return float((st["x"] * wx[:, :3]).sum() + (st["v"] * wv[:, :3]).sum() + (st["omega"] * om_w).sum()
                     + (st["theta"] * wth).sum())

    import copy
    rng = np.random.default_rng(7)
    picks = []
    for _ in range(6):
        picks.append(("act", (int(rng.integers(10)), int(rng.integers(2)), int(rng.integers(2)), int(rng.integers(6)))))
    for _ in range(4):
        picks.append(("x0", (int(rng.integers(p.x0.shape[0])), int(rng.integers(3)))))
    for b in range(2):
        picks.append(("E", b))
        picks.append(("yield_curv", b))
    picks.append(("v0", (3, 2)))
    picks.append(("v0", (20, 0)))
    n_ok = 0
    for name, idx in picks:
        base = {"act": p.actions, "x0": p.x0, "v0": p.v0, "E": p.E, "yield_curv": p.yield_curv}[name]
        scale = max(abs(float(np.asarray(base)[idx])), 1e-3 if name in ("act", "x0", "v0") else 1.0)
        h = 1e-6 * scale
        vals = []
        for sgn in (1, -1):
            q = copy.deepcopy(p)
            arr = {"act": q.actions, "x0": q.x0, "v0": q.v0, "E": q.E, "yield_curv": q.yield_curv}[name]
            arr[idx] += sgn * h
            vals.append(loss(q))
        fd = (vals[0] - vals[1]) / (2 * h)
        if name == "act":
            g = got["act"][idx]
        elif name in ("x0", "v0"):
            g = got[name][idx]
        else:
            g = got["material"][idx, {"E": 1, "yield_curv": 3}[name]]
        print("central difference", name, idx, "device %.6e fd %.6e rel %.2e" % (g, fd, abs(g - fd) / max(abs(fd), 1e-300)))
        assert g == pytest.approx(fd, rel=1e-3, abs=1e-6 * np.abs(got["act"]).max()), (name, idx, g, fd)
        n_ok += 1
    assert n_ok == 16


def test_checkpoint_interval_does_not_change_gradients():
    p = inputs.small_case("trajopt", n_rods=3, n=16, frames=6)
    wx, wv, wth = weights(p)
    outs = []
    for K in (1, 2, 6):
        sim = sim_for(p, checkpoint_every=K)
        outs.append(device_gradients(sim, p, 6, wx, wv, wth))
        sim.close()
    for k in GROUPS:
        for o in outs[1:]:
            np.testing.assert_allclose(o[k], outs[0][k], rtol=1e-4, atol=1e-6 * np.abs(outs[0][k]).max())


def test_backward_requires_a_recorded_rollout():
    from paper_2606_04206_gb300.dlo import DloError
    p = inputs.small_case("trajopt", n_rods=2, n=12, frames=2)
    sim = sim_for(p)
    sim.reset()
    with pytest.raises(DloError) as ei:
        sim.backward()
    assert ei.value.status == 7
    sim.begin_rollout(2)
    sim.step(None, 1)
    with pytest.raises(DloError) as ei:
        sim.backward()
    assert ei.value.status == 7


def test_backward_without_candidates_is_bitwise_reproducible():
    """Without self-contact candidates the reverse adds every cotangent in a fixed order (no
    floating-point atomics with more than two terms), so two backward passes of the same
    rollout, on two contexts, agree bit for bit in every gradient group."""
    p = inputs.trajopt(n_rods=6, frames=6, seed=17, n=48, self_contact=False)
    wx, wv, wth = weights(p, seed=3)
    outs = []
    for _ in range(2):
        sim = sim_for(p)
        outs.append(device_gradients(sim, p, 6, wx, wv, wth))
        sim.close()
    for k in GROUPS:
        assert np.array_equal(outs[0][k], outs[1][k]), k
