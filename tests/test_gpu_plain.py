"""The plain per-phase GPU comparator (dlo_step_plain: one launch per phase per substep,
state in HBM) against the FP64 oracle, and against the persistent forward kernel, at the
forward path's tolerances: vertex positions within 1e-5 m after 100 contact-free frames of
the plain workload, and a per-frame relative error <= 1e-5 from the same state with contact."""
import numpy as np
import pytest
import torch

from oracle import OracleSim
from paper_2606_04206_gb300 import inputs
from gpu_util import sim_for, oracle_from_device_state, actions_dev, rel_inf

pytestmark = pytest.mark.gpu


def test_plain_comparator_contact_free_against_oracle():
    p = inputs.plain(100)
    sim = sim_for(p)
    sim.reset()
    sim.step_plain(actions_dev(p), 100)
    o = OracleSim(p)
    o.set_state(p.x0, p.v0, p.theta0, p.omega0)
    o.step(p.actions, 100)
    x = sim.get_state()[0][:, :3].double().cpu().numpy()
    assert np.abs(x - o.get_state()["x"]).max() <= 1e-5


@pytest.mark.parametrize("kind,warm", [("trajopt", 20), ("selfcontact", 5), ("batching", 5), ("diff", 5)])
def test_plain_comparator_one_frame_with_contact(kind, warm):
    p = inputs.small_case(kind, n_rods=4, n=40, frames=warm + 1)
    sim = sim_for(p)
    sim.reset()
    acts = actions_dev(p)
    sim.step_plain(acts[:warm].contiguous(), warm)
    o = oracle_from_device_state(p, sim)
    sim.step_plain(acts[warm:warm + 1].contiguous(), 1)
    o.step(p.actions[warm:warm + 1], 1)
    fo, fg = o.get_state(), sim.full_state_numpy()
    assert rel_inf(fg["x"], fo["x"]) <= 1e-5
    assert rel_inf(fg["v"], fo["v"]) <= 2e-3
    assert np.abs(fg["theta"] - fo["theta"]).max() <= 1e-4


@pytest.mark.parametrize("kind", ["trajopt", "selfcontact", "batching"])
def test_plain_comparator_follows_the_persistent_kernel(kind):
    p = inputs.small_case(kind, n_rods=6, n=48, frames=3)
    sim = sim_for(p)
    acts = actions_dev(p)
    sim.reset()
    sim.step(acts, 3)
    a = sim.full_state_numpy()
    sim.reset()
    sim.step_plain(acts, 3)
    b = sim.full_state_numpy()
    assert rel_inf(b["x"], a["x"]) <= 1e-5
    assert rel_inf(b["v"], a["v"]) <= 1e-3
    for k in ("d1b", "tb", "kbar", "gp"):
        assert np.abs(b[k] - a[k]).max() <= 1e-4, k
    assert not sim.query(2).any()            # DLO_Q_STATUS: finite, no pair overflow


# ---------------------------------------------------------------------- the plain backward

def plain_gradients(sim, prob, frames, wx, wv, wth, record_plain=True, plain_bwd=True):
    """A recorded rollout (dlo_step_plain or dlo_step) differentiated by dlo_backward_plain or
    dlo_backward; numpy arrays in the oracle's layout (as gpu_util.device_gradients)."""
    dev = sim.device
    sim.reset()
    sim.begin_rollout(frames)
    acts = torch.as_tensor(np.ascontiguousarray(prob.actions[:frames], np.float32), device=dev)
    (sim.step_plain if record_plain else sim.step)(acts, frames)
    g = sim.backward(torch.as_tensor(wx, dtype=torch.float32, device=dev), torch.as_tensor(wv, dtype=torch.float32, device=dev),
                     torch.as_tensor(wth, dtype=torch.float32, device=dev), plain=plain_bwd)
    g = {k: v.double().cpu().numpy() for k, v in g.items()}
    vo, eo = prob.vert_off, prob.edge_off
    om = np.zeros(int(eo[-1]))
    for b in range(prob.batch):
        om[eo[b]:eo[b + 1]] = g["v0"][vo[b]:vo[b] + eo[b + 1] - eo[b], 3]
    return dict(x0=g["x0"][:, :3], v0=g["v0"][:, :3], om0=om, th0=g["theta0"], act=g["actions"],
                material=g["material"])


@pytest.mark.parametrize("kind", ["trajopt", "diff", "batching", "selfcontact"])
def test_plain_backward_matches_oracle_autograd(kind):
    """dlo_step_plain + dlo_backward_plain against the FP64 oracle's reverse mode, at the
    gradient bar (relative L2 <= 1e-3, cosine >= 0.999; material as p dL/dp)."""
    from gpu_util import oracle_gradients, grad_agreement
    from test_gpu_backward import weights, log_sens, GROUPS
    p = inputs.small_case(kind, n_rods=3, n=12 if kind != "selfcontact" else 30, frames=3)
    wx, wv, wth = weights(p)
    ref, _ = oracle_gradients(p, 3, wx, wv, wth)
    sim = sim_for(p)
    got = plain_gradients(sim, p, 3, wx, wv, wth)
    got["material"], ref["material"] = log_sens(p, got["material"]), log_sens(p, ref["material"])
    report = {k: grad_agreement(got[k], ref[k]) for k in GROUPS}
    print("plain backward vs oracle (rel L2, cosine):", {k: (f"{r:.2e}", f"{c:.6f}") for k, (r, c) in report.items()})
    assert all(r <= 1e-3 and c >= 0.999 for r, c in report.values()), report


@pytest.mark.parametrize("kind,ck", [("trajopt", 2), ("selfcontact", 3)])
def test_plain_backward_equals_the_fused_adjoint(kind, ck):
    """The same recorded rollout differentiated by both adjoints, with checkpoints every ck
    frames (the plain one re-runs the frames before each frame of a segment): equal to float
    rounding."""
    from gpu_util import grad_agreement
    from test_gpu_backward import weights, GROUPS
    p = inputs.small_case(kind, n_rods=4, n=32, frames=6)
    wx, wv, wth = weights(p, 1)
    sim = sim_for(p, checkpoint_every=ck)
    fused = plain_gradients(sim, p, 6, wx, wv, wth, record_plain=False, plain_bwd=False)
    plain = plain_gradients(sim, p, 6, wx, wv, wth, record_plain=True, plain_bwd=True)
    for k in GROUPS:
        rel, cos = grad_agreement(plain[k], fused[k])
        assert rel <= 1e-4 and cos >= 0.999999, (k, rel, cos)
