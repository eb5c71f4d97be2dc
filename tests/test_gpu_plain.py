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
