"""The contact impulses dlo_step accumulates (dlo_reaction) against the oracle's accounting
(pinned in tests/test_oracle_reaction.py): one frame from a shared state with the ground and
both grippers in contact, a rod at rest carrying its weight, and the accumulate / reset /
disabled behaviour."""
import numpy as np
import pytest
import torch

from paper_2606_04206_gb300 import dlo, inputs
from gpu_util import sim_for, oracle_from_device_state, actions_dev

pytestmark = pytest.mark.gpu


def box_scene(frames):
    """One rod lying on a box (0.3 x 0.3 x 0.1 m at the origin), one on the ground beside it."""
    a = np.zeros((24, 3))
    a[:, 0] = np.linspace(-0.1, 0.1, 24)
    a[:, 2] = 0.1 + 0.002
    b = a.copy()
    b[:, 1] = 0.3
    b[:, 2] = 0.002
    return inputs.custom([a, b], frames=frames, K=1e5, E=1e4, G=0.0,
                         planes=np.array([[0.0, 0.0, 1.0, 0.0]]),
                         boxes=np.array([[0.0, 0.0, 0.05, 0.15, 0.15, 0.05]]))


@pytest.mark.parametrize("kind", ["trajopt", "box"])
def test_reaction_matches_oracle_one_frame(kind):
    """trajopt: 128-vertex rods on the ground, the grippers' neighbours touching the capsules;
    box: the box and plane slots."""
    p = inputs.small_case("trajopt", n_rods=3, n=128, frames=42) if kind == "trajopt" else box_scene(42)
    sim = sim_for(p, reaction=1)
    sim.reset()
    sim.step(actions_dev(p, 0, 40), 40)              # settle, grippers moving
    o = oracle_from_device_state(p, sim)
    sim.reaction(reset=True)
    sim.step(actions_dev(p, 40, 41), 1)
    got_rod, got_v = sim.reaction(per_vertex=True)
    o.track_reaction()
    o.step(p.actions[40:41], 1)
    ref_rod, ref_v = o.reaction()
    got_rod, got_v = got_rod.double().cpu().numpy(), got_v.double().cpu().numpy()
    scale = np.abs(ref_rod).max()
    if kind == "trajopt":
        assert np.abs(ref_rod[:, 0, 2]).min() > 0 and np.abs(ref_rod[:, 2:]).max() > 0   # ground and a gripper
    else:
        assert ref_rod[0, 1, 2] > 0 and ref_rod[1, 0, 2] > 0 and ref_rod[0, 0, 2] == 0
    assert np.abs(got_rod - ref_rod).max() <= 1e-4 * scale, np.abs(got_rod - ref_rod).max() / scale
    assert np.abs(got_v - ref_v).max() <= 1e-4 * np.abs(ref_v).max()


def test_rod_at_rest_carries_its_weight():
    x = np.zeros((16, 3))
    x[:, 0] = np.linspace(0.0, 0.5, 16)
    x[:, 2] = 0.002
    p = inputs.custom([x], frames=4, K=1e5, E=1e4, G=0.0, damping=0.0,
                      planes=np.array([[0.0, 0.0, 1.0, 0.0]]))
    sim = sim_for(p, reaction=1)
    sim.reset()
    sim.step(actions_dev(p), 4)
    per_rod, _ = sim.reaction()
    M = float(sim.query(dlo.Q_MASS)[:, 0].sum())
    assert per_rod[0, 0].cpu().numpy() == pytest.approx([0.0, 0.0, M * p.gravity * 4 * p.dt], rel=1e-5, abs=1e-12)


def test_accumulate_reset_and_disabled():
    p = box_scene(4)
    sim = sim_for(p, reaction=1)
    sim.reset()
    sim.step(actions_dev(p, 0, 2), 2)
    a, _ = sim.reaction()
    sim.step(actions_dev(p, 2, 4), 2)
    ab, _ = sim.reaction(reset=True)
    z, _ = sim.reaction()
    assert not z.any()
    assert a[0, 1, 2] > 0 and torch.allclose(ab, 2 * a, rtol=1e-4)      # at rest: two equal pairs of frames
    plain = sim_for(p)
    with pytest.raises(RuntimeError):
        plain.reaction()
