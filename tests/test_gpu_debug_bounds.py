"""The bounds-checking debug build of the library (build(debug_bounds=True), compiled with
-DDLO_DEBUG_BOUNDS): every index the kernels take from data (candidate pairs, kinematic kinds,
recorded pair counts, work-queue items) is checked before use, and a failed check would set
status bit 8 and give DLO_ERR_BOUNDS.

On valid contact-heavy runs (forward, fused backward, plain forward and backward) the checks
stay silent, and the debug library's results equal the release library's to float rounding
(the checks change no arithmetic; the two builds may contract multiply-adds differently).
No test feeds an invalid index to a kernel."""
import numpy as np
import pytest
import torch

from paper_2606_04206_gb300 import build, dlo, inputs
from gpu_util import sim_for, actions_dev, device_gradients, grad_agreement, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def debug_lib():
    build.build(debug_bounds=True)
    return dlo.load(dlo.LIB_DEBUG_PATH)


def run(sim, p, frames, wx):
    g = device_gradients(sim, p, frames, wx, np.zeros_like(wx), np.zeros(int(p.edge_off[-1])))
    x = sim.full_state_numpy()["x"]
    return x, g


@pytest.mark.parametrize("kind", ["selfcontact", "separation", "trajopt"])
def test_debug_build_is_silent_and_equal_on_valid_runs(kind, debug_lib):
    assert debug_lib.dlo_build_flags() == 1
    n = 30 if kind != "separation" else 14
    p = inputs.small_case(kind, n_rods=4, n=n, frames=6)
    wx = np.zeros((int(p.vert_off[-1]), 4))
    wx[:, :3] = np.random.default_rng(1).normal(size=(len(wx), 3))
    rel = sim_for(p)
    assert rel.lib.dlo_build_flags() == 0
    x_r, g_r = run(rel, p, 6, wx)
    dbg = dlo.DloSim(p, debug_bounds=True)
    x_d, g_d = run(dbg, p, 6, wx)
    assert not (dbg.query(dlo.Q_STATUS) & dlo.STATUS_BOUNDS).any()
    assert rel_inf(x_d, x_r) <= 1e-6
    for k in ("x0", "act", "material"):
        r, c = grad_agreement(g_d[k], g_r[k])
        assert r <= 1e-5 and c >= 0.99999, (k, r, c)
    # the plain comparator's kernels, forward and backward, in the debug build
    dbg.reset()
    dbg.begin_rollout(6)
    dbg.step_plain(actions_dev(p), 6)
    gz = torch.zeros(dbg.V, 4, device=dbg.device)
    gz[:, 2] = 1.0
    dbg.backward(dL_dx=gz, plain=True)
    assert not (dbg.query(dlo.Q_STATUS) & dlo.STATUS_BOUNDS).any()
