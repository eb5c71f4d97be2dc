"""Failure detection through the C ABI, with every failure made on the host or by the method's
own inputs (no device fault, trap or hang is provoked):

  * an allocator that returns NULL gives DLO_ERR_OOM from dlo_create, dlo_begin_rollout and
    dlo_backward, and the context works again once memory is available;
  * a coil denser than the pair list's capacity (4 per vertex of the rod's size class) drops
    the extra candidates, sets the rod's overflow bit and gives DLO_ERR_CAPACITY naming it;
  * a stiff rod forced to one substep per frame (far beyond the explicit stability limit)
    becomes non-finite and gives DLO_ERR_NONFINITE naming it; dlo_set_state clears it.
"""
import numpy as np
import pytest
import torch

from paper_2606_04206_gb300 import inputs
from paper_2606_04206_gb300.dlo import DloError, DloSim, Q_STATUS, STATUS_PAIR_OVERFLOW
from gpu_util import sim_for

pytestmark = pytest.mark.gpu

OOM, CAPACITY, NONFINITE = 3, 5, 4


class Budget:
    """Device allocations through torch, refused once `left` reaches zero (None = no limit)."""

    def __init__(self, left=None):
        self.left = left
        self.calls = 0

    def alloc(self, nbytes):
        self.calls += 1
        if self.left is not None:
            if self.left <= 0:
                return None
            self.left -= 1
        return torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), torch.cuda.current_stream())

    def free(self, ptr):
        torch.cuda.caching_allocator_delete(ptr)


def test_allocator_returning_null_gives_oom_and_the_context_recovers():
    from paper_2606_04206_gb300 import build
    build.build()
    p = inputs.small_case("trajopt", n_rods=3, n=24, frames=3)
    # dlo_create: refuse the first allocation, then the last one it needs
    with pytest.raises(DloError) as e:
        DloSim(p, allocator=(Budget(0).alloc, Budget(0).free))
    assert e.value.status == OOM
    count = Budget()
    DloSim(p, allocator=(count.alloc, count.free)).close()
    assert count.calls > 1
    with pytest.raises(DloError) as e:
        DloSim(p, allocator=(Budget(count.calls - 1).alloc, Budget().free))
    assert e.value.status == OOM
    # dlo_begin_rollout: the checkpoint ring, then the action record
    bud = Budget()
    sim = DloSim(p, allocator=(bud.alloc, bud.free))
    sim.reset()
    for allowed in (0, 1):
        bud.left = allowed
        with pytest.raises(DloError) as e:
            sim.begin_rollout(3)
        assert e.value.status == OOM and "allocation failed" in str(e.value)
    bud.left = None
    sim.begin_rollout(3)
    acts = torch.as_tensor(np.ascontiguousarray(p.actions, np.float32), device="cuda")
    sim.step(acts, 3)
    # dlo_backward: its workspace
    bud.left = 0
    with pytest.raises(DloError) as e:
        sim.backward(dL_dx=torch.ones(sim.V, 4, device="cuda"))
    assert e.value.status == OOM
    bud.left = None
    g = sim.backward(dL_dx=torch.ones(sim.V, 4, device="cuda"))
    assert all(bool(torch.isfinite(v).all()) for v in g.values())
    sim.close()


def test_pair_list_overflow_gives_capacity_error_naming_the_rod():
    # rod 1: 32 vertices wound 6 turns on a 5 mm helix of 0.4 mm pitch, about 340 candidate
    # pairs against a capacity of 4 x 32 = 128; rod 0: a straight rod with none
    s = np.linspace(0.0, 12.0 * np.pi, 32)
    coil = np.stack([0.005 * np.cos(s), 0.005 * np.sin(s), 0.05 + 0.0004 * s / (2 * np.pi)], 1)
    straight = np.stack([np.linspace(0.0, 0.2, 32), np.full(32, 0.3), np.full(32, 0.05)], 1)
    p = inputs.custom([straight, coil], frames=1, K=1e5, E=1e4, G=1e3, gravity=0.0, self_contact=True)
    sim = sim_for(p)
    sim.reset()
    sim.step(None, 1)
    st = sim.query(Q_STATUS)
    assert not (st[0] & STATUS_PAIR_OVERFLOW) and (st[1] & STATUS_PAIR_OVERFLOW), st
    assert len(sim.pair_sets()[1]) == 128              # the list holds its capacity
    with pytest.raises(DloError) as e:
        sim.get_state()
    assert e.value.status == CAPACITY and "rod 1" in str(e.value)


def test_stiff_rod_forced_to_one_substep_becomes_nonfinite():
    # rod 1: K = E = 1e8 Pa with 1.6 cm edges needs ~64 substeps per 1 ms frame (stretching
    # frequency ~6e4 /s); one substep puts omega h near 60, far past the limit 2
    rng = np.random.default_rng(4)
    t = np.linspace(0.0, 1.0, 64)
    bent = np.stack([t, 0.05 * np.sin(3 * t) + 0.002 * rng.normal(size=64), np.full(64, 0.3)], 1)
    soft = bent + np.array([0.0, 0.5, 0.0])
    p = inputs.custom([soft, bent], frames=1, K=[1e3, 1e8], E=[1e2, 1e8], G=[0.0, 4e7])
    sim = sim_for(p)
    assert sim.query(1)[1] > 20                        # DLO_Q_SUBSTEPS: the rod's own count
    sim.reset()
    err = None
    for _ in range(40):
        sim.step(None, 1, substeps=1)
        try:
            sim.get_state()
        except DloError as e:
            err = e
            break
    assert err is not None and err.status == NONFINITE and "rod 1" in str(err), err
    # a fresh state clears the status; the rod's own substep count keeps it finite
    sim.reset()
    sim.step(None, 3)
    x = sim.get_state()[0]
    assert bool(torch.isfinite(x).all())
