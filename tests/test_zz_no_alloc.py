"""dlo_backward_noalloc: the rollout adjoint with every temporary in the library's static
scratch.  Compared with dlo_backward on the same recorded rollout, twice in a row; the
library's allocator callback must not be called and the context's device bytes must not
change during the call; a rollout whose per-rod recompute buffers exceed the static scratch
is rejected with DLO_ERR_CAPACITY.  Kept in its own file, collected after the other GPU
tests, and meant to pass both alone in a fresh process and after them."""
import numpy as np
import pytest
import torch

from paper_2606_04206_gb300 import inputs
from paper_2606_04206_gb300.dlo import DloError, Q_BYTES
from gpu_util import sim_for, grad_agreement

pytestmark = pytest.mark.gpu

GROUPS = ("actions", "material", "x0", "v0", "theta0")


def rollout(sim, p, frames, substeps=0):
    sim.reset()
    sim.begin_rollout(frames)
    acts = torch.as_tensor(np.ascontiguousarray(p.actions[:frames], np.float32), device=sim.device)
    sim.step(acts, frames, substeps)


def loss_weights(p, seed=0):
    rng = np.random.default_rng(seed)
    V, E = int(p.vert_off[-1]), int(p.edge_off[-1])
    wx = torch.zeros(V, 4, device="cuda")
    wx[:, :3] = torch.as_tensor(rng.normal(size=(V, 3)), dtype=torch.float32)
    wv = torch.zeros(V, 4, device="cuda")
    wv[:, :3] = torch.as_tensor(rng.normal(size=(V, 3)) * 1e-2, dtype=torch.float32)
    wth = torch.as_tensor(rng.normal(size=E) * 1e-2, dtype=torch.float32, device="cuda")
    return wx, wv, wth


def noalloc_then_backward(sim, p, frames, monkeypatch):
    """On a freshly recorded rollout: dlo_backward_noalloc first (so that no earlier call has
    grown the context's workspace), counting the library's allocator calls, then dlo_backward
    as the reference, then dlo_backward_noalloc again."""
    w = loss_weights(p)
    calls = []
    real = torch.cuda.caching_allocator_alloc
    monkeypatch.setattr(torch.cuda, "caching_allocator_alloc", lambda *a, **k: calls.append(a) or real(*a, **k))
    outs = []
    for rep in range(2):
        # the outputs are the caller's: allocate them before counting the library's calls
        F = frames
        out = {"actions": torch.zeros(F, p.batch, 2, 6, device="cuda"), "material": torch.zeros(p.batch, 5, device="cuda"),
               "x0": torch.zeros(sim.V, 4, device="cuda"), "v0": torch.zeros(sim.V, 4, device="cuda"),
               "theta0": torch.zeros(sim.E, device="cuda")}
        bytes_before = sim.query(Q_BYTES)
        n_calls = len(calls)
        st = sim.lib.dlo_backward_noalloc(sim.ctx, w[0].data_ptr(), w[1].data_ptr(), w[2].data_ptr(),
                                          out["actions"].data_ptr(), out["material"].data_ptr(),
                                          out["x0"].data_ptr(), out["v0"].data_ptr(), out["theta0"].data_ptr())
        sim._check(st, "dlo_backward_noalloc")
        assert len(calls) == n_calls, "the library allocated during dlo_backward_noalloc"
        assert sim.query(Q_BYTES) == bytes_before
        outs.append(out)
        if rep == 0:
            ref = sim.backward(*w)
            torch.cuda.synchronize()
    for rep, out in enumerate(outs):
        for k in GROUPS:
            a, b = out[k].double().cpu().numpy(), ref[k].double().cpu().numpy()
            rel, cos = grad_agreement(a, b)
            assert rel <= 1e-3 and cos >= 0.999, (rep, k, rel, cos)
    # the binding's method gives the same
    again = sim.backward_noalloc(*w)
    for k in GROUPS:
        rel, cos = grad_agreement(again[k].double().cpu().numpy(), ref[k].double().cpu().numpy())
        assert rel <= 1e-3 and cos >= 0.999, (k, rel, cos)


@pytest.mark.parametrize("kind", ["trajopt", "selfcontact"])
def test_noalloc_matches_backward_twice_in_a_row(kind, monkeypatch):
    p = inputs.small_case(kind, n_rods=3, n=30, frames=6)
    sim = sim_for(p)
    rollout(sim, p, 6)
    noalloc_then_backward(sim, p, 6, monkeypatch)


def test_noalloc_with_more_resident_rods_than_the_static_scratch_holds(monkeypatch):
    """400 rods of 128 vertices, checkpoints every 50 frames: each resident rod needs ~1.1 MB of
    recompute scratch, so the static array holds fewer rods at once (~240) than the backward
    keeps resident when it allocates (three per SM); the rods then run in fewer, longer-lived
    slots, with the same gradients."""
    p = inputs.small_case("trajopt", n_rods=400, n=128, frames=50)
    sim = sim_for(p, checkpoint_every=50)
    rollout(sim, p, 50)
    noalloc_then_backward(sim, p, 50, monkeypatch)


def test_noalloc_rejects_a_rollout_beyond_the_static_scratch():
    # one 256-vertex rod, one frame of 2000 substeps: the per-rod recompute buffers of one
    # frame alone are ~450 MB, above the 256 MiB static scratch
    x = np.zeros((256, 3))
    x[:, 0] = np.linspace(0.0, 1.0, 256)
    x[:, 2] = 0.5
    p = inputs.custom([x], frames=1)
    sim = sim_for(p)
    rollout(sim, p, 1, substeps=2000)
    with pytest.raises(DloError) as e:
        sim.backward_noalloc(*loss_weights(p))
    assert e.value.status == 5 and "static scratch" in str(e.value)
