"""How far an exact float32 evaluation of the algorithm can sit from its FP64 result.

The oracle run in float32 (same code, same inputs) against the FP64 oracle: the gradients
with respect to the initial state and the actions agree to better than 1e-3, but the
material sensitivities p * dL/dp drift by a few 1e-3, because twist strains of nearly
untwisted rods (~1e-6 rad) sit close to the float32 resolution of the reference twist and
edge twist inertias are ~1e-9 kg m^2.  The device tests therefore hold material gradients to
1e-2 (relative L2 of the log-sensitivities) and everything else to 1e-3; this test keeps
that allowance tied to a measured float32 floor."""
import numpy as np
import pytest
import torch

from oracle import OracleSim
from paper_2606_04206_gb300 import inputs

NAMES = ("K", "E", "G", "yield_curv", "damping")


def gradients(p, frames, w, dtype):
    T = torch
    wx, wv, wth = w
    x0 = T.tensor(p.x0, dtype=dtype, requires_grad=True)
    act = T.tensor(p.actions[:frames], dtype=dtype, requires_grad=True)
    mats = {k: T.tensor(np.asarray(getattr(p, k)), dtype=dtype, requires_grad=True) for k in NAMES}
    sim = OracleSim(p, params=mats, dtype=dtype)
    sim.set_state(x0, T.tensor(p.v0, dtype=dtype), T.tensor(p.theta0, dtype=dtype), T.tensor(p.omega0, dtype=dtype))
    sim.step(act, frames, diff=True)
    st = sim.get_state(as_numpy=False)
    L = ((st["x"] * T.tensor(wx, dtype=dtype)).sum() + (st["v"] * T.tensor(wv, dtype=dtype)).sum()
         + (st["theta"] * T.tensor(wth, dtype=dtype)).sum())
    g = T.autograd.grad(L, [mats[k] for k in NAMES] + [x0, act], allow_unused=True)
    m = np.stack([(gi.double().numpy() if gi is not None else np.zeros(p.batch)) * np.asarray(getattr(p, k))
                  for gi, k in zip(g[:5], NAMES)], 1)
    return m, g[5].double().numpy(), g[6].double().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.slow
def test_float32_floor_of_material_sensitivities():
    p = inputs.small_case("trajopt", n_rods=3, n=12, frames=3)
    rng = np.random.default_rng(0)
    V, E = int(p.vert_off[-1]), int(p.edge_off[-1])
    w = (rng.normal(size=(V, 3)), rng.normal(size=(V, 3)) * 1e-2, rng.normal(size=E) * 1e-2)
    m64, x64, a64 = gradients(p, 3, w, torch.float64)
    m32, x32, a32 = gradients(p, 3, w, torch.float32)
    assert rel(x32, x64) < 1e-3 and rel(a32, a64) < 1e-3
    r = rel(m32, m64)
    assert 1e-4 < r < 1e-2, r           # well above 1e-3, inside the 1e-2 device allowance
