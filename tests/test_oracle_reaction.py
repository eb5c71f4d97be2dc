"""Pins of the oracle's rigid-contact impulse accounting (the two-way coupling diagnostic of
Sec. 3.2): a rod lying on the ground receives exactly its weight times the frame time from
the plane, and for a free rod falling and sliding on the ground the momentum balance
dP = J - M g t holds (internal forces sum to zero and the projections keep momentum)."""
import numpy as np
import pytest

from oracle import OracleSim
from paper_2606_04206_gb300 import inputs

R = 0.002
PLANE = np.array([[0.0, 0.0, 1.0, 0.0]])


def straight(n, z, tilt=0.0):
    x = np.zeros((n, 3))
    x[:, 0] = np.linspace(0.0, 0.5, n)
    x[:, 2] = z + tilt * np.linspace(0.0, 1.0, n)
    return x


def test_rod_at_rest_on_the_ground_carries_its_weight():
    p = inputs.custom([straight(16, R)], frames=3, K=1e5, E=1e4, G=0.0, damping=0.0, planes=PLANE)
    o = OracleSim(p)
    o.set_state(p.x0, p.v0, p.theta0, p.omega0)
    o.track_reaction()
    o.step(np.zeros((3, 1, 2, 6)), 3)
    per_rod, per_v = o.reaction()
    M = float(o.rod_constants()["mass"].sum())
    assert per_rod[0, 0] == pytest.approx([0.0, 0.0, M * p.gravity * 3 * p.dt], rel=1e-12, abs=1e-18)
    assert not per_rod[0, 1:].any()
    # every vertex carries its own weight
    m = o.rod_constants()["mass"]
    assert np.allclose(per_v[:, 0, 2], m * p.gravity * 3 * p.dt, rtol=1e-12)


def test_momentum_balance_of_a_falling_sliding_rod():
    p = inputs.custom([straight(20, 0.004, tilt=0.01)], frames=12, K=1e5, E=1e4, G=1e3, damping=0.0,
                      planes=PLANE)
    v0 = np.zeros_like(p.v0)
    v0[:] = [0.4, 0.1, -0.5]
    o = OracleSim(p)
    o.set_state(p.x0, v0, p.theta0, p.omega0)
    P0 = o.momentum()[0]
    o.track_reaction()
    o.step(np.zeros((12, 1, 2, 6)), 12)
    J = o.reaction()[0][0].sum(0)
    M = float(o.rod_constants()["mass"].sum())
    dP = o.momentum()[0] - P0
    want = J - np.array([0.0, 0.0, M * p.gravity * 12 * p.dt])
    assert J[2] > 0 and abs(J[0]) > 0                                  # it landed and slid (friction)
    assert np.allclose(dP, want, rtol=1e-9, atol=1e-12 * M)
