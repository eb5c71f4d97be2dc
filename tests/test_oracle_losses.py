"""Pins of the FP64 task-loss definitions (oracle/losses.py) against closed forms: Chamfer
distances of simple sets, winding numbers of circles and arcs about a post, the linking
number of a Hopf link (an exact integer for the pair integral), and symmetries of the
crossing sum (planar curves give 0, a mirror image flips the sign, rigid motions and scaling
leave it unchanged), the minimum distance to a point and the self-repulsion penalty against
sampled segment distances."""
import math

import numpy as np
import pytest
import torch

from oracle.losses import chamfer, winding, gauss_pair, crossing, linking, mindist, repulsion

T = lambda a: torch.as_tensor(np.asarray(a, np.float64))


def circle(n, r=1.0, c=(0.0, 0.0, 0.0), plane="xy", a0=0.0, a1=2 * math.pi, closed=True):
    s = np.linspace(a0, a1, n, endpoint=not closed)
    u, v = r * np.cos(s), r * np.sin(s)
    z = np.zeros(n)
    pts = {"xy": (u, v, z), "xz": (u, z, v)}[plane]
    return T(np.stack(pts, 1) + np.asarray(c))


def test_chamfer_closed_forms():
    rng = np.random.default_rng(0)
    x = T(rng.uniform(-1, 1, (20, 3)))
    assert float(chamfer(x, x)) == 0.0
    assert float(chamfer(T([[0, 0, 0]]), T([[3, 4, 0]]))) == pytest.approx(50.0, rel=1e-15)
    g = T(np.stack(np.meshgrid(np.arange(4.0), np.arange(4.0), [0.0], indexing="ij"), -1).reshape(-1, 3))
    d = T([0.1, -0.2, 0.05])          # small against the unit spacing: nearest points stay paired
    assert float(chamfer(g, g + d)) == pytest.approx(2 * float((d * d).sum()), rel=1e-14)


def test_winding_of_circles_and_arcs():
    c = circle(64)
    assert float(winding(c, (0, 0), closed=True)) == pytest.approx(1.0, abs=1e-13)
    assert float(winding(torch.flip(c, [0]), (0, 0), closed=True)) == pytest.approx(-1.0, abs=1e-13)
    assert float(winding(c, (3, 0), closed=True)) == pytest.approx(0.0, abs=1e-13)
    arc = circle(33, a0=0.2, a1=2.0, closed=False)
    assert float(winding(arc, (0, 0))) == pytest.approx((2.0 - 0.2) / (2 * math.pi), abs=1e-13)


def test_linking_number_of_a_hopf_link_is_an_integer():
    a = circle(64, plane="xy")
    b = circle(64, plane="xz", c=(1.0, 0.0, 0.0))
    lk = float(linking(a, b))
    assert abs(abs(lk) - 1.0) < 1e-10, lk
    assert float(linking(a, torch.flip(b, [0]))) == pytest.approx(-lk, abs=1e-10)
    assert float(linking(a, circle(64, plane="xz", c=(3.0, 0.0, 0.0)))) == pytest.approx(0.0, abs=1e-10)
    # coarse polygons still link exactly: the pair integral is exact for straight segments
    assert abs(abs(float(linking(circle(7, plane="xy"), circle(5, plane="xz", c=(1.0, 0, 0))))) - 1.0) < 1e-10


def test_pair_integral_is_symmetric_and_zero_when_coplanar():
    rng = np.random.default_rng(1)
    p = [T(rng.normal(size=3)) for _ in range(4)]
    assert float(gauss_pair(*p)) == pytest.approx(float(gauss_pair(p[2], p[3], p[0], p[1])), rel=1e-12)
    q = [T(np.append(rng.normal(size=2), 0.0)) for _ in range(4)]
    assert float(gauss_pair(*q)) == 0.0


def test_crossing_sum_symmetries():
    rng = np.random.default_rng(2)
    s = np.linspace(0, 1, 40)
    x = T(np.stack([np.cos(7 * s) + 0.1 * s, np.sin(5 * s), 0.6 * np.sin(11 * s)], 1) + 0.01 * rng.normal(size=(40, 3)))
    w = float(crossing(x))
    assert abs(w) > 1e-3
    planar = x.clone()
    planar[:, 2] = 0.0
    assert float(crossing(planar)) == 0.0
    mirror = x.clone()
    mirror[:, 2] = -mirror[:, 2]
    assert float(crossing(mirror)) == pytest.approx(-w, rel=1e-12)
    th = 0.7
    Rz = T([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    assert float(crossing(2.5 * x @ Rz.T + T([1.0, -2.0, 0.5]))) == pytest.approx(w, rel=1e-12)


def test_mindist_closed_form_and_gradient():
    x = T(np.stack([np.linspace(0, 1, 11), np.zeros(11), np.zeros(11)], 1))
    o = T([0.43, 0.3, 0.4])
    xr = x.clone().requires_grad_(True)
    d = mindist(xr, o)
    assert float(d) == pytest.approx(math.sqrt(0.03 ** 2 + 0.3 ** 2 + 0.4 ** 2), rel=1e-14)
    g, = torch.autograd.grad(d, [xr])
    want = np.zeros((11, 3))
    want[4] = (np.array([0.4, 0.0, 0.0]) - [0.43, 0.3, 0.4]) / float(d)
    assert np.allclose(g.numpy(), want, atol=1e-14)


def sampled_distance(p, q, r, t, m=401):
    s = np.linspace(0, 1, m)
    a = p[None] + s[:, None] * (q - p)[None]
    b = r[None] + s[:, None] * (t - r)[None]
    return np.sqrt(((a[:, None] - b[None]) ** 2).sum(-1)).min()


def test_repulsion_against_sampled_distances():
    # a hairpin: out along y = 0, a short bend, back along y = h (plus a little lift)
    h, e = 0.006, 0.004
    out = np.stack([np.arange(12) * e, np.zeros(12), np.zeros(12)], 1)
    back = np.stack([np.arange(11, -1, -1) * e + 0.0005, np.full(12, h), np.full(12, 0.001)], 1)
    x = np.concatenate([out, back])
    delta, k = 2 * e, 2
    pen = float(repulsion(T(x), delta, k))
    ne = len(x) - 1
    want = 0.0
    for a in range(ne):
        for b in range(a + k + 1, ne):
            d = sampled_distance(x[a], x[a + 1], x[b], x[b + 1])
            want += max(0.0, delta - d) ** 2
    assert pen > 0 and pen == pytest.approx(want, rel=2e-3)


def test_repulsion_closed_forms():
    e = 0.004
    line = T(np.stack([np.arange(30) * e, np.zeros(30), np.zeros(30)], 1))
    assert float(repulsion(line, 2 * e, 2)) < 1e-30            # a straight rod is free at k = 2 (d = delta)
    assert float(repulsion(line, 2 * e, 1)) == pytest.approx(27 * e * e, rel=1e-12)   # pairs 2 apart: d = e
    # two parallel edges h apart, overlapping: (delta - h)^2 for the one pair
    x = T([[0, 0, 0], [1, 0, 0], [1, 5, 0], [0.2, 0.3, 0], [0.9, 0.3, 0]])
    assert float(repulsion(x, 0.5, 2)) == pytest.approx(0.2 ** 2, rel=1e-12)
