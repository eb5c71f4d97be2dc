"""Pins of the FP64 silhouette definition (oracle/silhouette.py): the pinhole projection by
hand, one edge's coverage against the logistic of its pixel distance, the union of two
distant edges, the covered area of a sharp capsule against 2 rho L + pi rho^2, and the loss
of an empty mask."""
import math

import numpy as np
import pytest
import torch

from oracle.silhouette import camera, project, render, silhouette_loss

DOWN = np.diag([1.0, -1.0, -1.0])       # looks down -z; image v grows with -y


def test_projection_by_hand():
    cam = camera(200.0, 180.0, 32.0, 24.0, DOWN, [0.0, 0.0, 1.5])
    x = torch.tensor([[0.0, 0.0, 0.0], [0.3, -0.15, 0.5]], dtype=torch.float64)
    uv, rho, Z = project(x, cam, 0.002)
    assert np.allclose(uv[0].numpy(), [32.0, 24.0])
    assert float(Z[1]) == pytest.approx(1.0)
    assert np.allclose(uv[1].numpy(), [32.0 + 200.0 * 0.3 / 1.0, 24.0 + 180.0 * 0.15 / 1.0])
    assert float(rho[0]) == pytest.approx(200.0 * 0.002 / 1.5)


def px_to_world(u, v, cam_h, f, cx, cy):
    """A world point on z = 0 that the DOWN camera at height cam_h maps to pixel (u, v)."""
    return [(u - cx) * cam_h / f, -(v - cy) * cam_h / f, 0.0]


def test_one_edge_is_the_logistic_of_the_pixel_distance():
    f, h, tau, r = 100.0, 1.0, 0.7, 0.03          # rho = 3 px
    cam = camera(f, f, 0.0, 0.0, DOWN, [0.0, 0.0, h])
    x = torch.tensor([px_to_world(10.0, 20.5, h, f, 0, 0), px_to_world(30.0, 20.5, h, f, 0, 0)], dtype=torch.float64)
    o = render(x, cam, 40, 40, tau, r)
    sig = lambda z: 1.0 / (1.0 + math.exp(-z))
    assert float(o[25, 15]) == pytest.approx(sig((3.0 - 5.0) / tau), rel=1e-12)       # 5 px below the axis
    d = math.hypot(35.5 - 30.0, 25.5 - 20.5)                                          # beyond the end cap
    assert float(o[25, 35]) == pytest.approx(sig((3.0 - d) / tau), rel=1e-12)


def test_two_distant_edges_compose_as_a_union():
    f, h, tau, r = 100.0, 1.0, 1.0, 0.02
    cam = camera(f, f, 0.0, 0.0, DOWN, [0.0, 0.0, h])
    pts = [px_to_world(u, v, h, f, 0, 0) for u, v in ((5.0, 5.0), (5.0, 15.0), (25.0, 15.0))]
    x = torch.tensor(pts, dtype=torch.float64)
    o = render(x, cam, 30, 30, tau, r)
    sig = lambda z: 1.0 / (1.0 + math.exp(-z))
    p = (15.5, 9.5)   # 10.5 px from edge 0's axis (u = 5), 5.5 px from edge 1's (v = 15)
    s0, s1 = sig((2.0 - 10.5) / tau), sig((2.0 - 5.5) / tau)
    assert float(o[9, 15]) == pytest.approx(1 - (1 - s0) * (1 - s1), rel=1e-12)


def test_sharp_capsule_covers_its_area():
    f, h, r = 100.0, 1.0, 0.06                    # rho = 6 px, L = 40 px
    cam = camera(f, f, 0.0, 0.0, DOWN, [0.0, 0.0, h])
    x = torch.tensor([px_to_world(20.3, 30.2, h, f, 0, 0), px_to_world(60.3, 30.2, h, f, 0, 0)], dtype=torch.float64)
    o = render(x, cam, 64, 80, 0.02, r)
    area = 2 * 6.0 * 40.0 + math.pi * 36.0
    assert float(o.sum()) == pytest.approx(area, rel=0.02)


def test_loss_of_an_empty_mask_is_the_mean_square_occupancy():
    f, h, tau, r = 100.0, 1.0, 0.5, 0.02
    cam = camera(f, f, 0.0, 0.0, DOWN, [0.0, 0.0, h])
    x = torch.tensor([px_to_world(5.0, 5.0, h, f, 0, 0), px_to_world(25.0, 12.0, h, f, 0, 0)], dtype=torch.float64)
    o = render(x, cam, 20, 30, tau, r)
    L = silhouette_loss(x, [cam], np.zeros((1, 20, 30)), tau, r)
    assert float(L) == pytest.approx(float((o ** 2).mean()), rel=1e-14)
    L1 = silhouette_loss(x, [cam], np.ones((1, 20, 30)), tau, r)
    assert float(L1) == pytest.approx(float(((1 - o) ** 2).mean()), rel=1e-14)
