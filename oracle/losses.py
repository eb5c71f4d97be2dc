"""FP64 definitions of the task losses of App. B ("Reward design"), written out plainly.

Test infrastructure: only tests/ (and the benchmark's CPU baseline) import this module.
Each function takes one rod's vertices as an [N, 3] float64 torch tensor (differentiable), so
gradients are torch.autograd of these definitions.

* target_mse   mean squared distance to per-vertex targets (the trajectory-optimisation loss)
* chamfer      symmetric Chamfer distance to a point set (Separation, Wiring-post)
* winding      winding number about a vertical post, from the signed angles the rod's
               segments subtend at the post in the xy-plane (Wrapping)
* crossing     signed crossing sum of all non-adjacent edge pairs (Unknotting's "discrete
               average crossing number"): reading: each pair contributes its exact Gauss
               double integral for straight segments, Omega / (4 pi) for each ordered pair,
               so the sum is the writhe of the polygon
* linking      the same pair integral summed across two closed polygons (their linking
               number; used to pin the pair integral, which must give an integer)
* mindist      the minimum distance from the rod's vertices to an object's centre (the
               rope-object contact terms of Gathering, Lifting and Wrapping)
* repulsion    Unknotting's self-repulsion penalty: sum over edge pairs more than k apart along
               the rod of max(0, delta - d)^2, d the distance between the two segments;
               reading: a quadratic hinge, with delta twice the rest edge length and k = 2 in the
               task (the smallest window that leaves a straight rod unpenalised)
"""
import math

import torch

from .dlo import closest_params

__all__ = ["target_mse", "chamfer", "winding", "gauss_pair", "crossing", "linking", "mindist", "repulsion"]


def target_mse(x, t):
    """(1/N) sum_i |x_i - t_i|^2."""
    return ((x - t) ** 2).sum(1).mean()


def chamfer(x, y):
    """(1/N) sum_i min_j |x_i - y_j|^2 + (1/M) sum_j min_i |x_i - y_j|^2."""
    d = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    return d.min(1).values.mean() + d.min(0).values.mean()


def winding(x, post, closed=False):
    """(1/2pi) sum over segments of the signed angle from (x_j - p) to (x_{j+1} - p) in the
    xy-plane (p the post's xy position); closed rods include the closing segment."""
    a = x[:, :2] - torch.as_tensor(post, dtype=x.dtype)[:2]
    b = torch.roll(a, -1, 0) if closed else a[1:]
    a = a if closed else a[:-1]
    cr = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
    dt = (a * b).sum(1)
    return torch.atan2(cr, dt).sum() / (2.0 * math.pi)


def _unit_cross(u, v):
    c = torch.cross(u, v, dim=-1)
    n = c.norm(dim=-1, keepdim=True)
    return c / n.clamp_min(1e-300), n[..., 0]


def gauss_pair(p1, p2, p3, p4):
    """Solid angle Omega of segment pair (p1 p2), (p3 p4): the Gauss double integral
    int int ((r_1 - r_2) . (dr_1 x dr_2)) / |r_1 - r_2|^3 over the two segments equals
    Omega (the closed form of the quadrilateral p1, p3, p2, p4 seen as four spherical
    triangles), signed by the orientation of the pair.  Zero for coplanar pairs."""
    r13, r14, r23, r24 = p3 - p1, p4 - p1, p3 - p2, p4 - p2
    n1, a1 = _unit_cross(r13, r14)
    n2, a2 = _unit_cross(r14, r24)
    n3, a3 = _unit_cross(r24, r23)
    n4, a4 = _unit_cross(r23, r13)
    s = lambda u, v: torch.asin((u * v).sum(-1).clamp(-1.0, 1.0))
    om = s(n1, n2) + s(n2, n3) + s(n3, n4) + s(n4, n1)
    sign = torch.sign((torch.cross(p4 - p3, p2 - p1, dim=-1) * r13).sum(-1))
    tiny = torch.minimum(torch.minimum(a1, a2), torch.minimum(a3, a4)) < 1e-14
    return torch.where(tiny, torch.zeros_like(om), om * sign)


def _edges(x, closed):
    n = x.shape[0]
    ne = n if closed else n - 1
    idx = torch.arange(ne)
    return idx, (idx + 1) % n, ne


def crossing(x, closed=False):
    """sum over ordered pairs (i, j) of non-adjacent edges of Omega_ij / (4 pi)."""
    i0, i1, ne = _edges(x, closed)
    a, b = torch.meshgrid(torch.arange(ne), torch.arange(ne), indexing="ij")
    sep = (a - b).abs()
    if closed:
        sep = torch.minimum(sep, ne - sep)
    keep = sep > 1
    a, b = a[keep], b[keep]
    om = gauss_pair(x[i0[a]], x[i1[a]], x[i0[b]], x[i1[b]])
    return om.sum() / (4.0 * math.pi)


def linking(xa, xb):
    """sum over edge i of closed polygon A and edge j of closed polygon B of Omega_ij / (4 pi)."""
    ia0, ia1, na = _edges(xa, True)
    ib0, ib1, nb = _edges(xb, True)
    a, b = torch.meshgrid(torch.arange(na), torch.arange(nb), indexing="ij")
    a, b = a.reshape(-1), b.reshape(-1)
    om = gauss_pair(xa[ia0[a]], xa[ia1[a]], xb[ib0[b]], xb[ib1[b]])
    return om.sum() / (4.0 * math.pi)


def mindist(x, o):
    """min_i |x_i - o|."""
    return (x - torch.as_tensor(o, dtype=x.dtype)[:3]).norm(dim=1).min()


def repulsion(x, delta, k, closed=False):
    """sum over edge pairs (a < b) whose index separation (cyclic for loops) exceeds k of
    max(0, delta - |c_a - c_b|)^2, c_a and c_b the closest points of the two segments (the
    clamped solve of closest_params, lower edge first)."""
    i0, i1, ne = _edges(x, closed)
    a, b = torch.triu_indices(ne, ne, 1)
    sep = b - a
    if closed:
        sep = torch.minimum(sep, ne - sep)
    keep = sep > k
    a, b = a[keep], b[keep]
    pa, qa, pb, qb = x[i0[a]], x[i1[a]], x[i0[b]], x[i1[b]]
    s, u = closest_params(pa, qa, pb, qb)
    d = ((pa + s[:, None] * (qa - pa)) - (pb + u[:, None] * (qb - pb))).norm(dim=1)
    return ((delta - d).clamp(min=0.0) ** 2).sum()
