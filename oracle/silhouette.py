"""FP64 definition of the system-identification silhouette loss (Sec. 5, "System
Identification": the pixel-wise difference between the projected simulated rope and a
camera's binary mask, back-propagated through the simulation to the material).

Test infrastructure: only tests/ (and the benchmark's CPU baseline) import this module.

Reading (the paper projects to a binary mask, which has no gradient): a soft silhouette.
  * pinhole camera: X_cam = R x + t, u = fx X/Z + cx, v = fy Y/Z + cy; the rod radius r
    projects to rho = fx r / Z at each vertex
  * each edge is a capsule of radius rho_e = (rho_a + rho_b) / 2 around its projected segment;
    it covers the pixel centre p with sigma(-s_e(p) / tau), s_e(p) = dist(p, segment) - rho_e
  * occupancy o(p) = 1 - prod_e (1 - sigma(-s_e(p) / tau)) over the drawn edges (both
    endpoints at Z > 1e-3)
  * loss = mean over cameras and pixels of (o - mask)^2
Every pixel is evaluated against every edge; pixel (i, j) is column i, row j, centre
(i + 0.5, j + 0.5).
"""
import torch
import torch.nn.functional as Fn

__all__ = ["camera", "project", "render", "silhouette_loss"]

NEAR = 1e-3


def camera(fx, fy, cx, cy, R, t):
    """The 16 floats of one pinhole camera: fx, fy, cx, cy, R (row major), t."""
    import numpy as np
    return np.concatenate([[fx, fy, cx, cy], np.asarray(R, np.float64).reshape(9), np.asarray(t, np.float64)])


def project(x, cam, r):
    """(u, v) [N, 2], rho [N], Z [N] of the vertices x [N, 3]."""
    cam = torch.as_tensor(cam, dtype=x.dtype)
    fx, fy, cx, cy = cam[0], cam[1], cam[2], cam[3]
    R, t = cam[4:13].reshape(3, 3), cam[13:16]
    Xc = x @ R.T + t
    Z = Xc[:, 2]
    uv = torch.stack([fx * Xc[:, 0] / Z + cx, fy * Xc[:, 1] / Z + cy], 1)
    return uv, fx * r / Z, Z


def render(x, cam, H, W, tau, r, closed=False):
    """Soft silhouette o [H, W] of one rod seen by one camera."""
    uv, rho, Z = project(x, cam, r)
    n = x.shape[0]
    ne = n if closed else n - 1
    i0 = torch.arange(ne)
    i1 = (i0 + 1) % n
    a, b = uv[i0], uv[i1]
    rho_e = 0.5 * (rho[i0] + rho[i1])
    drawn = (Z[i0] > NEAR) & (Z[i1] > NEAR)
    jj, ii = torch.meshgrid(torch.arange(H), torch.arange(W), indexing="ij")
    p = torch.stack([ii.reshape(-1), jj.reshape(-1)], 1).to(x.dtype) + 0.5          # [HW, 2]
    d = b - a                                                                      # [E, 2]
    l2 = (d * d).sum(1)
    proj = ((p[:, None, :] - a[None]) * d[None]).sum(-1) / torch.where(l2 > 0, l2, torch.ones_like(l2))
    t = torch.where(l2 > 0, proj.clamp(0.0, 1.0), torch.zeros_like(proj))          # [HW, E]
    c = a[None] + t[..., None] * d[None]
    s = (p[:, None, :] - c).norm(dim=-1) - rho_e[None]
    logkeep = -Fn.softplus(-s / tau)                                               # log(1 - sigma(-s / tau))
    S = torch.where(drawn[None], logkeep, torch.zeros_like(logkeep)).sum(1)
    return (-torch.expm1(S)).reshape(H, W)


def silhouette_loss(x, cams, masks, tau, r, closed=False):
    """mean over cameras c and pixels of (render_c - masks[c])^2; masks [C, H, W] in {0, 1}."""
    C, H, W = masks.shape
    total = 0.0
    for c in range(C):
        o = render(x, cams[c], H, W, tau, r, closed)
        total = total + ((o - torch.as_tensor(masks[c], dtype=x.dtype)) ** 2).mean()
    return total / C
