"""FP64 CPU oracle of the DLO-Lab discrete-elastic-rod stepper (test infrastructure only).

Each function restates one passage of the paper (arXiv 2606.04206, "DLO-Lab"):

* rod representation, adapted frames, reference frame + twist angle: Sec. 3.1, App. A.1
* stretching / bending / twisting energies: App. A.1, eqs. for epsilon^j, U_s, (kappa b)_i,
  kappa_i, U_b, B_i, tau_i, U_t
* forces dU/dX and symplectic Euler time stepping: Sec. 3.1
* inextensibility projections (N_C iterations): App. A.1 "Inextensibility Constraint"
* bending plasticity (yield threshold, creep rate): App. A.1 "Bending Plasticity"
* loop holonomy frame initialisation: App. A.1 "Loop Topology"
* self-collision projections and friction: App. A.1 "Self-collision and Friction"
* soft SDF rigid contact, kinematic gripper vertices: Sec. 3.2 "Rigid Body"
* frame time 1e-3 s, 5 substeps: App. B.1

Where the paper is silent, ambiguous or garbled the oracle takes one stated reading; each
such place is marked "reading:" below.  Forces are the autograd gradient of the elastic
energy (the definition F = -dU/dx), never a hand-derived closed form.  Everything runs in
float64 on the CPU with plain torch ops; nothing here is blocked, fused or reordered beyond
vectorising independent elements.
"""
from __future__ import annotations

import math
import numpy as np
import torch

F64 = torch.float64
TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------- vector helpers

def dot(a, b):
    return (a * b).sum(-1)


def cross(a, b):
    return torch.linalg.cross(a, b, dim=-1)


def norm(a):
    return torch.sqrt(dot(a, a))


def safe_norm(a):
    """|a| with a zero (not NaN) derivative at a = 0, for quantities tested against zero."""
    n2 = dot(a, a)
    pos = n2 > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, n2, torch.ones_like(n2))), torch.zeros_like(n2))


def unit(a):
    return a / norm(a)[..., None]


def transport(a, b, d):
    """Parallel transport of d from unit tangent a to unit tangent b.

    The rotation about a x b that takes a onto b (Rodrigues' formula written with
    k = a x b and c = a . b, so it stays smooth when a == b)."""
    c = dot(a, b)[..., None]
    k = cross(a, b)
    return c * d + cross(k, d) + dot(k, d)[..., None] * k / (1.0 + c)


def adapt(d, t):
    """Project d onto the plane normal to t and renormalise (keeps d1 adapted, Sec. 3.1)."""
    d = d - dot(d, t)[..., None] * t
    return unit(d)


def signed_angle(u, v, axis):
    """Signed angle from u to v about axis."""
    return torch.atan2(dot(cross(u, v), axis), dot(u, v))


def wrap(a):
    """Map an angle to (-pi, pi]; its derivative is 1 almost everywhere."""
    return a - TWO_PI * torch.round(a / TWO_PI)


def hat(w):
    z = torch.zeros_like(w[..., 0])
    return torch.stack([torch.stack([z, -w[..., 2], w[..., 1]], -1),
                        torch.stack([w[..., 2], z, -w[..., 0]], -1),
                        torch.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def expmap(phi):
    """Rotation matrix exp([phi]x) (Rodrigues), with its Taylor series near zero."""
    th2 = dot(phi, phi)[..., None, None]
    small = th2 < 1e-8
    th2s = torch.where(small, torch.ones_like(th2), th2)
    th = torch.sqrt(th2s)
    A = torch.where(small, 1.0 - th2 / 6.0, torch.sin(th) / th)
    Bc = torch.where(small, 0.5 - th2 / 24.0, (1.0 - torch.cos(th)) / th2s)
    K = hat(phi)
    eye = torch.eye(3, dtype=phi.dtype).expand(K.shape)
    return eye + A * K + Bc * (K @ K)


# --------------------------------------------------------------------------- rod topology

def edges_of(x, closed: bool):
    """Edge vectors e^j = x_{j+1} - x_j (the closing edge N_e-1 -> 0 for loops)."""
    if closed:
        return torch.roll(x, -1, dims=-2) - x
    return x[..., 1:, :] - x[..., :-1, :]


def hinge_sides(q, closed: bool):
    """Edge-indexed quantity -> (value on edge i-1, value on edge i) for every hinge i.

    reading: 0-based indices; open rods have hinges at vertices 1..N_v-2, loops at every vertex."""
    if closed:
        return torch.roll(q, 1, dims=1), q
    return q[:, :-1], q[:, 1:]


def build_frames(x, closed: bool):
    """Initial adapted reference frames (App. A.1, "Loop Topology").

    d1 on edge 0 is the projection of a fixed axis (z, or x when the first edge is within
    ~25 degrees of z); later edges get it by space-parallel transport.  For loops the
    holonomy angle psi_H (the mismatch after transporting the last frame across the closing
    hinge) is spread as phi^j = -psi_H * j / N_e (0-based j) and each (d1, d2) is rotated
    by phi^j.  Returns tangents, d1 and psi_H."""
    t = unit(edges_of(x, closed))
    B, E = t.shape[:2]
    ez = torch.tensor([0.0, 0.0, 1.0], dtype=x.dtype).expand(B, 3)
    ex = torch.tensor([1.0, 0.0, 0.0], dtype=x.dtype).expand(B, 3)
    a = torch.where((t[:, 0, 2].abs() < 0.9)[:, None], ez, ex)
    d = [adapt(a, t[:, 0])]
    for j in range(1, E):
        d.append(adapt(transport(t[:, j - 1], t[:, j], d[-1]), t[:, j]))
    d1 = torch.stack(d, 1)
    psi = torch.zeros(B, dtype=x.dtype)
    if closed:
        u = adapt(transport(t[:, E - 1], t[:, 0], d1[:, E - 1]), t[:, 0])
        psi = signed_angle(d1[:, 0], u, t[:, 0])
        phi = -psi[:, None] * torch.arange(E, dtype=x.dtype)[None] / E
        d1 = torch.cos(phi)[..., None] * d1 + torch.sin(phi)[..., None] * cross(t, d1)
    return t, d1, psi


def edge_frames(x, theta, tb, d1b, closed: bool):
    """Reference frame by time-parallel transport from the stored base (tb, d1b) to the
    current tangent, and the material frame rotated from it by theta (App. A.1: material
    frame = reference frame rotated by the twist angle).

    reading: the reference frame follows the discrete-elastic-rod time-parallel transport,
    which the paper cites but does not restate."""
    e = edges_of(x, closed)
    ell = norm(e)
    t = e / ell[..., None]
    d1r = adapt(transport(tb, t, d1b), t)
    d2r = cross(t, d1r)
    c, s = torch.cos(theta)[..., None], torch.sin(theta)[..., None]
    d1 = c * d1r + s * d2r
    d2 = -s * d1r + c * d2r
    return t, ell, d1r, d1, d2


def hinge_strains(t, d1r, d1, d2, theta, mprev, closed: bool):
    """Curvature binormal, material curvature and twist at every hinge (App. A.1).

    (kappa b)_i = 2 t^{i-1} x t^i / (1 + t^{i-1} . t^i)
    kappa_i     = 1/2 sum_{j=i-1,i} ((kappa b)_i . d2^j, (kappa b)_i . d1^j)   (paper's sign)
    m_i         = theta^i - theta^{i-1} + reference twist
    reading: the reference twist is the signed angle about t^i from the space-transported
    reference d1 of edge i-1 to that of edge i, unwrapped against its previous value."""
    ta, tb_ = hinge_sides(t, closed)
    d1a, d1b_ = hinge_sides(d1, closed)
    d2a, d2b = hinge_sides(d2, closed)
    ra, rb = hinge_sides(d1r, closed)
    tha, thb = hinge_sides(theta, closed)
    kb = 2.0 * cross(ta, tb_) / (1.0 + dot(ta, tb_))[..., None]
    kappa = 0.5 * torch.stack([dot(kb, d2a + d2b), dot(kb, d1a + d1b_)], -1)
    ang = signed_angle(transport(ta, tb_, ra), rb, tb_)
    mref = mprev + wrap(ang - mprev)
    m = thb - tha + mref
    return kappa, mref, m


def elastic_energy(x, theta, tb, d1b, mprev, kbar, R, closed: bool, strands=None):
    """Total elastic energy per rod, U = U_s + U_b + U_t (App. A.1).

    U_s = 1/2 sum_j K A (|e^j|/|ebar^j| - 1)^2 |ebar^j|        (off for inextensible rods)
    U_b = 1/2 sum_i (1/lbar_i) (kappa_i - kbar_i)^T B_i (kappa_i - kbar_i), B_i = E A r^2/4 I
    U_t = 1/2 sum_i beta_i (m_i - mbar_i)^2 / lbar_i,           beta_i = G A r^2 / 2
    ``R`` holds the per-rod constants (see OracleSim._group).  ``strands``: the vertex ranges
    of an environment's DLOs (see ``strand_parts``); its energy is the sum of theirs."""
    if strands is not None:
        return sum(elastic_energy(x[:, vs], theta[:, es], tb[:, es], d1b[:, es], mprev[:, hs], kbar[:, hs],
                                  strand_constants(R, es, hs), False)
                   for vs, es, hs in strand_parts(strands))
    t, ell, d1r, d1, d2 = edge_frames(x, theta, tb, d1b, closed)
    kappa, mref, m = hinge_strains(t, d1r, d1, d2, theta, mprev, closed)
    Us = 0.5 * R["kA"][:, None] * (ell / R["ebar"] - 1.0) ** 2 * R["ebar"]
    Ub = 0.5 * R["Bm"][:, None] / R["lbar"] * ((kappa - kbar) ** 2).sum(-1)
    Ut = 0.5 * R["beta"][:, None] * (m - R["mbar"]) ** 2 / R["lbar"]
    return Us.sum(1) + Ub.sum(1) + Ut.sum(1)


# --------------------------------------------------------------------------- environments of several DLOs
#
# Several DLOs of one environment (two ropes in Separation, the ropes of Letter Art; Sec. 4)
# are stored as one record whose vertices are the DLOs' vertices back to back ("strands").
# reading: the DLOs interact only through the self-collision projection and friction of
# App. A.1, applied between segments of different strands exactly as between segments of
# one; every other term (stretching, bending, twisting, plasticity, the length projection)
# belongs to one strand.  With strands (v0, v1), edge j joins vertices j and j + 1 and hinge
# index h sits at vertex h + 1, as for a single open rod; the edge v1 - 1 between two
# strands ("break") and the hinges at its two ends are not part of the model.  A break edge
# keeps the frame it was given (tangent z, d1 = x) and its twist angle only decays under
# damping.

def strand_parts(strands):
    """(vertex slice, edge slice, hinge slice) of every strand of an open record."""
    return [(slice(v0, v1), slice(v0, v1 - 1), slice(v0, v1 - 2)) for v0, v1 in strands]


def strand_constants(R, es, hs):
    """The constants of ``elastic_energy`` restricted to one strand's edges and hinges."""
    return dict(kA=R["kA"], Bm=R["Bm"], beta=R["beta"], ebar=R["ebar"][:, es], lbar=R["lbar"][:, hs],
                mbar=R["mbar"][:, hs])


def _fill(default, parts):
    """``default`` (dim 1) with the slices of ``parts`` [(slice, values)] replaced."""
    out, pos = [], 0
    for sl, val in parts:
        if sl.start > pos:
            out.append(default[:, pos:sl.start])
        out.append(val)
        pos = sl.stop
    if pos < default.shape[1]:
        out.append(default[:, pos:])
    return torch.cat(out, 1)


def frames_of(x, theta, tb, d1b, closed: bool, strands=None):
    """``edge_frames`` of a record; a break edge keeps its stored frame (length 0)."""
    if strands is None:
        return edge_frames(x, theta, tb, d1b, closed)
    parts = [(es, edge_frames(x[:, vs], theta[:, es], tb[:, es], d1b[:, es], False))
             for vs, es, hs in strand_parts(strands)]
    dflt = (tb, torch.zeros_like(theta), d1b, d1b, cross(tb, d1b))
    return tuple(_fill(dflt[k], [(es, f[k]) for es, f in parts]) for k in range(5))


def strains_of(t, d1r, d1, d2, theta, mprev, closed: bool, strands=None):
    """``hinge_strains`` of a record; hinges at the ends of a break edge have no strain and
    keep their reference twist."""
    if strands is None:
        return hinge_strains(t, d1r, d1, d2, theta, mprev, closed)
    parts = [(hs, hinge_strains(t[:, es], d1r[:, es], d1[:, es], d2[:, es], theta[:, es], mprev[:, hs], False))
             for vs, es, hs in strand_parts(strands)]
    B, H = mprev.shape
    dflt = (torch.zeros(B, H, 2, dtype=mprev.dtype), mprev, torch.zeros_like(mprev))
    return tuple(_fill(dflt[k], [(hs, f[k]) for hs, f in parts]) for k in range(3))


def build_frames_of(x, closed: bool, strands=None):
    """Initial frames (``build_frames``) of every strand on its own; break edges get
    tangent z and d1 = x."""
    if strands is None:
        return build_frames(x, closed)
    B, N = x.shape[:2]
    tz = torch.zeros(B, N - 1, 3, dtype=x.dtype)
    tz[..., 2] = 1.0
    dx = torch.zeros(B, N - 1, 3, dtype=x.dtype)
    dx[..., 0] = 1.0
    parts = [(es, build_frames(x[:, vs], False)) for vs, es, hs in strand_parts(strands)]
    t = _fill(tz, [(es, f[0]) for es, f in parts])
    d1 = _fill(dx, [(es, f[1]) for es, f in parts])
    return t, d1, torch.zeros(B, dtype=x.dtype)


def initial_reference_twist(t, d1r, closed: bool, strands=None):
    """First reference twist of every hinge: the plain signed angle from the space-transported
    reference d1 of edge i-1 to that of edge i (0 at the hinges of a break edge)."""
    def one(t, d1r, closed):
        ra, rb = hinge_sides(d1r, closed)
        ta, tb_ = hinge_sides(t, closed)
        return signed_angle(transport(ta, tb_, ra), rb, tb_)
    if strands is None:
        return one(t, d1r, closed)
    B = t.shape[0]
    H = t.shape[1] - 1
    return _fill(torch.zeros(B, H, dtype=t.dtype), [(hs, one(t[:, es], d1r[:, es], False))
                                                     for vs, es, hs in strand_parts(strands)])


class ElasticGradient(torch.autograd.Function):
    """(dU/dx, dU/dtheta) of ``elastic_energy`` as one differentiable operation, for rollouts
    that are differentiated.

    The values are the autograd gradient of the written-out energy, as everywhere else.  The
    evaluation runs on detached copies of its inputs, so each substep's autograd call walks
    only the energy's own graph; called on inputs that carry the rollout's history it would
    walk all of that history first, and a rollout's cost would grow with the square of its
    length.  The backward applies the energy's second derivatives to the incoming cotangents
    (a double backward through the same graph), with respect to every input: positions, twist
    angles, reference frames, reference twist, rest curvature and the moduli k_s, B, beta."""

    @staticmethod
    def forward(ctx, x, th, tb, d1b, mprev, kbar, kA, Bm, beta, R, closed, strands=None):
        leaves = [a.detach().requires_grad_(True) for a in (x, th, tb, d1b, mprev, kbar, kA, Bm, beta)]
        with torch.enable_grad():
            R2 = dict(R, kA=leaves[6], Bm=leaves[7], beta=leaves[8])
            U = elastic_energy(*leaves[:6], R2, closed, strands)
            gx, gth = torch.autograd.grad(U.sum(), leaves[:2], create_graph=True, allow_unused=True)
            gx = torch.zeros_like(leaves[0]) if gx is None else gx
            gth = torch.zeros_like(leaves[1]) if gth is None else gth
        ctx.leaves, ctx.outs = leaves, (gx, gth)
        return gx.detach(), gth.detach()

    @staticmethod
    def backward(ctx, ggx, ggth):
        outs = [o for o in ctx.outs if o.requires_grad]
        cots = [c for o, c in zip(ctx.outs, (ggx, ggth)) if o.requires_grad]
        g = torch.autograd.grad(outs, ctx.leaves, cots, allow_unused=True)
        return (*g, None, None, None)


# --------------------------------------------------------------------------- contact geometry

def sdf_plane(x, n, off):
    """Signed distance to the plane n.x = off and its gradient."""
    n = n.expand(x.shape)
    return dot(x, n) - off, n


def sdf_box(x, c, hl):
    """Signed distance to an axis-aligned box (center c, half extents hl) and its gradient."""
    p = x - c
    q = p.abs() - hl
    qo = q.clamp(min=0.0)
    out_len = safe_norm(qo)
    inside = q.max(-1).values.clamp(max=0.0)
    sdf = out_len + inside
    sgn = torch.where(p >= 0, 1.0, -1.0).to(x.dtype)
    n_out = sgn * qo / torch.where(out_len > 0, out_len, torch.ones_like(out_len))[..., None]
    k = q.argmax(-1)
    n_in = sgn * torch.nn.functional.one_hot(k, 3).to(x.dtype)
    n = torch.where((out_len > 0)[..., None], n_out, n_in)
    return sdf, n


def sdf_capsule(x, a, b, rc):
    """Signed distance to the capsule of radius rc around segment ab and its gradient."""
    ab = b - a
    s = (dot(x - a, ab) / dot(ab, ab)).clamp(0.0, 1.0)
    c = a + s[..., None] * ab
    dv = x - c
    dist = safe_norm(dv)
    return dist - rc, dv / torch.where(dist > 0, dist, torch.ones_like(dist))[..., None]


def closest_params(p1, q1, p2, q2):
    """Barycentric parameters (t, u) in [0,1]^2 of the closest points of segments p1q1 and
    p2q2 (App. A.1, "Self-collision").  reading: the clamped closed-form solve for the
    closest points of two segments (Ericson, Real-Time Collision Detection, 5.1.9);
    near-parallel segments (a e - b^2 <= 1e-6 a e) take t = 0 with u clamped."""
    d1 = q1 - p1
    d2 = q2 - p2
    r = p1 - p2
    a = dot(d1, d1)
    e = dot(d2, d2)
    f = dot(d2, r)
    c = dot(d1, r)
    b = dot(d1, d2)
    den = a * e - b * b
    par = den <= 1e-6 * a * e
    s = torch.where(par, torch.zeros_like(a),
                    ((b * f - c * e) / torch.where(par, torch.ones_like(den), den)).clamp(0.0, 1.0))
    u = (b * s + f) / e
    s = torch.where(u < 0, (-c / a).clamp(0.0, 1.0), torch.where(u > 1, ((b - c) / a).clamp(0.0, 1.0), s))
    u = u.clamp(0.0, 1.0)
    return s, u


def substeps_for(dt, n_min, density, radius, K, E, G, inextensible, l_min):
    """Per-rod substep count (reading: the paper's 5 substeps per 1 ms frame are kept as the
    minimum, raised where explicit stability needs more):
    n = max(n_min, ceil(dt * omega_max)), omega_max the largest of the stretching
    2 sqrt(K/rho)/l, bending 2 r sqrt(E/rho)/l^2 and twisting 2 sqrt(G/rho)/l frequencies of
    the shortest rest edge l (a 2x margin under the symplectic-Euler limit omega h < 2)."""
    w_b = 2.0 * radius * math.sqrt(E / density) / (l_min * l_min)
    w_s = 0.0 if inextensible else 2.0 * math.sqrt(K / density) / l_min
    w_t = 2.0 * math.sqrt(G / density) / l_min
    return max(int(n_min), int(math.ceil(dt * max(w_b, w_s, w_t))))


# --------------------------------------------------------------------------- simulator

class OracleSim:
    """FP64 oracle for a batch of rods described by a workload object (see the package's
    ``inputs.Problem``: only its attributes are read).  Rods are stepped in groups of equal
    vertex count, topology and substep count."""

    GRAD_PARAMS = ("K", "E", "G", "yield_curv", "damping")

    def __init__(self, prob, params=None, dtype=F64):
        """``dtype`` is float64 for every reference result; float32 exists only to measure how
        far a float32 evaluation of the same algorithm drifts from it (conditioning)."""
        self.dtype = dtype
        self.p = prob
        B = prob.batch
        self.vo = np.concatenate([[0], np.cumsum(prob.n_verts)]).astype(np.int64)
        ne = prob.n_verts - 1 + prob.closed.astype(np.int64)
        self.eo = np.concatenate([[0], np.cumsum(ne)]).astype(np.int64)
        # material tensors; callers may pass leaf tensors to differentiate through them
        self.mat = {k: torch.as_tensor(np.asarray(getattr(prob, k), np.float64)).to(dtype) for k in self.GRAD_PARAMS}
        if params:
            self.mat.update(params)
        # strands of each record (one for a single DLO), rest lengths (0 on break edges) and
        # substep counts per record
        starts = getattr(prob, "strand_start", None)
        self.ebar, self.nsub, self.strands = [], [], []
        for b in range(B):
            n = int(prob.n_verts[b])
            st = [0] if starts is None else [0] + [i for i in range(1, n) if starts[self.vo[b] + i]]
            st.append(n)
            self.strands.append(tuple(zip(st[:-1], st[1:])))
            if len(st) > 2 and (prob.closed[b] or min(np.diff(st)) < 2):
                raise ValueError(f"record {b}: strands need an open record and >= 2 vertices each")
            xr = prob.x_rest[self.vo[b]:self.vo[b + 1]]
            e = (np.roll(xr, -1, 0) - xr) if prob.closed[b] else np.diff(xr, axis=0)
            eb = np.sqrt((e * e).sum(1))
            for v0, v1 in self.strands[b][:-1]:
                eb[v1 - 1] = 0.0
            self.ebar.append(eb)
            self.nsub.append(substeps_for(prob.dt, prob.substeps_min, float(prob.density[b]),
                                          float(prob.radius[b]), float(prob.K[b]), float(prob.E[b]),
                                          float(prob.G[b]), bool(prob.inextensible[b]), float(eb[eb > 0].min())))
        keys = {}
        for b in range(B):
            keys.setdefault((int(prob.n_verts[b]), bool(prob.closed[b]), self.nsub[b], self.strands[b]), []).append(b)
        self.groups = [self._group(np.array(ids), *k) for k, ids in sorted(keys.items())]
        self.state = None
        # branch trace: when set to a list, every branch decision of the step (rigid contact
        # active, yield, strain-limit projection active, candidate pair set) is appended to it
        # in order, so that two runs can be checked for taking the same branches
        self.trace = None

    # ------------------------------------------------------------------ static per-group data
    def _group(self, ids, N, closed, nsub, strands):
        p = self.p
        t64 = lambda a: torch.as_tensor(np.asarray(a, np.float64)).to(self.dtype)
        G = dict(ids=ids, N=N, closed=closed, nsub=nsub, E=N - 1 + int(closed), H=N if closed else N - 2,
                 strands=strands if len(strands) > 1 else None)
        # edges and hinges that belong to a strand (all of them for a single DLO), strand of each edge
        sid = np.full(G["E"], -1, np.int64)
        for k, (v0, v1) in enumerate(strands):
            sid[v0:v1 - 1] = k
        if closed:
            sid[:] = 0
        G["sid"] = torch.as_tensor(sid)
        G["ereal"] = torch.as_tensor(sid >= 0)
        hreal = np.ones(G["H"], bool)
        if not closed:
            hreal = (sid[:-1] >= 0) & (sid[1:] >= 0)
        G["hreal"] = torch.as_tensor(hreal)
        r = t64(p.radius[ids])
        rho = t64(p.density[ids])
        A = math.pi * r ** 2
        ebar = t64(np.stack([self.ebar[b] for b in ids]))
        if closed:
            lv = 0.5 * (ebar + torch.roll(ebar, 1, 1))
        else:
            z = torch.zeros_like(ebar[:, :1])
            lv = 0.5 * (torch.cat([z, ebar], 1) + torch.cat([ebar, z], 1))
        ea, eb_ = hinge_sides(ebar, closed)
        mass = rho[:, None] * A[:, None] * lv                 # reading: lumped Voronoi mass
        inertia = 0.5 * rho[:, None] * A[:, None] * ebar * r[:, None] ** 2   # reading: solid-cylinder axial inertia
        # break edges, and every edge of a rod with no twist stiffness (G = 0, the table's
        # "Twisting -"; reading O41): no twist dynamics, the twist angle keeps its value
        twist = (self.mat["G"][ids].detach() > 0)[:, None]
        inertia = torch.where(G["ereal"] & twist, inertia, torch.full_like(inertia, math.inf))
        # kinematic vertices: pinned, or grasped by a gripper (Sec. 3.2)
        kind = np.zeros((len(ids), N), np.int64)
        off = np.zeros((len(ids), N, 3))
        for i, b in enumerate(ids):
            xr = p.x_rest[self.vo[b]:self.vo[b + 1]]
            kind[i, p.pinned[self.vo[b]:self.vo[b + 1]]] = 1
            for g in range(int(p.n_grippers[b])):
                Rg, pg = p.grip_rot[b, g], p.grip_pos[b, g]
                ax = Rg[:, 2]
                a0, a1 = pg - ax * p.grip_half_len, pg + ax * p.grip_half_len
                s = np.clip((xr - a0) @ (a1 - a0) / ((a1 - a0) @ (a1 - a0)), 0, 1)
                sd = np.linalg.norm(xr - (a0 + s[:, None] * (a1 - a0)), axis=1) - p.grip_radius
                # reading: every vertex touching the capsule at grasp time, and at least the nearest
                grab = sd < p.radius[b]
                grab[np.argmin(sd)] = True
                grab &= kind[i] == 0
                kind[i, grab] = 2 + g
                off[i, grab] = (xr[grab] - pg) @ Rg
        G["kind"] = torch.as_tensor(kind)
        G["off"] = t64(off)
        w = torch.where(torch.as_tensor(kind) == 0, 1.0 / mass, torch.zeros_like(mass))
        mat = {k: v[ids] for k, v in self.mat.items()}
        R = dict(ebar=ebar, lbar=0.5 * (ea + eb_), mass=mass, w=w, inertia=inertia, r=r,
                 kA=torch.where(t64(p.inextensible[ids].astype(float)) > 0, 0.0, 1.0) * mat["K"] * A,
                 Bm=mat["E"] * A * r ** 2 / 4.0, beta=mat["G"] * A * r ** 2 / 2.0,
                 sy=mat["yield_curv"], rc=t64(p.creep_rate[ids]), cd=mat["damping"],
                 plastic=torch.as_tensor(p.plastic[ids].astype(bool)),
                 inext=torch.as_tensor(p.inextensible[ids].astype(bool)),
                 slim=t64(p.strain_limit[ids]))
        # rest curvature / rest twist (reading: open rods rest straight; loops rest as a
        # planar circle of the same length, kbar = (0, 2 tan(pi/N_e)); rest twist = the
        # twist of the initial (rest) frames, so the rest state stores no twist energy)
        xr = t64(np.stack([p.x_rest[self.vo[b]:self.vo[b + 1]] for b in ids]))
        st = G["strands"]
        t0, d10, _ = build_frames_of(xr, closed, st)
        zero = torch.zeros(len(ids), G["E"], dtype=self.dtype)
        _, _, d1r0, d1m0, d2m0 = frames_of(xr, zero, t0, d10, closed, st)
        _, mref0, m0 = strains_of(t0, d1r0, d1m0, d2m0, zero, torch.zeros(len(ids), G["H"], dtype=self.dtype),
                                  closed, st)
        R["mbar"] = m0
        kb = torch.zeros(len(ids), G["H"], 2, dtype=self.dtype)
        if closed:
            kb[..., 1] = 2.0 * math.tan(math.pi / G["E"])
        R["kbar0"] = kb
        # self-contact exclusion window (reading: edge pairs at most k apart along the rod are
        # never tested; k = max(1, ceil(2r / shortest rest edge)) is the smallest window that
        # leaves a straight rod at its rest lengths with no pair inside the contact distance 2r,
        # so edges two apart still collide and keep a hinge from folding through itself)
        R["excl"] = [max(1, int(math.ceil(2 * float(p.radius[b]) / float(self.ebar[b][self.ebar[b] > 0].min()))))
                     for b in ids]
        G["R"] = R
        G["gpos0"] = t64(p.grip_pos[ids])
        G["grot0"] = t64(p.grip_rot[ids])
        G["ngrip"] = torch.as_tensor(p.n_grippers[ids].astype(np.int64))
        # inextensibility colouring (reading: red-black Gauss-Seidel, even edges then odd;
        # loops with an odd edge count give the closing edge a third colour)
        # (reading: in an environment of several DLOs an edge's colour is the parity of its
        # index in the record, break edges are skipped)
        E = G["E"]
        ev = [j for j in range(0, E - (1 if closed and E % 2 == 1 else 0), 2) if sid[j] >= 0]
        colors = [ev, [j for j in range(1, E, 2) if sid[j] >= 0]]
        if closed and E % 2 == 1:
            colors.append([E - 1])
        G["colors"] = [torch.as_tensor(c, dtype=torch.long) for c in colors if c]
        return G

    # ------------------------------------------------------------------ state in / out
    def _split(self, arr, G, per="v"):
        off = self.vo if per == "v" else self.eo
        return torch.stack([torch.as_tensor(arr[off[b]:off[b + 1]]) if not torch.is_tensor(arr)
                            else arr[off[b]:off[b + 1]] for b in G["ids"]])

    def set_state(self, x, v, theta, omega):
        """Initial state; reference frames rebuilt from x (space-parallel + holonomy)."""
        self.state = []
        for G in self.groups:
            dt = self.dtype
            xs = self._split(x, G).to(dt)
            t, d1, _ = build_frames_of(xs, G["closed"], G["strands"])
            th = self._split(theta, G, "e").to(dt)
            S = dict(x=xs, v=self._split(v, G).to(dt), theta=th, omega=self._split(omega, G, "e").to(dt),
                     tb=t, d1b=d1, kbar=G["R"]["kbar0"].clone(), gp=G["gpos0"].clone(), gR=G["grot0"].clone())
            z = torch.zeros(len(G["ids"]), G["H"], dtype=dt)
            _, _, d1r, d1m, d2m = frames_of(xs, th, t, d1, G["closed"], G["strands"])
            # reading: the first reference twist is the plain signed angle (nothing to unwrap against)
            S["mprev"] = initial_reference_twist(t, d1r, G["closed"], G["strands"]) + z
            self.state.append(S)

    def set_full_state(self, st):
        """Load every state array (as dumped by ``get_state``), e.g. a float32 device state."""
        self.state = []
        for G in self.groups:
            ids = G["ids"]
            hv = (lambda a: a) if G["closed"] else (lambda a: a[:, 1:-1])
            S = dict(x=self._split(st["x"], G), v=self._split(st["v"], G),
                     theta=self._split(st["theta"], G, "e"), omega=self._split(st["omega"], G, "e"),
                     tb=self._split(st["tb"], G, "e"), d1b=self._split(st["d1b"], G, "e"),
                     mprev=hv(self._split(st["mprev"], G)), kbar=hv(self._split(st["kbar"], G)),
                     gp=torch.as_tensor(np.asarray(st["gp"])[ids]), gR=torch.as_tensor(np.asarray(st["gR"])[ids]))
            self.state.append({k: v.to(self.dtype) for k, v in S.items()})

    def get_state(self, as_numpy=True):
        """Concatenated state in workload order.  Hinge arrays (mprev, kbar) are indexed by
        vertex: open rods store hinge i at vertex i (vertices 0 and N-1 hold zeros)."""
        p = self.p
        V, Et, B = int(self.vo[-1]), int(self.eo[-1]), p.batch
        out = {k: [None] * B for k in ("x", "v", "theta", "omega", "tb", "d1b", "mprev", "kbar")}
        gp, gR = [None] * B, [None] * B
        for G, S in zip(self.groups, self.state):
            for i, b in enumerate(G["ids"]):
                for k in ("x", "v", "theta", "omega", "tb", "d1b"):
                    out[k][b] = S[k][i]
                if G["closed"]:
                    out["mprev"][b], out["kbar"][b] = S["mprev"][i], S["kbar"][i]
                else:
                    zm = torch.zeros(1, dtype=S["mprev"].dtype)
                    zk = torch.zeros(1, 2, dtype=S["kbar"].dtype)
                    out["mprev"][b] = torch.cat([zm, S["mprev"][i], zm])
                    out["kbar"][b] = torch.cat([zk, S["kbar"][i], zk])
                gp[b], gR[b] = S["gp"][i], S["gR"][i]
        res = {k: torch.cat(v) for k, v in out.items()}
        res["gp"], res["gR"] = torch.stack(gp), torch.stack(gR)
        if as_numpy:
            res = {k: v.detach().numpy() for k, v in res.items()}
        return res

    # ------------------------------------------------------------------ per-frame
    def step(self, actions, frames=None, diff=False):
        """Advance ``frames`` frames with per-frame gripper actions [F, B, 2, 6]."""
        act = torch.as_tensor(actions) if not torch.is_tensor(actions) else actions
        act = act.to(self.dtype)
        frames = act.shape[0] if frames is None else frames
        for gi, G in enumerate(self.groups):
            S = self.state[gi]
            for f in range(frames):
                S = self.frame(G, S, act[f, torch.as_tensor(G["ids"])], diff)
            self.state[gi] = S

    def frame(self, G, S, act, diff=False):
        pairs = self.candidates(G, S["x"]) if self.p.self_contact else None
        for s in range(G["nsub"]):
            S = self.substep(G, S, act, s, pairs, diff)
        S = dict(S)
        S["gp"] = S["gp"] + act[..., :3]
        S["gR"] = expmap(act[..., 3:]) @ S["gR"]
        return S

    # ------------------------------------------------------------------ one substep
    def substep(self, G, S, act, s, pairs=None, diff=False):
        p, R, closed = self.p, G["R"], G["closed"]
        n = G["nsub"]
        h = p.dt / n
        x, v, th, om = S["x"], S["v"], S["theta"], S["omega"]
        # A0: gripper pose interpolated over the frame (reading: linear in translation,
        # exponential map of the scaled rotation increment)
        dp, dphi = act[..., :3], act[..., 3:]
        p0 = S["gp"] + (s / n) * dp
        R0 = expmap((s / n) * dphi) @ S["gR"]
        p1 = S["gp"] + ((s + 1) / n) * dp
        R1 = expmap(((s + 1) / n) * dphi) @ S["gR"]
        # A1/A3: frames at x, then bending plasticity on the rest curvature
        st = G["strands"]
        t, ell, d1r, d1, d2 = frames_of(x, th, S["tb"], S["d1b"], closed, st)
        kappa, mref, _ = strains_of(t, d1r, d1, d2, th, S["mprev"], closed, st)
        kbar = self.plastic_update(G, kappa, S["kbar"])
        # A2: F = -dU/dx, tau = -dU/dtheta (autograd of the energy at the updated kbar)
        if diff:
            gx, gth = ElasticGradient.apply(x, th, S["tb"], S["d1b"], S["mprev"], kbar, R["kA"], R["Bm"],
                                            R["beta"], R, closed, st)
        else:
            dx = torch.zeros_like(x, requires_grad=True)
            dth = torch.zeros_like(th, requires_grad=True)
            with torch.enable_grad():
                U = elastic_energy(x + dx, th + dth, S["tb"], S["d1b"], S["mprev"], kbar, R, closed, st)
                gx, gth = torch.autograd.grad(U.sum(), [dx, dth])
        # A4/A5: gravity, damping, symplectic Euler velocity update
        grav = torch.tensor([0.0, 0.0, -p.gravity], dtype=self.dtype)
        w = R["w"][..., None]
        free = (G["kind"] == 0)[..., None]
        acc = -w * gx + grav - R["cd"][:, None, None] * v
        v1 = torch.where(free, v + h * acc, v)
        om1 = om + h * (-gth / R["inertia"] - R["cd"][:, None] * om)
        # A6: soft SDF rigid contact on the velocity at x
        v2 = self.rigid_contact(G, x, v1, p0, R0, dp / p.dt, dphi / p.dt)
        # A5: positions; kinematic vertices follow the gripper, pinned stay
        xs = x + h * v2
        xs = torch.where((G["kind"] == 1)[..., None], x, xs)
        for g in range(2):
            tgt = p1[:, g, None, :] + (R1[:, g, None] @ G["off"][..., None]).squeeze(-1)
            xs = torch.where((G["kind"] == 2 + g)[..., None], tgt, xs)
        th1 = th + h * om1
        # A8: N_C iterations of inextensibility / strain-limit sweeps, then self-contact
        fr = None
        need_pbd = bool(R["inext"].any() or (R["slim"] > 0).any() or pairs is not None)
        if need_pbd:
            for it in range(p.n_iter):
                for col in G["colors"]:
                    xs = self.inext_sweep(G, xs, col)
                if pairs is not None:
                    xs, info = self.contact_sweep(G, xs, pairs)
                    if it == 0:
                        fr = info
        # A9: velocity from positions, then self-contact friction
        v3 = (xs - x) / h
        if fr is not None:
            v3 = self.self_friction(G, v3, fr, h)
        return dict(x=xs, v=v3, theta=th1, omega=om1, tb=t, d1b=d1r, mprev=mref, kbar=kbar,
                    gp=S["gp"], gR=S["gR"])

    # ------------------------------------------------------------------ phases
    def plastic_update(self, G, kappa, kbar):
        """App. A.1 "Bending Plasticity": if |kappa_el| > yield, kbar += r_c (|k_el|-y)/|k_el| k_el.
        reading: kappa is an integrated (dimensionless) curvature, so the yield curvature
        sigma_y (1/m) is compared as sigma_y * lbar_i."""
        R = G["R"]
        if not bool(R["plastic"].any()):
            return kbar
        kel = kappa - kbar
        nk = safe_norm(kel)
        thr = R["sy"][:, None] * R["lbar"]
        y = R["plastic"][:, None] & (nk > thr) & G["hreal"][None]
        self._note("yield", y)
        nks = torch.where(y, nk, torch.ones_like(nk))
        upd = kbar + (R["rc"][:, None] * (nk - thr) / nks)[..., None] * kel
        return torch.where(y[..., None], upd, kbar)

    def rigid_contact(self, G, x, v, p0, R0, vp, wv):
        """Sec. 3.2 soft coupling: d = r - SDF(p), f = min(exp(d/eps_s), 1); where f > 0.1 the
        relative velocity is split along the SDF gradient, restitution acts on the normal part
        and Coulomb friction on the tangential part.
        reading: samples are the vertices; eps_s = 0.5 r; the response is blended as
        v <- v + f (v_rel' - v_rel); primitives act one after another in the order planes,
        boxes, gripper 0, gripper 1; kinematic vertices are skipped."""
        p, R = self.p, G["R"]
        r = R["r"][:, None]
        free = G["kind"] == 0

        def respond(v, sdf, nrm, vrig, mask):
            d = r - sdf
            f = torch.exp(d / (p.eps_soft * r)).clamp(max=1.0)
            act = (f > 0.1) & free & mask
            self._note("rigid", act)
            nrm = torch.where(act[..., None], nrm, torch.zeros_like(nrm))
            vr = v - vrig
            vn = dot(vr, nrm)
            vt = vr - vn[..., None] * nrm
            vn2 = torch.maximum(vn, -p.restitution * vn)
            dvn = vn2 - vn
            vtn = safe_norm(vt)
            ok = vtn > 1e-12
            sc = torch.where(ok, (1.0 - p.mu_rigid * dvn / torch.where(ok, vtn, torch.ones_like(vtn))).clamp(min=0.0),
                             torch.ones_like(vtn))
            vr2 = vn2[..., None] * nrm + sc[..., None] * vt
            return torch.where(act[..., None], v + f[..., None] * (vr2 - vr), v)

        acc = G.get("react")

        def track(slot, v_before, v_after):
            # impulse m (v' - v) the response gave each vertex (Sec. 3.2: the rigid body gets
            # the opposite); a diagnostic, kept out of any autograd graph
            if acc is not None:
                acc[:, :, slot] += (R["mass"][..., None] * (v_after - v_before)).detach()
            return v_after

        zero = torch.zeros_like(v)
        allm = torch.ones_like(free)
        for pl in p.planes:
            n = torch.as_tensor(pl[:3], dtype=self.dtype)
            sdf, nrm = sdf_plane(x, n, float(pl[3]))
            v = track(0, v, respond(v, sdf, nrm, zero, allm))
        for bx in p.boxes:
            sdf, nrm = sdf_box(x, torch.as_tensor(bx[:3], dtype=self.dtype), torch.as_tensor(bx[3:], dtype=self.dtype))
            v = track(1, v, respond(v, sdf, nrm, zero, allm))
        for g in range(2):
            on = (G["ngrip"] > g)
            if not bool(on.any()):
                continue
            ax = R0[:, g, :, 2]
            a = p0[:, g] - ax * p.grip_half_len
            b = p0[:, g] + ax * p.grip_half_len
            sdf, nrm = sdf_capsule(x, a[:, None], b[:, None], p.grip_radius)
            vrig = vp[:, g, None] + cross(wv[:, g, None].expand(x.shape), x - p0[:, g, None])
            v = track(2 + g, v, respond(v, sdf, nrm, vrig, on[:, None].expand(free.shape)))
        return v

    def inext_sweep(self, G, xs, col):
        """One colour of the inextensibility projection (App. A.1):
        C = |x_{j+1} - x_j| - |ebar^j|, lambda = C/(w_j + w_{j+1}),
        dx_j = lambda w_j t^j, dx_{j+1} = -lambda w_{j+1} t^j.
        reading: a '20 % stretchable' rod projects only edges outside [0.8, 1.2] |ebar| back to
        the violated bound; inextensible rods project every edge to |ebar|."""
        R = G["R"]
        j0 = col
        j1 = (col + 1) % G["N"]
        xa, xb = xs[:, j0], xs[:, j1]
        e = xb - xa
        ell = norm(e)
        t = e / ell[..., None]
        eb = R["ebar"][:, col]
        sl = R["slim"][:, None]
        hi, lo = (1.0 + sl) * eb, (1.0 - sl) * eb
        inext = R["inext"][:, None].expand(ell.shape)
        lim = (sl > 0) & ~inext
        target = torch.where(inext, eb, torch.where(ell > hi, hi, lo))
        active = inext | (lim & ((ell > hi) | (ell < lo)))
        wa, wb = R["w"][:, j0], R["w"][:, j1]
        ws = wa + wb
        active = active & (ws > 0)
        self._note("length", active)
        lam = torch.where(active, (ell - target) / torch.where(active, ws, torch.ones_like(ws)), torch.zeros_like(ws))
        da = (lam * wa)[..., None] * t
        db = -(lam * wb)[..., None] * t
        delta = torch.zeros_like(xs).index_add(1, j0, da).index_add(1, j1, db)
        return xs + delta

    def candidates(self, G, x):
        """Self-contact candidate pairs for one frame, per rod: edge pairs (a < b) outside the
        exclusion window whose segments are closer than 2r + margin at the frame start.  In an
        environment of several DLOs the window applies within a strand only, and break edges
        are no segments.
        reading: the paper does not describe its broad phase; the candidate set is defined
        here by this distance test (any exact broad phase returns the same set)."""
        out = []
        closed, E, N = G["closed"], G["E"], G["N"]
        ia, ib = torch.triu_indices(E, E, offset=1)
        sep = ib - ia
        if closed:
            sep = torch.minimum(sep, E - sep)
        # edges of two different strands (DLOs of one environment) are never excluded
        sid = G["sid"]
        real = (sid[ia] >= 0) & (sid[ib] >= 0)
        other = sid[ia] != sid[ib]
        for i, b in enumerate(G["ids"]):
            k = G["R"]["excl"][i]
            keep = real & ((sep > k) | other)
            a, c = ia[keep], ib[keep]
            xb = x[i].detach()
            s, u = closest_params(xb[a], xb[(a + 1) % N], xb[c], xb[(c + 1) % N])
            ca = xb[a] + s[:, None] * (xb[(a + 1) % N] - xb[a])
            cb = xb[c] + u[:, None] * (xb[(c + 1) % N] - xb[c])
            rr = float(self.p.radius[b])
            near = norm(ca - cb) < 2 * rr + self.p.contact_margin * rr
            out.append(torch.stack([a[near], c[near]], 1))
            self._note("pairs", out[-1])
        return out

    def contact_sweep(self, G, xs, pairs):
        """One Jacobi sweep of the self-collision projection (App. A.1):
        d = (r_a + r_b) - |c_a - c_b|; if d > 0, dx_i = d w_i (1-t) n / W with
        W = w_i(1-t)^2 + w_{i+1} t^2 + w_j(1-u)^2 + w_{j+1} u^2, n = (c_a - c_b)/|c_a - c_b|,
        and the b side moved by -d w_j (1-u) n / W, -d w_{j+1} u n / W.
        reading: all pairs read the same positions and their corrections are summed (Jacobi)."""
        N, R = G["N"], G["R"]
        outs, infos = [], []
        for i in range(xs.shape[0]):
            P = pairs[i]
            xi = xs[i]
            if P.shape[0] == 0:
                outs.append(xi)
                infos.append(None)
                continue
            a0, c0 = P[:, 0], P[:, 1]
            a1, c1 = (a0 + 1) % N, (c0 + 1) % N
            s, u = closest_params(xi[a0], xi[a1], xi[c0], xi[c1])
            ca = xi[a0] + s[:, None] * (xi[a1] - xi[a0])
            cb = xi[c0] + u[:, None] * (xi[c1] - xi[c0])
            dv = ca - cb
            dist = safe_norm(dv)
            d = 2 * R["r"][i] - dist
            w = R["w"][i]
            W = w[a0] * (1 - s) ** 2 + w[a1] * s ** 2 + w[c0] * (1 - u) ** 2 + w[c1] * u ** 2
            act = (d > 0) & (dist > 1e-12) & (W > 0)
            nrm = dv / torch.where(act, dist, torch.ones_like(dist))[:, None]
            k = torch.where(act, d / torch.where(act, W, torch.ones_like(W)), torch.zeros_like(W))
            delta = torch.zeros_like(xi)
            delta = delta.index_add(0, a0, (k * w[a0] * (1 - s))[:, None] * nrm)
            delta = delta.index_add(0, a1, (k * w[a1] * s)[:, None] * nrm)
            delta = delta.index_add(0, c0, -(k * w[c0] * (1 - u))[:, None] * nrm)
            delta = delta.index_add(0, c1, -(k * w[c1] * u)[:, None] * nrm)
            outs.append(xi + delta)
            infos.append(dict(a0=a0, a1=a1, c0=c0, c1=c1, s=s, u=u, n=nrm, d=d, W=W, act=act))
        return torch.stack(outs), infos

    def self_friction(self, G, v, infos, h):
        """Velocity-level Coulomb friction on the pairs in contact at the first projection
        (App. A.1).  reading: the normal velocity change is taken as d/h, so the relative
        tangential velocity at the contact is reduced by min(1, mu d / (h |v_t|)); the change
        is spread over the four vertices with the same inverse-mass and barycentric weights
        as the position correction (momentum is conserved)."""
        R = G["R"]
        outs = []
        for i in range(v.shape[0]):
            I = infos[i]
            vi = v[i]
            if I is None:
                outs.append(vi)
                continue
            s, u, nrm, w = I["s"], I["u"], I["n"], R["w"][i]
            vrel = ((1 - s)[:, None] * vi[I["a0"]] + s[:, None] * vi[I["a1"]]
                    - (1 - u)[:, None] * vi[I["c0"]] - u[:, None] * vi[I["c1"]])
            vt = vrel - dot(vrel, nrm)[:, None] * nrm
            vtn = safe_norm(vt)
            act = I["act"] & (vtn > 1e-12)
            vts = torch.where(act, vtn, torch.ones_like(vtn))
            coef = torch.where(act, torch.clamp(self.p.mu_self * I["d"] / (h * vts), max=1.0), torch.zeros_like(vtn))
            Ws = torch.where(act, I["W"], torch.ones_like(I["W"]))
            dv = -(coef / Ws)[:, None] * vt
            delta = torch.zeros_like(vi)
            delta = delta.index_add(0, I["a0"], (w[I["a0"]] * (1 - s))[:, None] * dv)
            delta = delta.index_add(0, I["a1"], (w[I["a1"]] * s)[:, None] * dv)
            delta = delta.index_add(0, I["c0"], -(w[I["c0"]] * (1 - u))[:, None] * dv)
            delta = delta.index_add(0, I["c1"], -(w[I["c1"]] * u)[:, None] * dv)
            outs.append(vi + delta)
        return torch.stack(outs)

    # ------------------------------------------------------------------ diagnostics
    def _note(self, kind, mask):
        if self.trace is not None:
            self.trace.append((kind, mask.detach().numpy().copy()))

    def track_reaction(self):
        """Start (or restart) accumulating the rigid-contact impulses per vertex in four slots:
        planes, boxes, gripper 0, gripper 1."""
        for G in self.groups:
            G["react"] = torch.zeros(len(G["ids"]), G["N"], 4, 3, dtype=self.dtype)

    def reaction(self):
        """(per rod [B, 4, 3], per vertex [V, 4, 3]) impulses accumulated since track_reaction."""
        B, V = self.p.batch, int(self.vo[-1])
        per_v = np.zeros((V, 4, 3))
        for G in self.groups:
            for i, b in enumerate(G["ids"]):
                per_v[self.vo[b]:self.vo[b + 1]] = G["react"][i].numpy()
        per_rod = np.stack([per_v[self.vo[b]:self.vo[b + 1]].sum(0) for b in range(B)])
        return per_rod, per_v

    def energies(self):
        """Per-rod (kinetic incl. twist, elastic, gravitational) energies of the current state."""
        out = np.zeros((self.p.batch, 3))
        for G, S in zip(self.groups, self.state):
            R = G["R"]
            U = elastic_energy(S["x"], S["theta"], S["tb"], S["d1b"], S["mprev"], S["kbar"], R, G["closed"],
                               G["strands"])
            Iw = torch.where(torch.isfinite(R["inertia"]), R["inertia"] * S["omega"] ** 2, torch.zeros_like(S["omega"]))
            ke = 0.5 * (R["mass"] * dot(S["v"], S["v"])).sum(1) + 0.5 * Iw.sum(1)
            pe = (R["mass"] * S["x"][..., 2]).sum(1) * self.p.gravity
            out[G["ids"]] = torch.stack([ke, U, pe], 1).detach().numpy()
        return out

    def momentum(self):
        """Total linear momentum per rod."""
        out = np.zeros((self.p.batch, 3))
        for G, S in zip(self.groups, self.state):
            out[G["ids"]] = (G["R"]["mass"][..., None] * S["v"]).sum(1).detach().numpy()
        return out

    def rod_constants(self):
        """Per-rod static values (substeps, masses, inverse masses, kinematic kinds), workload order."""
        B = self.p.batch
        res = dict(nsub=np.array(self.nsub), mass=[None] * B, w=[None] * B, kind=[None] * B)
        for G in self.groups:
            for i, b in enumerate(G["ids"]):
                res["mass"][b] = G["R"]["mass"][i].numpy()
                res["w"][b] = G["R"]["w"][i].numpy()
                res["kind"][b] = G["kind"][i].numpy()
        for k in ("mass", "w", "kind"):
            res[k] = np.concatenate(res[k])
        return res
