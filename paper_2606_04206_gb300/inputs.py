"""Seeded synthetic workloads for the batched rod stepper.

This module only draws inputs: rod shapes, material parameters taken from the
paper's parameter table (Appendix B, Table "sim_params"), gripper poses and
per-frame gripper actions.  It holds none of the simulator's arithmetic
(no energies, frames, masses, substep counts or contact rules), so that the CPU
oracle and the CUDA path can both be fed from it without sharing method code.

Every floating-point value is rounded to float32 and stored as float64, so the
FP64 oracle and the FP32 device path start from bit-identical inputs.

Workloads (seeds are ``numpy.random.default_rng(config_index*1000 + repeat)``):

* ``plain``      1 rod, 32 vertices, 1 m straight along +x at z=1, vertex 0
                 pinned, K=E=1e6 Pa, G=4e5 Pa, no contact, 200 frames.
* ``batching``   1024 rods, 16..256 vertices, 0.3..2 m, E log-uniform in
                 [1e4, 1e8] Pa (K=E, G=0.4E), plastic (yield 1..20 1/m),
                 random smooth curves resting on a table (the ground plane),
                 two capsule grippers with smooth random 6-DoF trajectories,
                 1000 frames.
* ``diff``       256 rods x 64 vertices on the table, half elastic rope
                 (Unknotting row), half plastic wire (Letter-Art row), 500
                 frames, checkpoints every 50, seeded smooth target curves.
* ``selfcontact``4096 closed bands x 200 vertices (trefoil-like knots, 1 m
                 circumference), half inextensible, half 20 % strain-limited,
                 ground + box obstacle, self-contact, 300 frames.
* ``trajopt``    4096 rods x 128 vertices (1 m, radius 2 mm) resting on the
                 table, one third each inextensible cable (Wiring-post row),
                 elastic rope (Unknotting row), plastic wire (Letter-Art row),
                 grasped at 1/4 and 3/4 of their length by two grippers with
                 smooth random 6-DoF trajectories, 2000 frames.
* ``separation`` 4096 environments of the Separation task: two tangled ropes
                 of 30 vertices (inextensible, E=5e3 Pa, G=1e3 Pa), 0.6 m,
                 stored as one record of two strands, one gripper on each,
                 pulled apart and lifted along smooth random trajectories,
                 self-contact (which couples the ropes), 2000 frames.
* ``cmaes``      one CMA-ES generation of Unknotting: 400 copies of one knotted
                 rope (128 vertices, opened trefoil-family curve on the table,
                 Unknotting row), mean gripper trajectory plus per-candidate
                 smooth perturbations of 5e-2 m / rad, self-contact, 2000 frames,
                 forward only, scored on the device.

The open rods of batching, diff and trajopt are smooth curves whose unit tangent is a
low-frequency random Fourier series (bending radius >= 2 cm), lying nearly horizontal
just above the ground plane, as the rods of the paper's manipulation tasks start out on
the table.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import numpy as np

__all__ = ["Problem", "plain", "batching", "diff", "selfcontact", "trajopt", "cmaes", "separation",
           "small_case", "custom", "f32"]


def f32(a):
    """Round to float32 and return float64 (bit-identical inputs for both sides)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@dataclass
class Problem:
    name: str
    n_verts: np.ndarray            # [B] int32
    closed: np.ndarray             # [B] bool
    x_rest: np.ndarray             # [V,3] rest (= initial) shape
    density: np.ndarray            # [B] kg/m^3
    radius: np.ndarray             # [B] m
    K: np.ndarray                  # [B] stretching modulus, Pa
    E: np.ndarray                  # [B] bending modulus, Pa
    G: np.ndarray                  # [B] twisting modulus, Pa (0 = no twist energy)
    inextensible: np.ndarray       # [B] bool
    strain_limit: np.ndarray       # [B] 0 = none, 0.2 = 20 %
    plastic: np.ndarray            # [B] bool
    yield_curv: np.ndarray         # [B] 1/m
    creep_rate: np.ndarray         # [B] r_c
    damping: np.ndarray            # [B] 1/s
    pinned: np.ndarray             # [V] bool
    n_grippers: np.ndarray         # [B] int (0..2)
    grip_pos: np.ndarray           # [B,2,3]
    grip_rot: np.ndarray           # [B,2,3,3] (columns = capsule frame, axis = column 2)
    actions: np.ndarray            # [F,B,2,6] per-frame (d_pos, d_rotvec) in world frame
    frames: int
    grip_radius: float = 0.01
    grip_half_len: float = 0.02
    planes: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))   # [P,4] (n, offset): n.x = offset
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))    # [Q,6] (center, half extents)
    dt: float = 1e-3
    n_iter: int = 10
    substeps_min: int = 5
    mu_self: float = 0.3
    mu_rigid: float = 0.5
    restitution: float = 0.0
    eps_soft: float = 0.5          # softness epsilon_s as a multiple of the radius
    contact_margin: float = 1.0    # self-contact candidate margin as a multiple of the radius
    self_contact: bool = False
    gravity: float = 9.81
    checkpoint_every: int = 50
    target: np.ndarray | None = None   # [V,3] loss target (diff / trajopt)
    strand_start: np.ndarray | None = None   # [V] bool: vertex begins another DLO of its environment
    x0: np.ndarray | None = None
    v0: np.ndarray | None = None
    theta0: np.ndarray | None = None
    omega0: np.ndarray | None = None

    def __post_init__(self):
        self.n_verts = np.asarray(self.n_verts, np.int32)
        self.closed = np.asarray(self.closed, bool)
        if self.strand_start is None:
            self.strand_start = np.zeros(len(self.x_rest), bool)
        self.strand_start = np.asarray(self.strand_start, bool)
        if self.x0 is None:
            self.x0 = self.x_rest.copy()
        if self.v0 is None:
            self.v0 = np.zeros_like(self.x_rest)
        ne = int(self.n_edges.sum())
        if self.theta0 is None:
            self.theta0 = np.zeros(ne)
        if self.omega0 is None:
            self.omega0 = np.zeros(ne)

    @property
    def batch(self) -> int:
        return int(self.n_verts.shape[0])

    @property
    def n_edges(self) -> np.ndarray:
        return self.n_verts - 1 + self.closed.astype(np.int32)

    @property
    def vert_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_verts)]).astype(np.int64)

    @property
    def edge_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_edges)]).astype(np.int64)

    def subset(self, rods, frames: int | None = None) -> "Problem":
        """The same workload restricted to the listed rods (and optionally fewer frames)."""
        rods = np.asarray(rods, np.int64)
        vo, eo = self.vert_off, self.edge_off
        vsel = np.concatenate([np.arange(vo[b], vo[b + 1]) for b in rods])
        esel = np.concatenate([np.arange(eo[b], eo[b + 1]) for b in rods])
        f = self.frames if frames is None else frames
        per_rod = {k: getattr(self, k)[rods] for k in (
            "n_verts", "closed", "density", "radius", "K", "E", "G", "inextensible",
            "strain_limit", "plastic", "yield_curv", "creep_rate", "damping",
            "n_grippers", "grip_pos", "grip_rot")}
        return replace(self, x_rest=self.x_rest[vsel], pinned=self.pinned[vsel],
                       strand_start=self.strand_start[vsel],
                       actions=self.actions[:f, rods], frames=f,
                       target=None if self.target is None else self.target[vsel],
                       x0=self.x0[vsel], v0=self.v0[vsel], theta0=self.theta0[esel],
                       omega0=self.omega0[esel], **per_rod)


# --------------------------------------------------------------------------- shapes

def _smooth_tangent_curve(rng, length: float, modes: int = 3, amp: float = 1.0,
                          zscale: float = 0.15, dense: int = 4096) -> np.ndarray:
    """Dense polyline of the given arc length whose unit tangent is a normalised
    low-frequency random Fourier series (a horizontal heading plus ``modes`` sine/cosine
    terms per axis, mode k at amplitude amp/k, the vertical terms scaled by ``zscale`` so
    the curve stays nearly horizontal).  Curvature stays bounded because the tangent field
    has no high-frequency content; there are no cusps."""
    s = np.linspace(0.0, 1.0, dense)
    d = np.append(rng.normal(size=2), 0.0)
    d /= np.linalg.norm(d)
    tan = np.tile(d, (dense, 1))
    scale = np.array([1.0, 1.0, zscale])
    for k in range(1, modes + 1):
        a = rng.uniform(-1.0, 1.0, (2, 3)) * scale * amp / k
        tan = tan + np.sin(2 * np.pi * k * s)[:, None] * a[0] + np.cos(2 * np.pi * k * s)[:, None] * a[1]
    tan /= np.maximum(np.linalg.norm(tan, axis=1), 1e-9)[:, None]
    step = 0.5 * (tan[1:] + tan[:-1]) * (length / (dense - 1))
    return np.concatenate([np.zeros((1, 3)), np.cumsum(step, axis=0)])


def _max_curvature(x: np.ndarray) -> float:
    """Largest discrete curvature (turning angle / edge length) of an open polyline."""
    e = np.diff(x, axis=0)
    ln = np.linalg.norm(e, axis=1)
    t = e / ln[:, None]
    ang = np.arccos(np.clip((t[:-1] * t[1:]).sum(1), -1.0, 1.0))
    return float((ang / (0.5 * (ln[:-1] + ln[1:]))).max()) if len(ang) else 0.0


def _resample(poly: np.ndarray, n: int, closed: bool = False) -> np.ndarray:
    """Points equally spaced in arc length along a polyline."""
    if closed:
        poly = np.concatenate([poly, poly[:1]])
    seg = np.linalg.norm(np.diff(poly, axis=0), axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    m = n if closed else n - 1
    q = np.linspace(0.0, s[-1], m + 1)[: n]
    return np.stack([np.interp(q, s, poly[:, k]) for k in range(3)], axis=1)


def _length(x: np.ndarray, closed: bool = False) -> float:
    d = np.diff(np.concatenate([x, x[:1]]) if closed else x, axis=0)
    return float(np.linalg.norm(d, axis=1).sum())


def _too_close(x: np.ndarray, min_dist: float, skip: int, closed: bool) -> bool:
    n = len(x)
    d = np.linalg.norm(x[:, None] - x[None], axis=2)
    i, j = np.triu_indices(n, k=skip + 1)
    if closed:
        keep = np.minimum(j - i, n - (j - i)) > skip
        i, j = i[keep], j[keep]
    return bool(len(i) and d[i, j].min() < min_dist)


def _spline_rod(rng, n: int, length: float, radius: float, z_min: float = 0.005,
                box=((-0.25, 0.25), (-0.25, 0.25)), max_curv: float = 50.0) -> np.ndarray:
    """A random smooth open 3D curve of n vertices and the given length lying on a table:
    nearly horizontal (a few cm of vertical undulation), its lowest vertex at ``z_min``
    above the ground plane z = 0 and its centroid uniform in ``box`` (x, y); redrawn until
    its bending radius stays above 1/max_curv everywhere and no two non-neighbouring
    vertices are closer than 4r."""
    amp = min(1.0, length)
    for _ in range(200):
        x = _resample(_smooth_tangent_curve(rng, length, amp=amp), n)
        c = np.array([rng.uniform(lo, hi) for lo, hi in box])
        x[:, :2] += c - x[:, :2].mean(0)
        x[:, 2] += z_min - x[:, 2].min()
        skip = max(2, int(np.ceil(4 * radius * (n - 1) / length)) + 1)
        if _max_curvature(x) <= max_curv and not _too_close(x, 4 * radius, skip, False):
            return x
    raise RuntimeError("could not draw a smooth non-self-intersecting rod")


def _knot_band(rng, n: int, circumference: float, radius: float, z_min: float) -> np.ndarray:
    s = np.linspace(0, 2 * np.pi, 2048, endpoint=False)
    for _ in range(200):
        sc = rng.uniform(0.8, 1.2, 3)
        base = np.stack([np.sin(s) + 2 * np.sin(2 * s), np.cos(s) - 2 * np.cos(2 * s),
                         -np.sin(3 * s)], axis=1) * sc
        # random rotation from a random unit quaternion
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, a, b, c = q
        R = np.array([[1 - 2 * (b * b + c * c), 2 * (a * b - c * w), 2 * (a * c + b * w)],
                      [2 * (a * b + c * w), 1 - 2 * (a * a + c * c), 2 * (b * c - a * w)],
                      [2 * (a * c - b * w), 2 * (b * c + a * w), 1 - 2 * (a * a + b * b)]])
        poly = base @ R.T
        poly *= circumference / _length(poly, True)
        # smooth noise of at most ~5 mm
        noise = np.zeros_like(poly)
        for k in range(1, 4):
            amp = rng.uniform(-1, 1, (2, 3)) * 0.005 / 3
            noise += np.sin(k * s)[:, None] * amp[0] + np.cos(k * s)[:, None] * amp[1]
        poly = poly + noise
        x = _resample(poly, n, closed=True)
        x *= circumference / _length(x, True)
        x = _resample(x, n, closed=True)
        x -= x.mean(0)
        x[:, 2] += z_min - x[:, 2].min()
        if not _too_close(x, 4 * radius, 3, True):
            return x
    raise RuntimeError("could not draw a knot band")


def _gripper_frame(t: np.ndarray) -> np.ndarray:
    """Capsule frame whose axis (column 2) is perpendicular to the rod tangent t."""
    up = np.array([0.0, 0.0, 1.0])
    ax = np.cross(t, up)
    if np.linalg.norm(ax) < 0.1:
        ax = np.cross(t, np.array([1.0, 0.0, 0.0]))
    ax /= np.linalg.norm(ax)
    c0 = t / np.linalg.norm(t)
    c0 = c0 - ax * (c0 @ ax)
    c0 /= np.linalg.norm(c0)
    c1 = np.cross(ax, c0)
    return np.stack([c0, c1, ax], axis=1)


def _smooth_actions(rng, frames: int, batch: int, dt: float, amp_pos: float = 0.05,
                    amp_rot: float = 0.3, fmin: float = 0.2, fmax: float = 2.0) -> np.ndarray:
    """Per-frame deltas of pose trajectories that are sums of 3 sinusoids per DoF."""
    t = np.arange(frames + 1) * dt
    freq = rng.uniform(fmin, fmax, (batch, 2, 6, 3))
    phase = rng.uniform(0, 2 * np.pi, (batch, 2, 6, 3))
    amp = rng.uniform(0, 1, (batch, 2, 6, 3)) / 3.0
    amp[..., :3, :] *= amp_pos
    amp[..., 3:, :] *= amp_rot
    traj = np.zeros((frames + 1, batch, 2, 6))
    for k in range(3):
        arg = 2 * np.pi * freq[None, ..., k] * t[:, None, None, None] + phase[None, ..., k]
        traj += amp[None, ..., k] * (np.sin(arg) - np.sin(phase[None, ..., k]))
    return np.diff(traj, axis=0)


def _grippers_for(rods_x, fractions=(0.25, 0.75)):
    B = len(rods_x)
    pos = np.zeros((B, 2, 3))
    rot = np.tile(np.eye(3), (B, 2, 1, 1))
    for b, x in enumerate(rods_x):
        n = len(x)
        for g, fr in enumerate(fractions):
            k = int(round(fr * (n - 1)))
            pos[b, g] = x[k]
            t = x[min(k + 1, n - 1)] - x[max(k - 1, 0)]
            rot[b, g] = _gripper_frame(t)
    return pos, rot


def _assemble(name, rods_x, closed, mats, frames, actions, n_grip, grip_pos, grip_rot,
              pinned=None, **opts) -> Problem:
    B = len(rods_x)
    x = np.concatenate(rods_x)
    if pinned is None:
        pinned = np.zeros(len(x), bool)
    full = dict(density=1000.0, radius=0.002, K=0.0, E=0.0, G=0.0, inextensible=False,
                strain_limit=0.0, plastic=False, yield_curv=0.0, creep_rate=1.0, damping=1.0)
    full.update(mats)
    m = {}
    for k, v in full.items():
        a = np.broadcast_to(np.asarray(v), (B,)).copy()
        m[k] = a.astype(bool) if k in ("inextensible", "plastic") else f32(a)
    return Problem(name=name, n_verts=np.array([len(r) for r in rods_x]), closed=np.asarray(closed, bool),
                   x_rest=f32(x), pinned=pinned, n_grippers=np.asarray(n_grip, np.int32),
                   grip_pos=f32(grip_pos), grip_rot=f32(grip_rot), actions=f32(actions),
                   frames=frames, **m, **opts)


# --------------------------------------------------------------------------- workloads

def plain(frames: int = 200) -> Problem:
    """1 rod, 32 vertices, horizontal, vertex 0 pinned, released under gravity."""
    n = 32
    x = np.zeros((n, 3))
    x[:, 0] = np.linspace(0.0, 1.0, n)
    x[:, 2] = 1.0
    pinned = np.zeros(n, bool)
    pinned[0] = True
    return _assemble("plain", [x], [False],
                     dict(K=1e6, E=1e6, G=4e5, damping=0.0), frames,
                     np.zeros((frames, 1, 2, 6)), [0], np.zeros((1, 2, 3)),
                     np.tile(np.eye(3), (1, 2, 1, 1)), pinned=pinned)


def batching(n_rods: int = 1024, frames: int = 1000, seed: int = 1000,
             vmin: int = 16, vmax: int = 256) -> Problem:
    rng = np.random.default_rng(seed)
    nv = rng.integers(vmin, vmax + 1, n_rods)
    L = rng.uniform(0.3, 2.0, n_rods)
    E = np.exp(rng.uniform(np.log(1e4), np.log(1e8), n_rods))
    sy = rng.uniform(1.0, 20.0, n_rods)
    rods = [_spline_rod(rng, int(nv[b]), float(L[b]), 0.002) for b in range(n_rods)]
    gp, gr = _grippers_for(rods)
    acts = _smooth_actions(rng, frames, n_rods, 1e-3)
    return _assemble("batching", rods, np.zeros(n_rods, bool),
                     dict(K=E, E=E, G=0.4 * E, plastic=True, yield_curv=sy, creep_rate=1.0),
                     frames, acts, np.full(n_rods, 2), gp, gr,
                     planes=np.array([[0.0, 0.0, 1.0, 0.0]]))


def diff(n_rods: int = 256, frames: int = 500, seed: int = 2000, n: int = 64) -> Problem:
    rng = np.random.default_rng(seed)
    rods = [_spline_rod(rng, n, 1.0, 0.002) for _ in range(n_rods)]
    plastic = np.arange(n_rods) >= n_rods // 2
    sy = np.where(plastic, rng.uniform(1.0, 20.0, n_rods), 0.0)
    gp, gr = _grippers_for(rods)
    acts = _smooth_actions(rng, frames, n_rods, 1e-3)
    target = np.concatenate([_spline_rod(rng, n, 1.0, 0.002) for _ in range(n_rods)])
    return _assemble("diff", rods, np.zeros(n_rods, bool),
                     dict(K=1e5, E=1e4, G=0.0, plastic=plastic, yield_curv=sy),
                     frames, acts, np.full(n_rods, 2), gp, gr,
                     planes=np.array([[0.0, 0.0, 1.0, 0.0]]), target=f32(target),
                     checkpoint_every=50)


def selfcontact(n_rods: int = 4096, frames: int = 300, seed: int = 3000, n: int = 200) -> Problem:
    rng = np.random.default_rng(seed)
    rods = [_knot_band(rng, n, 1.0, 0.002, z_min=0.13) for _ in range(n_rods)]
    inext = np.arange(n_rods) % 2 == 0
    return _assemble("selfcontact", rods, np.ones(n_rods, bool),
                     dict(K=np.where(inext, 0.0, 1e5), E=1e4, G=1e3, inextensible=inext,
                          strain_limit=np.where(inext, 0.0, 0.2)),
                     frames, np.zeros((frames, n_rods, 2, 6)), np.zeros(n_rods),
                     np.zeros((n_rods, 2, 3)), np.tile(np.eye(3), (n_rods, 2, 1, 1)),
                     planes=np.array([[0.0, 0.0, 1.0, 0.0]]),
                     boxes=np.array([[0.0, 0.0, 0.05, 0.15, 0.15, 0.05]]),
                     self_contact=True)


def trajopt(n_rods: int = 4096, frames: int = 2000, seed: int = 4000, n: int = 128,
            self_contact: bool = False) -> Problem:
    rng = np.random.default_rng(seed)
    rods = [_spline_rod(rng, n, 1.0, 0.002) for _ in range(n_rods)]
    kind = np.arange(n_rods) % 3          # 0 cable, 1 rope, 2 wire
    gp, gr = _grippers_for(rods)
    acts = _smooth_actions(rng, frames, n_rods, 1e-3)
    target = np.concatenate([_spline_rod(rng, n, 1.0, 0.002) for _ in range(n_rods)])
    return _assemble("trajopt", rods, np.zeros(n_rods, bool),
                     dict(K=np.where(kind == 0, 0.0, 1e5), E=1e4,
                          G=np.where(kind == 0, 1e3, 0.0), inextensible=kind == 0,
                          plastic=kind == 2, yield_curv=np.where(kind == 2, 5.0, 0.0)),
                     frames, acts, np.full(n_rods, 2), gp, gr,
                     planes=np.array([[0.0, 0.0, 1.0, 0.0]]), target=f32(target),
                     self_contact=self_contact)


def cmaes(pop: int = 400, frames: int = 2000, seed: int = 5000, n: int = 128, sigma: float = 5e-2) -> Problem:
    """One CMA-ES generation of the Unknotting task: ``pop`` copies of one knotted rope (a
    trefoil-family curve of 1 m, opened, resting on the ground; Unknotting row: K = 1e5,
    E = 1e4, no twist stiffness), each with the population mean's gripper trajectory plus
    its own smooth perturbation of amplitude ``sigma`` (m and rad)."""
    rng = np.random.default_rng(seed)
    for _ in range(200):
        # a knot band of n + 3 vertices, opened by dropping three (the ends start four edges
        # apart) and flattened onto the table; the crossings keep their over/under order
        m = n + 3
        x = _knot_band(rng, m, m / (n - 1), 0.002, z_min=0.005)[:n]
        x[:, 2] *= 0.4
        x = _resample(x, n)
        x = (x - x.mean(0)) / _length(x)
        x[:, 2] += 0.005 - x[:, 2].min()
        if not _too_close(x, 4 * 0.002, 3, False):
            break
    else:
        raise RuntimeError("could not draw a flat knotted rope")
    rods = [x] * pop
    gp, gr = _grippers_for(rods)
    mean = _smooth_actions(rng, frames, 1, 1e-3)
    acts = mean + _smooth_actions(rng, frames, pop, 1e-3, amp_pos=sigma, amp_rot=sigma)
    return _assemble("cmaes", rods, np.zeros(pop, bool), dict(K=1e5, E=1e4, G=0.0),
                     frames, acts, np.full(pop, 2), gp, gr,
                     planes=np.array([[0.0, 0.0, 1.0, 0.0]]), self_contact=True)


def _tangled_pair(rng, n: int, length: float, radius: float, z_min: float):
    """Two ropes of n vertices and the given length lying across each other on the table.

    Both follow x over the same span; across it the offsets (y, z) = +-(a sin th, d cos th)
    with th = 2 pi k s + phi put them on opposite sides of a common centre line, so they
    cross wherever sin th = 0, one over and one under, the order alternating from crossing to
    crossing (a braid: the ropes are tangled).  At every parameter s they are at least 2 d
    apart, d = 1.5 r, a gap of one radius.  A shared smooth sideways wiggle, a random heading
    and a random place on the table follow.  The span is 0.85 of the length, so each rope is
    about ``length`` long.  Returns the two (n, 3) ropes."""
    dense = 2048
    d = 1.5 * radius
    for _ in range(200):
        k = rng.uniform(1.2, 1.8)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        a = rng.uniform(0.03, 0.05)
        s = np.linspace(0.0, 1.0, dense)
        th = 2.0 * np.pi * k * s + phi
        wig = np.zeros(dense)
        for m in range(1, 3):
            wig += rng.uniform(-0.02, 0.02) / m * np.sin(2.0 * np.pi * m * s + rng.uniform(0.0, 2.0 * np.pi))
        span = length * 0.85
        base = np.stack([(s - 0.5) * span, wig, np.full(dense, z_min + d)], axis=1)
        off = np.stack([np.zeros(dense), a * np.sin(th), d * np.cos(th)], axis=1)
        ropes = [_resample(base + sign * off, n) for sign in (1.0, -1.0)]
        ang = rng.uniform(0.0, 2.0 * np.pi)
        Rz = np.array([[np.cos(ang), -np.sin(ang), 0.0], [np.sin(ang), np.cos(ang), 0.0], [0.0, 0.0, 1.0]])
        c = np.append(rng.uniform(-0.25, 0.25, 2), 0.0)
        ropes = [r @ Rz.T + c for r in ropes]
        gap = np.linalg.norm(ropes[0][:, None] - ropes[1][None], axis=2).min()
        crossings = np.count_nonzero(np.diff(np.sign(np.sin(th))) != 0)
        if gap >= 2.5 * radius and crossings >= 2 and _max_curvature(ropes[0]) <= 50.0:
            return ropes
    raise RuntimeError("could not draw a tangled pair of ropes")


def separation(n_envs: int = 4096, frames: int = 2000, seed: int = 6000, n: int = 30,
               length: float = 0.6) -> Problem:
    """The Separation task's scene, repeated over environments: two tangled ropes of n
    vertices each (Separation rows: inextensible, E = 5e3 Pa, G = 1e3 Pa), stored as one
    record of two strands, on the table.  Gripper 0 holds the first rope and gripper 1 the
    second, each at the vertex of its half where the ropes are furthest apart; they follow
    smooth random 6-DoF trajectories (3 cm, 0.1 rad) plus a drift that pulls the ropes apart
    sideways (0.15 m over the episode) and lifts them by 3 cm.  Self-contact on, which is what couples the
    two ropes."""
    rng = np.random.default_rng(seed)
    recs, gp, gr, drift = [], np.zeros((n_envs, 2, 3)), np.tile(np.eye(3), (n_envs, 2, 1, 1)), []
    for b in range(n_envs):
        A, Bp = _tangled_pair(rng, n, length, 0.002, 0.005)
        recs.append(np.concatenate([A, Bp]))
        sep = np.linalg.norm(A - Bp, axis=1)
        lo, hi = int(0.15 * (n - 1)), int(0.4 * (n - 1))
        ka = lo + int(np.argmax(sep[lo:hi + 1]))
        kb = (n - 1 - hi) + int(np.argmax(sep[n - 1 - hi:n - lo]))
        for g, (rope, k) in enumerate(((A, ka), (Bp, kb))):
            gp[b, g] = rope[k]
            gr[b, g] = _gripper_frame(rope[min(k + 1, n - 1)] - rope[max(k - 1, 0)])
        out = A[ka] - Bp[kb]
        out[2] = 0.0
        out /= max(np.linalg.norm(out), 1e-9)
        drift.append(out)
    acts = _smooth_actions(rng, frames, n_envs, 1e-3, amp_pos=0.03, amp_rot=0.1)
    dirs = np.stack(drift)
    acts[:, :, 0, :3] += (0.15 / frames) * dirs[None]
    acts[:, :, 1, :3] -= (0.15 / frames) * dirs[None]
    acts[:, :, :, 2] += 0.03 / frames
    start = np.zeros(2 * n * n_envs, bool)
    start[n::2 * n] = True
    return _assemble("separation", recs, np.zeros(n_envs, bool),
                     dict(K=0.0, E=5e3, G=1e3, inextensible=True),
                     frames, acts, np.full(n_envs, 2), gp, gr,
                     planes=np.array([[0.0, 0.0, 1.0, 0.0]]), self_contact=True, strand_start=start)


def custom(rods_x, closed=None, frames: int = 1, actions=None, n_grippers=None, grip_pos=None,
           grip_rot=None, pinned=None, **kw) -> Problem:
    """A hand-made workload: explicit rod shapes plus material / option overrides."""
    B = len(rods_x)
    closed = np.zeros(B, bool) if closed is None else np.asarray(closed, bool)
    mats = {k: kw.pop(k) for k in list(kw) if k in (
        "density", "radius", "K", "E", "G", "inextensible", "strain_limit", "plastic",
        "yield_curv", "creep_rate", "damping")}
    if actions is None:
        actions = np.zeros((frames, B, 2, 6))
    if n_grippers is None:
        n_grippers = np.zeros(B, np.int32)
    if grip_pos is None:
        grip_pos = np.zeros((B, 2, 3))
    if grip_rot is None:
        grip_rot = np.tile(np.eye(3), (B, 2, 1, 1))
    return _assemble("custom", [np.asarray(r, np.float64) for r in rods_x], closed, mats, frames,
                     actions, n_grippers, grip_pos, grip_rot, pinned=pinned, **kw)


def small_case(kind: str, n_rods: int = 4, n: int = 24, frames: int = 10, seed: int = 7) -> Problem:
    """Reduced versions of the workloads for parity tests (same recipes, fewer rods)."""
    if kind == "plain":
        return plain(frames)
    if kind == "batching":
        return batching(n_rods, frames, seed, vmin=max(4, n // 2), vmax=n)
    if kind == "diff":
        return diff(n_rods, frames, seed, n)
    if kind == "selfcontact":
        return selfcontact(n_rods, frames, seed, n)
    if kind == "cmaes":
        return cmaes(n_rods, frames, seed, n)
    if kind == "trajopt":
        return trajopt(n_rods, frames, seed, n, self_contact=True)
    if kind == "separation":
        return separation(n_rods, frames, seed, n)
    raise ValueError(kind)
