"""ctypes binding of libdlo.so (include/dlo.h) plus a torch ``autograd.Function``.

Argument marshalling only: every step of the simulation runs in the library's CUDA
kernels.  PyTorch provides device memory (its caching allocator, passed to the library as
``dlo_allocator``) and the CUDA stream.  There is no CPU fallback: if the library is
missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libdlo.so")
LIB_DEBUG_PATH = os.path.join(_PKG, "_lib_debug", "libdlo.so")   # build(debug_bounds=True)
HEADER = os.path.join(os.path.dirname(_PKG), "include", "dlo.h")

STATUS = {0: "DLO_OK", 1: "DLO_ERR_INVALID_ARG", 2: "DLO_ERR_CUDA", 3: "DLO_ERR_OOM", 4: "DLO_ERR_NONFINITE",
          5: "DLO_ERR_CAPACITY", 6: "DLO_ERR_TIMEOUT", 7: "DLO_ERR_STATE"}
Q_SUBSTEPS, Q_STATUS, Q_BYTES, Q_CONFIG, Q_RESIDUAL, Q_PAIRS, Q_LAUNCHES, Q_MASS, Q_PAIR_LIST = range(1, 10)
PAIR_LIST_STRIDE = 1024   # candidates per rod row of Q_PAIR_LIST (4 per vertex of 256 vertices)
STATUS_NONFINITE, STATUS_PAIR_OVERFLOW, STATUS_MOVED_PAST_MARGIN, STATUS_BOUNDS = 1, 2, 4, 8
MATERIAL_KEYS = ("K", "E", "G", "yield_curv", "damping")
LOSS_TARGET, LOSS_CHAMFER, LOSS_WINDING, LOSS_CROSSING, LOSS_MINDIST, LOSS_REPULSION = range(1, 7)
N_MAT_GRAD = 5      # K_stretch, E_bend, G_twist, yield_curv, damping


class DloError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Material(C.Structure):
    _fields_ = [("density", C.c_float), ("radius", C.c_float), ("K_stretch", C.c_float), ("E_bend", C.c_float),
                ("G_twist", C.c_float), ("inextensible", C.c_int), ("strain_limit", C.c_float),
                ("plastic", C.c_int), ("yield_curv", C.c_float), ("creep_rate", C.c_float),
                ("damping", C.c_float), ("closed", C.c_int)]


class Scene(C.Structure):
    _fields_ = [("n_planes", C.c_int), ("planes", C.POINTER(C.c_float)), ("n_boxes", C.c_int),
                ("boxes", C.POINTER(C.c_float)), ("n_grippers", C.POINTER(C.c_int)),
                ("grip_pose", C.POINTER(C.c_float)), ("grip_radius", C.c_float), ("grip_half_len", C.c_float),
                ("pinned", C.POINTER(C.c_ubyte)), ("strand_start", C.POINTER(C.c_ubyte))]


class Options(C.Structure):
    _fields_ = [("dt", C.c_float), ("n_iter_pbd", C.c_int), ("substeps_min", C.c_int), ("gravity", C.c_float),
                ("mu_self", C.c_float), ("mu_rigid", C.c_float), ("restitution", C.c_float),
                ("eps_soft", C.c_float), ("contact_margin", C.c_float), ("self_contact", C.c_int),
                ("checkpoint_every", C.c_int), ("hbm_budget", C.c_size_t), ("warps_per_cta", C.c_int),
                ("reaction", C.c_int), ("broad_phase", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


_libs = {}


def load(path: str | None = None):
    """Load libdlo.so (built by ``paper_2606_04206_gb300.build``); raises if it is missing."""
    p = path or LIB_PATH
    if p in _libs:
        return _libs[p]
    if not os.path.exists(p):
        raise RuntimeError(f"libdlo.so not found at {p}: run paper_2606_04206_gb300.build.build() first")
    lib = C.CDLL(p)
    vp, fp, ip, st = C.c_void_p, C.POINTER(C.c_float), C.c_int, C.c_int
    lib.dlo_create.argtypes = [C.POINTER(vp), ip, C.POINTER(C.c_int), C.POINTER(Material), fp, C.POINTER(Scene),
                               C.POINTER(Options), C.POINTER(Allocator), vp]
    lib.dlo_create.restype = st
    lib.dlo_build_flags.argtypes = []
    lib.dlo_build_flags.restype = C.c_int
    lib.dlo_set_material.argtypes = [vp, C.POINTER(Material)]
    lib.dlo_set_material.restype = st
    lib.dlo_set_state.argtypes = [vp, vp, vp, vp]
    lib.dlo_set_state.restype = st
    lib.dlo_get_state.argtypes = [vp, vp, vp, vp]
    lib.dlo_get_state.restype = st
    lib.dlo_get_internal.argtypes = [vp, vp, vp, vp, vp]
    lib.dlo_get_internal.restype = st
    lib.dlo_begin_rollout.argtypes = [vp, ip]
    lib.dlo_begin_rollout.restype = st
    lib.dlo_step.argtypes = [vp, vp, ip, ip, vp]
    lib.dlo_step.restype = st
    lib.dlo_step_plain.argtypes = [vp, vp, ip, ip]
    lib.dlo_step_plain.restype = st
    lib.dlo_backward.argtypes = [vp] * 9
    lib.dlo_backward.restype = st
    lib.dlo_backward_plain.argtypes = [vp] * 9
    lib.dlo_backward_plain.restype = st
    lib.dlo_backward_noalloc.argtypes = [vp] * 9
    lib.dlo_backward_noalloc.restype = st
    lib.dlo_loss.argtypes = [vp, ip, vp, vp, ip, vp, vp, vp]
    lib.dlo_loss.restype = st
    lib.dlo_loss_silhouette.argtypes = [vp, vp, vp, ip, ip, ip, vp, C.c_float, vp, vp, vp, vp]
    lib.dlo_loss_silhouette.restype = st
    lib.dlo_reaction.argtypes = [vp, vp, vp, ip]
    lib.dlo_reaction.restype = st
    lib.dlo_query.argtypes = [vp, ip, vp]
    lib.dlo_query.restype = st
    lib.dlo_measure_fp32_peak.argtypes = [C.c_double, vp, C.POINTER(C.c_double)]
    lib.dlo_measure_fp32_peak.restype = st
    lib.dlo_status_string.argtypes = [st]
    lib.dlo_status_string.restype = C.c_char_p
    lib.dlo_last_error.argtypes = [vp]
    lib.dlo_last_error.restype = C.c_char_p
    lib.dlo_destroy.argtypes = [vp]
    lib.dlo_destroy.restype = None
    _libs[p] = lib
    return lib


def header_functions(path: str = HEADER):
    """Names of the functions the public header declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dlo_[a-z_]+)\s*\(", txt)))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def options_from(prob, **over) -> Options:
    o = Options(dt=prob.dt, n_iter_pbd=prob.n_iter, substeps_min=prob.substeps_min, gravity=prob.gravity,
                mu_self=prob.mu_self, mu_rigid=prob.mu_rigid, restitution=prob.restitution,
                eps_soft=prob.eps_soft, contact_margin=prob.contact_margin, self_contact=int(prob.self_contact),
                checkpoint_every=0, hbm_budget=0, warps_per_cta=0, reaction=0, broad_phase=0)
    for k, v in over.items():
        setattr(o, k, v)
    return o


class DloSim:
    """One library context over the rods of a workload (``inputs.Problem``).

    Device memory comes from torch's caching allocator, or from ``allocator``: a pair of
    callables (alloc(nbytes) -> device address or None, free(address)) handed to the
    library as its dlo_allocator."""

    def __init__(self, prob, torch_alloc: bool = True, allocator=None, debug_bounds: bool = False, **opt):
        import torch
        self.torch = torch
        self.lib = load(LIB_DEBUG_PATH if debug_bounds else None)
        self.p = prob
        self.B = prob.batch
        self.V = int(prob.vert_off[-1])
        self.E = int(prob.edge_off[-1])
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream()
        B = self.B
        self._keep = []
        self._mat = np.stack([np.asarray(getattr(prob, k), np.float32) for k in MATERIAL_KEYS], 1)
        mats = self._materials(self._mat)
        self.rollout_id = 0   # advanced by every call that replaces or ends the recorded rollout
        nv = np.ascontiguousarray(prob.n_verts, np.int32)
        xr = np.ascontiguousarray(prob.x_rest, np.float32)
        planes = np.ascontiguousarray(prob.planes, np.float32).reshape(-1)
        boxes = np.ascontiguousarray(prob.boxes, np.float32).reshape(-1)
        ng = np.ascontiguousarray(prob.n_grippers, np.int32)
        pose = np.zeros((B, 2, 12), np.float32)
        pose[..., :3] = prob.grip_pos
        pose[..., 3:] = np.asarray(prob.grip_rot).reshape(B, 2, 9)
        pinned = np.ascontiguousarray(prob.pinned, np.uint8)
        st = getattr(prob, "strand_start", None)
        starts = None if st is None or not np.any(st) else np.ascontiguousarray(st, np.uint8)
        self._keep += [mats, nv, xr, planes, boxes, ng, pose, pinned, starts]
        scene = Scene(len(prob.planes), _fptr(planes) if len(planes) else None, len(prob.boxes),
                      _fptr(boxes) if len(boxes) else None, ng.ctypes.data_as(C.POINTER(C.c_int)),
                      _fptr(pose), prob.grip_radius, prob.grip_half_len,
                      pinned.ctypes.data_as(C.POINTER(C.c_ubyte)),
                      None if starts is None else starts.ctypes.data_as(C.POINTER(C.c_ubyte)))
        self.options = options_from(prob, **opt)
        alloc = None
        if allocator is not None:
            ua, uf = allocator

            def _alloc(n, user):
                try:
                    return ua(int(n))
                except Exception:
                    return None

            def _free(p, user):
                uf(p)

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            alloc = Allocator(self._cb[0], self._cb[1], None)
        elif torch_alloc:
            dev = self.device.index
            stream = self.stream

            def _alloc(n, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(n), dev, stream)
                except Exception:
                    return None

            def _free(p, user):
                torch.cuda.caching_allocator_delete(p)

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            alloc = Allocator(self._cb[0], self._cb[1], None)
        ctx = C.c_void_p()
        st = self.lib.dlo_create(C.byref(ctx), B, nv.ctypes.data_as(C.POINTER(C.c_int)), mats, _fptr(xr),
                                 C.byref(scene), C.byref(self.options), C.byref(alloc) if alloc else None,
                                 C.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise DloError(st, "dlo_create failed")
        self.ctx = ctx

    # ------------------------------------------------------------------ helpers
    def _materials(self, vals):
        """dlo_material[B] from the workload with (K, E, G, yield_curv, damping) = vals [B, 5]."""
        p = self.p
        mats = (Material * self.B)()
        for b in range(self.B):
            K, E, G, sy, cd = (float(v) for v in vals[b])
            mats[b] = Material(p.density[b], p.radius[b], K, E, G, int(p.inextensible[b]), p.strain_limit[b],
                               int(p.plastic[b]), sy, p.creep_rate[b], cd, int(p.closed[b]))
        return mats

    def _check(self, st, what):
        if st != 0:
            raise DloError(st, f"{what}: {self.lib.dlo_last_error(self.ctx).decode()}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dlo_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tensors_from_problem(self, x=None, v=None, theta=None, omega=None):
        """Device state tensors (x [V,4], v [V,4], theta [E]) from workload arrays."""
        torch, p = self.torch, self.p
        x = p.x0 if x is None else x
        v = p.v0 if v is None else v
        theta = p.theta0 if theta is None else theta
        omega = p.omega0 if omega is None else omega
        X = np.zeros((self.V, 4), np.float32)
        X[:, :3] = x
        Vv = np.zeros((self.V, 4), np.float32)
        Vv[:, :3] = v
        vo, eo = p.vert_off, p.edge_off
        for b in range(self.B):
            ne = eo[b + 1] - eo[b]
            Vv[vo[b]:vo[b] + ne, 3] = omega[eo[b]:eo[b + 1]]
        dev = self.device
        return (torch.as_tensor(X, device=dev), torch.as_tensor(Vv, device=dev),
                torch.as_tensor(np.asarray(theta, np.float32), device=dev))

    # ------------------------------------------------------------------ API
    def set_state(self, x, v, theta):
        self.rollout_id += 1
        self._check(self.lib.dlo_set_state(self.ctx, _ptr(x), _ptr(v), _ptr(theta)), "dlo_set_state")

    def set_material(self, values):
        """dlo_set_material: per-rod (K_stretch, E_bend, G_twist, yield_curv, damping) = values
        [B, 5] (array or tensor) for the next steps; ends any recorded rollout."""
        vals = np.asarray(values.detach().cpu().numpy() if hasattr(values, "detach") else values, np.float32)
        assert vals.shape == (self.B, N_MAT_GRAD), vals.shape
        self.rollout_id += 1
        self._check(self.lib.dlo_set_material(self.ctx, self._materials(vals)), "dlo_set_material")
        self._mat = vals.copy()

    def reset(self):
        self.set_state(*self.tensors_from_problem())

    def get_state(self):
        torch = self.torch
        x = torch.empty(self.V, 4, device=self.device)
        v = torch.empty(self.V, 4, device=self.device)
        th = torch.empty(self.E, device=self.device)
        self._check(self.lib.dlo_get_state(self.ctx, _ptr(x), _ptr(v), _ptr(th)), "dlo_get_state")
        return x, v, th

    def get_internal(self):
        torch = self.torch
        ref = torch.empty(self.E, 4, device=self.device)
        tan = torch.empty(self.E, 4, device=self.device)
        hinge = torch.empty(self.V, 4, device=self.device)
        grip = torch.empty(self.B, 2, 12, device=self.device)
        self._check(self.lib.dlo_get_internal(self.ctx, _ptr(ref), _ptr(tan), _ptr(hinge), _ptr(grip)),
                    "dlo_get_internal")
        return ref, tan, hinge, grip

    def full_state_numpy(self):
        """Every state array as float64 numpy in the oracle's layout."""
        x, v, th = self.get_state()
        ref, tan, hinge, grip = self.get_internal()
        x, v, th, ref, tan, hinge, grip = (a.double().cpu().numpy() for a in (x, v, th, ref, tan, hinge, grip))
        p = self.p
        om = np.zeros(self.E)
        vo, eo = p.vert_off, p.edge_off
        for b in range(self.B):
            ne = eo[b + 1] - eo[b]
            om[eo[b]:eo[b + 1]] = v[vo[b]:vo[b] + ne, 3]
        return dict(x=x[:, :3], v=v[:, :3], theta=th, omega=om, d1b=ref[:, :3], tb=tan[:, :3],
                    kbar=hinge[:, :2], mprev=hinge[:, 3], mbar=hinge[:, 2], gp=grip[..., :3],
                    gR=grip[..., 3:].reshape(self.B, 2, 3, 3))

    def begin_rollout(self, n_frames):
        self.rollout_id += 1
        self._rec_left = 0
        self._check(self.lib.dlo_begin_rollout(self.ctx, int(n_frames)), "dlo_begin_rollout")
        self._rec_left = int(n_frames)
        self._rollout_frames = int(n_frames)

    def step(self, actions=None, frames=None, substeps=0, x_frames=None):
        if frames is None:
            frames = actions.shape[0]
        if actions is not None:
            assert actions.is_cuda and actions.dtype == self.torch.float32 and actions.is_contiguous()
            assert actions.numel() >= frames * self.B * 12
        self._check(self.lib.dlo_step(self.ctx, _ptr(actions), int(frames), int(substeps), _ptr(x_frames)),
                    "dlo_step")
        if frames > 0:
            if getattr(self, "_rec_left", 0) >= frames:
                self._rec_left -= frames     # part of the armed recording
            else:
                self.rollout_id += 1         # a step past the recording ends it
                self._rec_left = 0

    def step_plain(self, actions=None, frames=None, substeps=0):
        if frames is None:
            frames = actions.shape[0]
        self._check(self.lib.dlo_step_plain(self.ctx, _ptr(actions), int(frames), int(substeps)), "dlo_step_plain")
        if frames > 0:   # recorded like dlo_step when a rollout is armed
            if getattr(self, "_rec_left", 0) >= frames:
                self._rec_left -= frames
            else:
                self.rollout_id += 1
                self._rec_left = 0

    def backward(self, dL_dx=None, dL_dv=None, dL_dtheta=None, want=("actions", "material", "x0", "v0", "theta0"),
                 plain=False):
        """dlo_backward (plain=True: dlo_backward_plain, the per-phase comparator)."""
        torch = self.torch
        n = getattr(self, "_rollout_frames", 0)
        out = {}
        if "actions" in want:
            out["actions"] = torch.zeros(n, self.B, 2, 6, device=self.device)
        if "material" in want:
            out["material"] = torch.zeros(self.B, N_MAT_GRAD, device=self.device)
        if "x0" in want:
            out["x0"] = torch.zeros(self.V, 4, device=self.device)
        if "v0" in want:
            out["v0"] = torch.zeros(self.V, 4, device=self.device)
        if "theta0" in want:
            out["theta0"] = torch.zeros(self.E, device=self.device)
        fn = self.lib.dlo_backward_plain if plain else self.lib.dlo_backward
        st = fn(self.ctx, _ptr(dL_dx), _ptr(dL_dv), _ptr(dL_dtheta), _ptr(out.get("actions")),
                _ptr(out.get("material")), _ptr(out.get("x0")), _ptr(out.get("v0")), _ptr(out.get("theta0")))
        self._check(st, "dlo_backward_plain" if plain else "dlo_backward")
        return out

    def backward_noalloc(self, dL_dx=None, dL_dv=None, dL_dtheta=None,
                         want=("actions", "material", "x0", "v0", "theta0")):
        """dlo_backward_noalloc: the same gradients with no allocation inside the library
        (the output tensors are the caller's, allocated here by torch before the call)."""
        torch = self.torch
        n = getattr(self, "_rollout_frames", 0)
        shapes = {"actions": (n, self.B, 2, 6), "material": (self.B, N_MAT_GRAD), "x0": (self.V, 4),
                  "v0": (self.V, 4), "theta0": (self.E,)}
        out = {k: torch.zeros(*shapes[k], device=self.device) for k in want}
        st = self.lib.dlo_backward_noalloc(self.ctx, _ptr(dL_dx), _ptr(dL_dv), _ptr(dL_dtheta),
                                           _ptr(out.get("actions")), _ptr(out.get("material")),
                                           _ptr(out.get("x0")), _ptr(out.get("v0")), _ptr(out.get("theta0")))
        self._check(st, "dlo_backward_noalloc")
        return out

    def query(self, what):
        if what == Q_SUBSTEPS:
            o = (C.c_int * self.B)()
        elif what == Q_STATUS:
            o = (C.c_uint * self.B)()
        elif what == Q_BYTES:
            o = C.c_size_t()
        elif what == Q_CONFIG:
            o = (C.c_int * 4)()
        elif what == Q_RESIDUAL:
            o = (C.c_double * self.B)()
        elif what == Q_PAIRS:
            o = (C.c_int * self.B)()
        elif what == Q_LAUNCHES:
            o = C.c_longlong()
        elif what == Q_MASS:
            o = (C.c_float * (4 * self.V))()
        elif what == Q_PAIR_LIST:
            o = (C.c_uint * ((1 + PAIR_LIST_STRIDE) * self.B))()
        else:
            raise ValueError(what)
        self._check(self.lib.dlo_query(self.ctx, what, C.byref(o)), "dlo_query")
        if hasattr(o, "value"):
            return o.value
        a = np.ctypeslib.as_array(o).copy()
        if what == Q_MASS:
            return a.reshape(self.V, 4)
        if what == Q_PAIR_LIST:
            return a.reshape(self.B, 1 + PAIR_LIST_STRIDE)
        return a

    def pair_sets(self):
        """Self-contact candidates of the last frame of the last dlo_step, per rod: a set of
        (edge a, edge b) with a < b (DLO_Q_PAIR_LIST)."""
        rows = self.query(Q_PAIR_LIST)
        return [{(int(e & 0xffff), int(e >> 16)) for e in r[1:1 + int(r[0])]} for r in rows]

    def loss(self, kind, x, aux=None, g=None, grad=True):
        """dlo_loss: per-rod task loss q [B] and (grad=True) dL/dx [V,4] for L = sum_b g_b q_b."""
        torch = self.torch
        q = torch.empty(self.B, device=self.device)
        gx = torch.empty(self.V, 4, device=self.device) if grad else None
        m = 0
        if kind == LOSS_CHAMFER:
            assert aux is not None and aux.dim() == 3 and aux.shape[0] == self.B and aux.shape[2] == 4
            m = aux.shape[1]
        self._check(self.lib.dlo_loss(self.ctx, int(kind), _ptr(x), _ptr(aux), int(m), _ptr(g), _ptr(q), _ptr(gx)),
                    "dlo_loss")
        return q, gx

    def silhouette(self, x, cams, masks, tau=1.0, g=None, grad=True, render=False):
        """dlo_loss_silhouette: per-rod mean squared difference between the soft silhouettes of
        the rods seen by pinhole cameras cams [C,16] and binary masks [B,C,H,W] (uint8); returns
        (q [B], dL/dx [V,4] or None, soft silhouettes [B,C,H,W] or None)."""
        torch = self.torch
        assert cams.is_cuda and cams.dtype == torch.float32 and cams.dim() == 2 and cams.shape[1] == 16
        assert masks.is_cuda and masks.dtype == torch.uint8 and masks.dim() == 4 and masks.shape[0] == self.B
        C_, H, W = masks.shape[1], masks.shape[2], masks.shape[3]
        assert cams.shape[0] == C_
        q = torch.empty(self.B, device=self.device)
        gx = torch.empty(self.V, 4, device=self.device) if grad else None
        img = torch.empty(self.B, C_, H, W, device=self.device) if render else None
        cams, masks = cams.contiguous(), masks.contiguous()
        self._check(self.lib.dlo_loss_silhouette(self.ctx, _ptr(x), _ptr(cams), int(C_), int(H), int(W), _ptr(masks),
                                                 float(tau), _ptr(g), _ptr(q), _ptr(gx), _ptr(img)),
                    "dlo_loss_silhouette")
        return q, gx, img

    def reaction(self, per_vertex=False, reset=False):
        """dlo_reaction: the contact impulses the rigid primitives gave each rod since the last
        reset, [B, 4, 3] (planes, boxes, gripper 0, gripper 1), and per vertex [V, 4, 3] if asked.
        The context must be created with reaction=1."""
        torch = self.torch
        pr = torch.empty(self.B, 4, 4, device=self.device)
        pv = torch.empty(self.V, 4, 4, device=self.device) if per_vertex else None
        self._check(self.lib.dlo_reaction(self.ctx, _ptr(pr), _ptr(pv), int(reset)), "dlo_reaction")
        return pr[..., :3], (pv[..., :3] if per_vertex else None)

    def material_tensor(self):
        """The context's current per-rod material as a [B, 5] tensor (K_stretch, E_bend, G_twist,
        yield_curv, damping): the input whose gradient DloRollout returns."""
        return self.torch.as_tensor(self._mat.copy(), device=self.device)


def _rollout_function():
    import torch

    class DloRollout(torch.autograd.Function):
        """A recorded rollout as a differentiable torch operation (Sec. 3.3).

        forward(sim, x0 [V,4], v0 [V,4], theta0 [E], actions [F,B,2,6], material [B,5])
        sets the material (dlo_set_material, when it differs from the context's) and the
        state, records and steps F frames, and returns the final (x, v, theta).
        backward runs dlo_backward on the recorded rollout; it raises if the context has
        recorded or reset anything since this forward (its record would belong to another
        rollout)."""

        @staticmethod
        def forward(ctx, sim, x0, v0, theta0, actions, material, plain=False):
            frames = actions.shape[0]
            mat = material.detach().float().cpu().numpy()
            if mat.shape != sim._mat.shape:
                raise ValueError(f"material must be [B, {N_MAT_GRAD}], got {tuple(mat.shape)}")
            if not np.array_equal(mat, sim._mat):
                sim.set_material(mat)
            sim.set_state(x0.contiguous(), v0.contiguous(), theta0.contiguous())
            sim.begin_rollout(frames)
            if plain:
                sim.step_plain(actions.contiguous(), frames)
            else:
                sim.step(actions.contiguous(), frames)
            x, v, th = sim.get_state()
            ctx.sim = sim
            ctx.plain = plain
            ctx.rollout_id = sim.rollout_id
            return x, v, th

        @staticmethod
        def backward(ctx, gx, gv, gth):
            if ctx.sim.rollout_id != ctx.rollout_id:
                raise RuntimeError("DloRollout.backward: the context has recorded or reset another rollout since "
                                   "this one ran; run its backward before the next rollout on the same DloSim")
            need = ctx.needs_input_grad
            want = [k for k, n in zip(("x0", "v0", "theta0", "actions", "material"), need[1:]) if n]
            g = ctx.sim.backward(None if gx is None else gx.contiguous(), None if gv is None else gv.contiguous(),
                                 None if gth is None else gth.contiguous(), want=tuple(want), plain=ctx.plain)
            return (None, g.get("x0"), g.get("v0"), g.get("theta0"), g.get("actions"), g.get("material"), None)

    return DloRollout


def rollout(sim, x0, v0, theta0, actions, material=None, plain=False):
    """Differentiable rollout through the library: final (x, v, theta) after actions.shape[0]
    frames, with gradients with respect to every tensor input (DloRollout).  plain=True runs
    the plain per-phase comparator (dlo_step_plain, dlo_backward_plain) instead."""
    if material is None:
        material = sim.material_tensor()
    return _rollout_function().apply(sim, x0, v0, theta0, actions, material, plain)


def measure_fp32_peak(seconds=1.0):
    """dlo_measure_fp32_peak on torch's current stream: the device's FP32 TFLOP/s."""
    import torch
    lib = load()
    out = C.c_double()
    st = lib.dlo_measure_fp32_peak(float(seconds), C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(out))
    if st != 0:
        raise DloError(st, "dlo_measure_fp32_peak failed")
    return out.value
