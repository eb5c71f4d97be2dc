"""The CUDA element functions (compiled here as host code) against the FP64 oracle.

The stepper's device math is written once as templates on the scalar type; this test
compiles those templates for the host and compares each element with the oracle:
hinge energy gradients (vs autograd of the oracle energy), second derivatives taken with
dual numbers (vs double autograd), rigid-contact response, segment closest points, the
exponential map.  It needs nvcc but no GPU."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest
import torch

from oracle.dlo import edge_frames, hinge_strains, expmap, closest_params, sdf_box, sdf_capsule, OracleSim
from paper_2606_04206_gb300 import build, inputs

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def H():
    out = os.path.join(tempfile.mkdtemp(), "libharness.so")
    cmd = [build.nvcc(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr",
           "-I", build.CSRC, os.path.join(HERE, "host_harness.cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = C.CDLL(out)
    for n in ("hinge_grad_host", "contact_host", "closest_host", "expmap_host", "capsule_rev_check",
              "plane_rev_check", "pair_vjp_check", "box_rev_check"):
        getattr(lib, n).argtypes = [C.c_void_p, C.c_void_p]
    lib.hinge_hvp_host.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.hinge_fold_host.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return lib


def fl(a):
    return np.ascontiguousarray(a, np.float32)


def call(fn, *arrs, n_out):
    out = np.zeros(n_out, np.float32)
    fn(*[a.ctypes.data for a in arrs], out.ctypes.data)
    return out


def rand_hinge(rng):
    x = np.cumsum(rng.normal(size=(3, 3)) * 0.02 + np.array([0.02, 0, 0]), axis=0)
    # bases: previous tangents slightly rotated from the current ones, adapted d1
    t = np.diff(x, axis=0)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    tb = t + rng.normal(size=t.shape) * 0.05
    tb /= np.linalg.norm(tb, axis=1, keepdims=True)
    d = rng.normal(size=t.shape)
    d -= (d * tb).sum(1, keepdims=True) * tb
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    th = rng.normal(size=2) * 0.4
    return x, tb, d, th


def oracle_hinge(x, tb, d, th, mprev, kbar, mbar, lbar, Bm, beta):
    X = torch.tensor(x[None], requires_grad=True)
    TH = torch.tensor(th[None], requires_grad=True)
    t, ell, d1r, d1, d2 = edge_frames(X, TH, torch.tensor(tb[None]), torch.tensor(d[None]), False)
    kap, mref, m = hinge_strains(t, d1r, d1, d2, TH, torch.tensor([[mprev]]), False)
    U = 0.5 * Bm / lbar * ((kap - torch.tensor(kbar)) ** 2).sum() + 0.5 * beta / lbar * ((m - mbar) ** 2).sum()
    gx, gth = torch.autograd.grad(U, [X, TH])
    return float(U.detach()), gx[0].numpy(), gth[0].numpy(), kap.detach()[0, 0].numpy(), float(mref), d1r.detach()[0].numpy()


def test_hinge_gradient_matches_oracle_autograd(H):
    rng = np.random.default_rng(0)
    for trial in range(20):
        x, tb, d, th = rand_hinge(rng)
        mprev = rng.normal() * 0.3
        kbar = rng.normal(size=2) * 0.05
        mbar, lbar, Bm, beta = rng.normal() * 0.1, 0.02, 3.0, 2.0
        inp = fl(np.concatenate([x.ravel(), tb[0], d[0], tb[1], d[1], th, [mprev], kbar, [mbar, lbar, Bm, beta]]))
        out = call(H.hinge_grad_host, inp, n_out=22)
        U, gx, gth, kap, mref, d1r = oracle_hinge(x.astype(np.float64), tb, d, th, mprev, kbar, mbar, lbar, Bm, beta)
        scale = np.abs(gx).max() + 1e-12
        assert out[0] == pytest.approx(U, rel=2e-4, abs=1e-9)
        np.testing.assert_allclose(out[1:10].reshape(3, 3), gx, atol=2e-4 * scale)
        np.testing.assert_allclose(out[10:12], gth, atol=2e-4 * (np.abs(gth).max() + 1e-9))
        np.testing.assert_allclose(out[13:15], kap, atol=2e-5)
        assert out[12] == pytest.approx(mref, abs=2e-5)
        np.testing.assert_allclose(out[16:22].reshape(2, 3), d1r, atol=2e-5)


def test_hinge_second_derivatives_match_double_autograd(H):
    """The adjoint's second-order pieces: directional derivatives of the hinge gradient with
    respect to every input (positions, bases, twist, rest values, stiffnesses)."""
    rng = np.random.default_rng(1)
    for trial in range(10):
        x, tb, d, th = rand_hinge(rng)
        mprev = rng.normal() * 0.3
        kbar = rng.normal(size=2) * 0.05
        vals = np.concatenate([x.ravel(), tb[0], d[0], tb[1], d[1], th, [mprev], kbar,
                               [rng.normal() * 0.1, 0.02, 3.0, 2.0]])
        dirv = rng.normal(size=30)
        dirv[23] = 0.0
        out = call(H.hinge_hvp_host, fl(vals), fl(dirv), n_out=30)
        z = torch.tensor(vals, requires_grad=True)

        def U(z):
            X = z[:9].reshape(1, 3, 3)
            tb_ = torch.stack([z[9:12], z[15:18]])[None]
            d_ = torch.stack([z[12:15], z[18:21]])[None]
            TH = z[21:23][None]
            t, ell, d1r, d1, d2 = edge_frames(X, TH, tb_, d_, False)
            kap, mref, m = hinge_strains(t, d1r, d1, d2, TH, z[23:24][None], False)
            return (0.5 * z[28] / z[27] * ((kap[0, 0] - z[24:26]) ** 2).sum()
                    + 0.5 * z[29] / z[27] * (m[0, 0] - z[26]) ** 2)

        g = torch.autograd.grad(U(z), z, create_graph=True)[0]
        hv = torch.autograd.grad(g, z, torch.tensor(dirv))[0].numpy()
        scale = np.abs(hv).max()
        np.testing.assert_allclose(out, hv, atol=5e-4 * scale)


def test_yielded_hinge_fold_equals_two_reverse_passes(H):
    """The backward reverses a yielded hinge in one dual pass, with the plastic cotangent of
    the curvature (App. A.1 rest-curvature update) added to the derivative part of the
    curvature seeds.  That equals the dual reverse of the unyielded seeds plus a float
    reverse from the plastic cotangent, because the hinge reverse is linear in its seeds."""
    rng = np.random.default_rng(2)
    for trial in range(50):
        x, tb, d, th = rand_hinge(rng)
        vals = np.concatenate([x.ravel(), tb[0], d[0], tb[1], d[1], th, [rng.normal() * 0.3]])
        dirv = rng.normal(size=24)
        dirv[9:21] = 0.0          # the bases are constants of the substep (no tangent)
        dirv[23] = 0.0
        seeds = rng.normal(size=8)
        out = call(H.hinge_fold_host, fl(vals), fl(dirv), fl(seeds), n_out=46)
        folded, two_pass = out[:23], out[23:]
        scale = max(np.abs(two_pass).max(), 1e-30)
        np.testing.assert_allclose(folded, two_pass, atol=2e-6 * scale)
        # without a tangent only first-order terms remain, so the plastic part is of the same
        # size as the rest: dropping it must change the result
        zero = np.zeros(24)
        f1 = call(H.hinge_fold_host, fl(vals), fl(zero), fl(seeds), n_out=46)
        s1 = max(np.abs(f1[23:]).max(), 1e-30)
        np.testing.assert_allclose(f1[:23], f1[23:], atol=2e-6 * s1)
        seeds0 = seeds.copy()
        seeds0[6:] = 0.0
        base = call(H.hinge_fold_host, fl(vals), fl(zero), fl(seeds0), n_out=46)[:23]
        assert np.abs(base - f1[:23]).max() > 1e-2 * s1


def test_contact_response_matches_oracle(H):
    rng = np.random.default_rng(2)
    p = inputs.custom([np.array([[0, 0, 0.5], [0.01, 0, 0.5]])], K=1e5, E=1e4)
    sim = OracleSim(p)
    r, eps, mu = 0.002, 0.001, 0.5
    for trial in range(60):
        kind = trial % 3
        x = rng.normal(size=3) * 0.004
        v = rng.normal(size=3) * 0.3
        vr = rng.normal(size=3) * 0.1 if kind == 2 else np.zeros(3)
        if kind == 0:
            n = np.array([0, 0, 1.0])
            prm = np.concatenate([n, [rng.normal() * 0.002], np.zeros(5)])
            sdf_o = float(x @ n - prm[3])
            nrm = n
        elif kind == 1:
            c, hl = np.array([0, 0, -0.01]), np.array([0.02, 0.02, 0.01])
            prm = np.concatenate([c, hl, np.zeros(3)])
            s, nn = sdf_box(torch.tensor(x)[None], torch.tensor(c), torch.tensor(hl))
            sdf_o, nrm = float(s[0]), nn[0].numpy()
        else:
            a, b = np.array([0, -0.01, -0.006]), np.array([0, 0.01, -0.006])
            prm = np.concatenate([a, b, [0.004], np.zeros(2)])
            s, nn = sdf_capsule(torch.tensor(x)[None], torch.tensor(a), torch.tensor(b), 0.004)
            sdf_o, nrm = float(s[0]), nn[0].numpy()
        inp = fl(np.concatenate([x, v, vr, [kind], prm, [r, eps, mu, 0.0]]))
        out = call(H.contact_host, inp, n_out=5)
        f = min(np.exp((r - sdf_o) / eps), 1.0)
        vrel = v - vr
        vn = vrel @ nrm
        vt = vrel - vn * nrm
        vn2 = max(vn, 0.0)
        sc = max(1 - mu * (vn2 - vn) / np.linalg.norm(vt), 0.0)
        expect = v + f * (vn2 * nrm + sc * vt - vrel) if f > 0.1 else v
        assert out[4] == pytest.approx(sdf_o, abs=1e-6)
        if abs(f - 0.1) > 1e-3:
            assert bool(out[3]) == (f > 0.1)
            np.testing.assert_allclose(out[:3], expect, atol=2e-5)


def test_closest_points_and_expmap(H):
    rng = np.random.default_rng(3)
    for trial in range(50):
        P = rng.normal(size=(4, 3))
        if trial % 10 == 0:
            P[3] = P[2] + (P[1] - P[0]) * 0.5
        out = call(H.closest_host, fl(P.ravel()), n_out=2)
        s, u = closest_params(*(torch.tensor(q) for q in P))
        np.testing.assert_allclose(out, [float(s), float(u)], atol=1e-4)
    for trial in range(20):
        phi = rng.normal(size=3) * (10.0 ** rng.uniform(-6, 0))
        out = call(H.expmap_host, fl(phi), n_out=9)
        np.testing.assert_allclose(out.reshape(3, 3), expmap(torch.tensor(phi)).numpy(), atol=2e-7)


def test_closed_form_contact_reverses_match_dual_numbers(H):
    """The adjoint's closed-form reverses of the plane and capsule-gripper contact responses
    equal the transpose-Jacobian products taken with dual numbers through the forward code."""
    rng = np.random.default_rng(5)
    n_active = 0
    for trial in range(200):
        x = rng.normal(size=3) * 0.006
        x[2] = abs(x[2]) + 0.009                 # around the capsule surface
        v = rng.normal(size=3) * 0.2
        p = np.zeros(3)
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        inp = fl(np.concatenate([x, v, p, ax, [0.02, 0.01], rng.normal(size=3) * 0.05, rng.normal(size=3),
                                 [0.002, 0.001, 0.5, 0.0], rng.normal(size=3)]))
        out = call(H.capsule_rev_check, inp, n_out=37)
        if out[36] == 0:
            continue                             # not in contact
        n_active += 1
        np.testing.assert_allclose(out[:18], out[18:36], rtol=2e-3, atol=2e-3 * np.abs(out[18:36]).max())
    assert n_active > 20
    for trial in range(100):
        x = np.array([0.0, 0.0, rng.uniform(-0.002, 0.004)])
        inp = fl(np.concatenate([x, rng.normal(size=3) * 0.3, [0, 0, 1.0], [0.0, 0.002, 0.001, 0.5, 0.0],
                                 rng.normal(size=3)]))
        out = call(H.plane_rev_check, inp, n_out=13)
        if out[12] == 0:
            continue
        np.testing.assert_allclose(out[:6], out[6:12], rtol=2e-3, atol=2e-3 * max(np.abs(out[6:12]).max(), 1e-6))


def test_closed_form_pair_reverses_match_dual_numbers(H):
    """The adjoint's closed-form vector-Jacobian products of the self-collision projection and of
    the pair friction (App. A.1) equal the transpose-Jacobian products taken with dual numbers
    through the forward code, in every branch of the clamped closest-point solve: interior
    points, one or both parameters clamped at a segment end, and near-parallel segments."""
    rng = np.random.default_rng(11)
    r = 0.002
    seen = {"proj": 0, "fric": 0, "end": 0, "parallel": 0}
    for trial in range(3000):
        kind = trial % 3
        p0 = rng.normal(size=3) * 0.004
        d1 = rng.normal(size=3)
        d1 *= 0.01 / np.linalg.norm(d1)
        if kind == 2:   # near-parallel second segment
            d2 = d1 + rng.normal(size=3) * 1e-4
        else:
            d2 = rng.normal(size=3)
            d2 *= 0.01 / np.linalg.norm(d2)
        # second segment crossing near the first one at a random parameter (beyond its ends for
        # kind 1), a random normal offset below the contact distance
        t = rng.uniform(-0.4, 1.4) if kind == 1 else rng.uniform(0.0, 1.0)
        off = rng.normal(size=3)
        off *= rng.uniform(0.2, 1.0) * 2 * r / np.linalg.norm(off)
        q0 = p0 + t * d1 + off - rng.uniform(0.0, 1.0) * d2
        P = np.concatenate([p0, p0 + d1, q0, q0 + d2])
        V = rng.normal(size=12) * 0.05
        w = rng.uniform(0.5, 2.0, size=4)
        w[rng.integers(0, 4)] *= rng.integers(0, 2)   # sometimes a kinematic end (w = 0)
        inp = fl(np.concatenate([P, V, w, [2 * r, 0.3, 2e-4], rng.normal(size=12), rng.normal(size=12)]))
        out = call(H.pair_vjp_check, inp, n_out=74)
        if out[72]:
            seen["proj"] += 1
            seen["end"] += kind == 1
            seen["parallel"] += kind == 2
            ref = out[12:24]
            np.testing.assert_allclose(out[:12], ref, rtol=2e-3, atol=2e-3 * max(np.abs(ref).max(), 1e-6))
        else:
            assert not np.any(out[12:24])
        if out[73]:
            seen["fric"] += 1
            ref = out[48:72]
            np.testing.assert_allclose(out[24:48], ref, rtol=2e-3, atol=2e-3 * max(np.abs(ref).max(), 1e-6))
        else:
            assert not np.any(out[48:72])
    assert min(seen.values()) > 100, seen


def test_closed_form_box_contact_reverse_matches_dual_numbers(H):
    """The adjoint's closed-form reverse of the soft contact with a box equals the transpose-
    Jacobian products taken with dual numbers through the forward code: outside the box near a
    face, an edge and a corner (the normal turns with the position), and inside it."""
    rng = np.random.default_rng(13)
    hl = np.array([0.15, 0.15, 0.05])
    seen = {"outside": 0, "inside": 0, "edge_or_corner": 0}
    for trial in range(600):
        # a point just outside or inside a random face, edge or corner region
        axes = rng.integers(1, 4)
        sign = rng.choice([-1.0, 1.0], size=3)
        x = rng.uniform(-1.0, 1.0, size=3) * hl * 0.9
        for k in rng.choice(3, size=axes, replace=False):
            x[k] = sign[k] * (hl[k] + rng.uniform(-0.003, 0.004))
        c = rng.normal(size=3) * 0.01
        inp = fl(np.concatenate([x + c, rng.normal(size=3) * 0.3, c, hl, [0.002, 0.001, 0.5, 0.0],
                                 rng.normal(size=3)]))
        out = call(H.box_rev_check, inp, n_out=13)
        if out[12] == 0:
            continue
        q = np.abs(x) - hl
        outside = bool(np.any(q > 0))
        seen["outside" if outside else "inside"] += 1
        seen["edge_or_corner"] += int(np.sum(q > 0) >= 2)
        ref = out[6:12]
        np.testing.assert_allclose(out[:6], ref, rtol=2e-3, atol=2e-3 * max(np.abs(ref).max(), 1e-6))
    assert min(seen.values()) > 20, seen


def test_closed_form_pair_reverses_match_the_oracles_autograd(H):
    """The same closed-form pair reverses against the FP64 oracle's own self-collision sweep and
    friction (App. A.1), differentiated by autograd: an independent definition of the
    projection, so a mistake shared by the device's forward and reverse would show here."""
    from types import SimpleNamespace
    rng = np.random.default_rng(23)
    r, mu, h = 0.002, 0.3, 2e-4
    n_cmp = 0
    for trial in range(400):
        p0 = rng.normal(size=3) * 0.004
        d1 = rng.normal(size=3)
        d1 *= 0.01 / np.linalg.norm(d1)
        d2 = rng.normal(size=3)
        d2 *= 0.01 / np.linalg.norm(d2)
        off = rng.normal(size=3)
        off *= rng.uniform(0.2, 1.0) * 2 * r / np.linalg.norm(off)
        q0 = p0 + rng.uniform(-0.2, 1.2) * d1 + off - rng.uniform(0.0, 1.0) * d2
        P = np.stack([p0, p0 + d1, q0, q0 + d2])
        V = rng.normal(size=(4, 3)) * 0.05
        w = rng.uniform(0.5, 2.0, size=4)
        lx, lv = rng.normal(size=(4, 3)), rng.normal(size=(4, 3))
        inp = fl(np.concatenate([P.ravel(), V.ravel(), w, [2 * r, mu, h], lx.ravel(), lv.ravel()]))
        out = call(H.pair_vjp_check, inp, n_out=74)
        # the oracle: one record of four vertices, the pair (0, 2): segments 0-1 and 2-3, in
        # FP64 and, for the float32 floor of these products, in float32
        res = {}
        for dt in (torch.float64, torch.float32):
            Pt = torch.tensor(P[None], dtype=dt, requires_grad=True)
            Vt = torch.tensor(V[None], dtype=dt, requires_grad=True)
            G = dict(N=4, R=dict(r=torch.tensor([r], dtype=dt), w=torch.tensor(w[None], dtype=dt)))
            xs, infos = OracleSim.contact_sweep(None, G, Pt, [torch.tensor([[0, 2]])])
            if not bool(infos[0]["act"][0]):
                res[dt] = None
                continue
            gp = torch.autograd.grad((xs * torch.tensor(lx[None], dtype=dt)).sum(), Pt, retain_graph=True)[0]
            vs = OracleSim.self_friction(SimpleNamespace(p=SimpleNamespace(mu_self=mu)), G, Vt, infos, h)
            gP, gV = torch.autograd.grad((vs * torch.tensor(lv[None], dtype=dt)).sum(), [Pt, Vt])
            res[dt] = (gp[0].double().numpy() - lx, np.concatenate([gP[0].double().numpy().ravel(),
                                                                     gV[0].double().numpy().ravel() - lv.ravel()]))
        if res[torch.float64] is None:
            assert out[72] == 0
            continue
        assert out[72] == 1 and out[73] == 1
        n_cmp += 1
        (gp, ref), f32 = res[torch.float64], res[torch.float32]
        # where float32 cannot resolve a product (a segment end close to the clamped closest-point
        # solve's boundary, the friction's division by h |v_t|), its float32 floor, taken from the
        # same definitions run in float32, bounds the comparison
        f0 = 0.0 if f32 is None else np.abs(f32[0].ravel() - gp.ravel()).max()
        f1 = 0.0 if f32 is None else np.abs(f32[1] - ref).max()
        np.testing.assert_allclose(out[:12], gp.ravel(), rtol=1e-3, atol=max(1e-3 * np.abs(gp).max(), 4.0 * f0))
        np.testing.assert_allclose(out[24:48], ref, rtol=1e-3, atol=max(1e-3 * np.abs(ref).max(), 4.0 * f1))
    assert n_cmp > 100


def test_closed_form_rigid_contact_reverses_match_the_oracles_autograd(H):
    """The closed-form reverses of the soft contact with a box and with a capsule gripper
    against the FP64 oracle's own rigid-contact response (Sec. 3.2) under autograd: the
    cotangents of the vertex position and velocity, and for the gripper of its position,
    linear and angular velocity."""
    from types import SimpleNamespace
    rng = np.random.default_rng(29)
    r, eps, mu = 0.002, 0.001, 0.5

    def fake(boxes=(), hl=0.02, rc=0.01):
        p = SimpleNamespace(eps_soft=eps / r, restitution=0.0, mu_rigid=mu, planes=[], boxes=list(boxes),
                            grip_half_len=hl, grip_radius=rc)
        return SimpleNamespace(p=p, dtype=torch.float64, _note=lambda *a: None)

    def group(ngrip):
        return dict(R=dict(r=torch.tensor([r], dtype=torch.float64), mass=torch.ones(1, 1, dtype=torch.float64)),
                    kind=torch.zeros(1, 1, dtype=torch.int64), ngrip=torch.tensor([ngrip]))

    n_box = 0
    hlb = np.array([0.15, 0.15, 0.05])
    for trial in range(300):
        x = rng.uniform(-1.0, 1.0, size=3) * hlb * 0.9
        for k in rng.choice(3, size=rng.integers(1, 4), replace=False):
            x[k] = rng.choice([-1.0, 1.0]) * (hlb[k] + rng.uniform(-0.003, 0.004))
        v, lo = rng.normal(size=3) * 0.3, rng.normal(size=3)
        out = call(H.box_rev_check, fl(np.concatenate([x, v, np.zeros(3), hlb, [r, eps, mu, 0.0], lo])), n_out=13)
        xt = torch.tensor(x[None, None], requires_grad=True)
        vt = torch.tensor(v[None, None], requires_grad=True)
        z = torch.zeros(1, 2, 3, dtype=torch.float64)
        vo = OracleSim.rigid_contact(fake(boxes=[np.concatenate([np.zeros(3), hlb])]), group(0), xt, vt, z,
                                     torch.eye(3, dtype=torch.float64).expand(1, 2, 3, 3), z, z)
        if out[12] == 0:
            continue
        n_box += 1
        gx, gv = torch.autograd.grad((vo * torch.tensor(lo)).sum(), [xt, vt])
        ref = np.concatenate([gx.numpy().ravel(), gv.numpy().ravel()])
        np.testing.assert_allclose(out[:6], ref, rtol=1e-3, atol=1e-3 * np.abs(ref).max())
    assert n_box > 50

    n_cap = 0
    for trial in range(300):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        # a frame whose third column is the capsule axis
        e1 = np.cross(ax, [1.0, 0.0, 0.0] if abs(ax[0]) < 0.9 else [0.0, 1.0, 0.0])
        e1 /= np.linalg.norm(e1)
        Rg = np.stack([e1, np.cross(ax, e1), ax], 1)
        x = rng.normal(size=3) * 0.006
        x[2] = abs(x[2]) + 0.009
        v, vp, w, lo = rng.normal(size=3) * 0.2, rng.normal(size=3) * 0.05, rng.normal(size=3), rng.normal(size=3)
        inp = fl(np.concatenate([x, v, np.zeros(3), ax, [0.02, 0.01], vp, w, [r, eps, mu, 0.0], lo]))
        out = call(H.capsule_rev_check, inp, n_out=37)
        if out[36] == 0:
            continue
        n_cap += 1
        xt = torch.tensor(x[None, None], requires_grad=True)
        vt = torch.tensor(v[None, None], requires_grad=True)
        p0 = torch.zeros(1, 2, 3, dtype=torch.float64, requires_grad=True)
        vpt = torch.tensor(np.stack([vp, np.zeros(3)])[None], requires_grad=True)
        wt = torch.tensor(np.stack([w, np.zeros(3)])[None], requires_grad=True)
        R0 = torch.tensor(np.stack([Rg, np.eye(3)])[None])
        vo = OracleSim.rigid_contact(fake(), group(1), xt, vt, p0, R0, vpt, wt)
        gx, gv, gp, gvp, gw = torch.autograd.grad((vo * torch.tensor(lo)).sum(), [xt, vt, p0, vpt, wt])
        ref = np.concatenate([gx.numpy().ravel(), gv.numpy().ravel(), gp[0, 0].numpy(), gvp[0, 0].numpy(),
                              gw[0, 0].numpy()])
        got = np.concatenate([out[0:3], out[3:6], out[6:9], out[12:15], out[15:18]])
        np.testing.assert_allclose(got, ref, rtol=1e-3, atol=1e-3 * np.abs(ref).max())
    assert n_cap > 20
