"""Pins of the FP64 oracle against closed forms, invariants and brute force.

None of these re-types the oracle's own formulas: each compares it with something the
paper or the mathematics fixes independently (closed-form energies of simple shapes,
Euler-Bernoulli statics, conservation laws, brute-force minimisation, discrete
Gauss-Bonnet for the loop holonomy, central finite differences of whole rollouts).
"""
import math
from pathlib import Path

import numpy as np
import pytest
import torch

from oracle import OracleSim, elastic_energy, closest_params, sdf_box, sdf_capsule
from oracle.dlo import build_frames, edges_of, hinge_sides, signed_angle, transport, unit, F64
from paper_2606_04206_gb300 import inputs


GOLDEN = Path(__file__).parent / "golden"


def straight(n, L, z=1.0):
    x = np.zeros((n, 3))
    x[:, 0] = np.linspace(0.0, L, n)
    x[:, 2] = z
    return x


def energy_forces(sim, gi=0):
    G, S = sim.groups[gi], sim.state[gi]
    x = S["x"].clone().requires_grad_(True)
    th = S["theta"].clone().requires_grad_(True)
    U = elastic_energy(x, th, S["tb"], S["d1b"], S["mprev"], S["kbar"], G["R"], G["closed"])
    gx, gth = torch.autograd.grad(U.sum(), [x, th])
    return U.detach(), -gx, -gth


def make(rods, x0=None, theta0=None, **kw):
    p = inputs.custom(rods, **kw)
    if x0 is not None:
        p.x0 = np.concatenate(x0)
    if theta0 is not None:
        p.theta0 = np.asarray(theta0, np.float64)
    sim = OracleSim(p)
    sim.set_state(p.x0, p.v0, p.theta0, p.omega0)
    return p, sim


R_, RHO = float(np.float32(0.002)), 1000.0     # inputs are float32-representable
A_ = math.pi * R_ ** 2


# ---------------------------------------------------------------------- P1 closed-form energies

def test_straight_rod_has_zero_energy_and_force():
    p, sim = make([straight(12, 0.5)], K=1e6, E=1e6, G=4e5)
    U, F, tau = energy_forces(sim)
    assert abs(float(U)) < 1e-20
    assert float(F.abs().max()) < 1e-12 and float(tau.abs().max()) < 1e-14


def test_uniform_stretch_energy():
    eps, L, K = 0.01, 0.5, 1e6
    p, sim = make([straight(12, L)], x0=[straight(12, L * (1 + eps))], K=K, E=1e6, G=4e5)
    U, _, _ = energy_forces(sim)
    A = math.pi * p.radius[0] ** 2
    eb = np.linalg.norm(np.diff(p.x_rest, axis=0), axis=1)
    e = np.linalg.norm(np.diff(p.x0, axis=0), axis=1)
    assert float(U) == pytest.approx((0.5 * K * A * (e / eb - 1) ** 2 * eb).sum(), rel=1e-10)
    assert float(U) == pytest.approx(0.5 * K * A_ * eps ** 2 * L, rel=1e-6)


def arc(n, l, Rc):
    phi = 2 * math.asin(l / (2 * Rc))
    a = np.arange(n) * phi
    return np.stack([Rc * np.sin(a), Rc * (1 - np.cos(a)), np.ones(n)], 1), phi


def test_planar_arc_bending_energy():
    n, l, Rc, E = 20, 0.01, 0.1, 1e6
    x, phi = arc(n, l, Rc)
    p, sim = make([straight(n, l * (n - 1))], x0=[x], K=1e6, E=E, G=4e5)
    U, _, _ = energy_forces(sim)
    kb = 2 * math.tan(phi / 2)
    eb = np.linalg.norm(np.diff(p.x_rest, axis=0), axis=1)
    lbar = 0.5 * (eb[1:] + eb[:-1])
    expect = 0.5 * (E * A_ * R_ ** 2 / 4) * (kb ** 2 / lbar).sum()
    assert float(U) == pytest.approx(expect, rel=1e-9)
    # continuum limit of a closed circle: U_b -> E I pi / R (checked at fine resolution)
    N = 400
    ang = np.arange(N) * 2 * math.pi / N
    circ = np.stack([Rc * np.cos(ang), Rc * np.sin(ang), np.ones(N)], 1)
    p2, sim2 = make([circ], closed=[True], K=1e6, E=E, G=0.0)
    G2 = sim2.groups[0]
    G2["R"]["kbar0"].zero_()
    sim2.state[0]["kbar"].zero_()
    U2, _, _ = energy_forces(sim2)
    EI = E * math.pi * R_ ** 4 / 4
    assert float(U2) == pytest.approx(EI * math.pi / Rc, rel=1e-3)


def test_uniform_twist_energy_and_end_torques():
    n, L, Gm = 10, 0.45, 4e5
    E = n - 1
    Phi = 0.7
    th = Phi * np.arange(E) / (E - 1)
    p, sim = make([straight(n, L)], theta0=th, K=1e6, E=1e6, G=Gm)
    U, F, tau = energy_forces(sim)
    eb = np.linalg.norm(np.diff(p.x_rest, axis=0), axis=1)
    lbar = 0.5 * (eb[1:] + eb[:-1])
    l = L / (n - 1)
    beta = Gm * A_ * R_ ** 2 / 2
    m = Phi / (E - 1)
    assert float(U) == pytest.approx(0.5 * beta * m ** 2 * (1 / lbar).sum(), rel=1e-10)
    t = tau[0].numpy()
    assert t[0] == pytest.approx(beta * m / lbar[0], rel=1e-10)
    assert t[-1] == pytest.approx(-beta * m / lbar[-1], rel=1e-10)
    np.testing.assert_allclose(t[1:-1], beta * m * (1 / lbar[1:] - 1 / lbar[:-1]), atol=1e-12 * beta * m / l)
    assert float(F.abs().max()) < 1e-10


# ---------------------------------------------------------------------- P2 derivatives

def test_force_matches_central_differences_of_energy():
    rng = np.random.default_rng(0)
    x = straight(7, 0.3) + rng.normal(scale=0.01, size=(7, 3))
    p, sim = make([straight(7, 0.3)], x0=[x], theta0=rng.normal(scale=0.3, size=6),
                  K=1e5, E=1e6, G=4e5)
    G, S = sim.groups[0], sim.state[0]
    U0, F, tau = energy_forces(sim)
    h = 1e-6

    def U_at(xx, tt):
        return float(elastic_energy(xx, tt, S["tb"], S["d1b"], S["mprev"], S["kbar"], G["R"], False))

    for (i, k) in [(0, 0), (2, 1), (3, 2), (6, 0)]:
        xp, xm = S["x"].clone(), S["x"].clone()
        xp[0, i, k] += h
        xm[0, i, k] -= h
        fd = -(U_at(xp, S["theta"]) - U_at(xm, S["theta"])) / (2 * h)
        assert fd == pytest.approx(float(F[0, i, k]), rel=1e-6, abs=1e-9)
    for j in [0, 3, 5]:
        tp, tm = S["theta"].clone(), S["theta"].clone()
        tp[0, j] += h
        tm[0, j] -= h
        fd = -(U_at(S["x"], tp) - U_at(S["x"], tm)) / (2 * h)
        assert fd == pytest.approx(float(tau[0, j]), rel=1e-6, abs=1e-12)


# ---------------------------------------------------------------------- P3 invariance

def rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, a, b, c = q
    return np.array([[1 - 2 * (b * b + c * c), 2 * (a * b - c * w), 2 * (a * c + b * w)],
                     [2 * (a * b + c * w), 1 - 2 * (a * a + c * c), 2 * (b * c - a * w)],
                     [2 * (a * c - b * w), 2 * (b * c + a * w), 1 - 2 * (a * a + b * b)]])


@pytest.mark.parametrize("closed", [False, True])
def test_rigid_motion_invariance_and_balance(closed):
    rng = np.random.default_rng(1)
    n = 14
    if closed:
        ang = np.arange(n) * 2 * math.pi / n
        x = np.stack([0.1 * np.cos(ang), 0.1 * np.sin(ang), 0.02 * np.sin(3 * ang)], 1)
    else:
        x = straight(n, 0.4) + rng.normal(scale=0.02, size=(n, 3))
    E = n if closed else n - 1
    p, sim = make([x], closed=[closed], theta0=rng.normal(scale=0.2, size=E),
                  K=1e5, E=1e6, G=4e5, plastic=True, yield_curv=1.0)
    sim.state[0]["kbar"] = sim.state[0]["kbar"] + torch.as_tensor(rng.normal(scale=0.05, size=sim.state[0]["kbar"].shape))
    U0, F, tau = energy_forces(sim)
    # net force and net moment vanish (moment includes twist torques about each tangent)
    assert float(F.sum(1).abs().max()) < 1e-10 * float(F.abs().max())
    S = sim.state[0]
    xs = S["x"][0]
    t = unit(edges_of(S["x"], closed))[0]
    M = torch.linalg.cross(xs, F[0], dim=-1).sum(0) + (tau[0][:, None] * t).sum(0)
    assert float(M.abs().max()) < 1e-10 * float((xs.norm(dim=1).max() * F.abs().max()))
    # rotate + translate the whole state: energy unchanged
    Q = torch.as_tensor(rand_rot(rng))
    c = torch.as_tensor(rng.normal(size=3))
    st = sim.get_state(as_numpy=False)
    rot = {k: v for k, v in st.items()}
    rot["x"] = st["x"] @ Q.T + c
    rot["tb"] = st["tb"] @ Q.T
    rot["d1b"] = st["d1b"] @ Q.T
    sim.set_full_state({k: v.numpy() for k, v in rot.items()})
    U1, _, _ = energy_forces(sim)
    assert float(U1) == pytest.approx(float(U0), rel=1e-12)


# ---------------------------------------------------------------------- P4 Euler-Bernoulli statics

@pytest.mark.parametrize("N", [16, 32, 64])
def test_cantilever_static_balance(N):
    """Euler-Bernoulli deflection w(s) = q s^2 (6L^2 - 4Ls + s^2) / (24 EI) of a clamped beam
    under its own weight: the oracle's internal forces at interior vertices must balance
    gravity, because the discrete bending force reproduces EI w'''' = q."""
    L, E = 0.2, 1e9
    EI = E * math.pi * R_ ** 4 / 4
    q = RHO * A_ * 9.81
    s = np.linspace(0, L, N)
    w = q * s ** 2 * (6 * L ** 2 - 4 * L * s + s ** 2) / (24 * EI)
    x = np.stack([s, np.zeros(N), 1.0 - w], 1)
    pinned = np.zeros(N, bool)
    pinned[:2] = True
    p, sim = make([straight(N, L)], x0=[x], E=E, G=0.4 * E, inextensible=True, pinned=pinned)
    _, F, _ = energy_forces(sim)
    m = sim.groups[0]["R"]["mass"][0]
    resid = (F[0, :, 2] - m * 9.81).numpy()
    inner = slice(3, N - 3)
    rel = np.abs(resid[inner]).max() / float(m[inner].max() * 9.81)
    assert rel < 0.02, rel
    # the tip deflection itself is the classical q L^4 / (8 EI)
    assert w[-1] == pytest.approx(q * L ** 4 / (8 * EI), rel=1e-12)


# ---------------------------------------------------------------------- P5 energy behaviour

@pytest.mark.slow
def test_energy_conservation_symplectic_euler():
    n, L = 10, 0.3
    x = straight(n, L)
    pinned = np.zeros(n, bool)
    pinned[0] = True
    drift = []
    for nmin in (10, 20):
        p = inputs.custom([x], frames=60, K=1e6, E=1e5, G=4e4, damping=0.0, pinned=pinned,
                          substeps_min=nmin)
        p.theta0 = np.linspace(0, 0.5, n - 1)
        sim = OracleSim(p)
        sim.set_state(p.x0, p.v0, p.theta0, p.omega0)
        e0 = sim.energies().sum()
        hist = []
        for f in range(60):
            sim.step(p.actions[f:f + 1], 1)
            hist.append(sim.energies().sum())
        hist = np.array(hist)
        scale = abs(sim.energies()[0, 2] - e0) + 1e-30
        drift.append(np.abs(hist - e0).max())
        # no secular drift: the last third stays within the band of the first two thirds
        assert np.abs(hist[40:] - e0).max() < 2.0 * np.abs(hist[:40] - e0).max() + 1e-12
    ratio = drift[0] / drift[1]
    assert 1.4 < ratio < 2.8, ratio     # first-order: halving h halves the energy error


# ---------------------------------------------------------------------- P6 inextensibility

def test_inextensibility_single_edge_exact_and_momentum():
    x = straight(2, 0.1)
    p, sim = make([x], x0=[x * np.array([1.5, 1, 1])], inextensible=True, E=1e4)
    G, S = sim.groups[0], sim.state[0]
    xs = sim.inext_sweep(G, S["x"], G["colors"][0])
    rest = float(np.linalg.norm(p.x_rest[1] - p.x_rest[0]))
    assert float((xs[0, 1] - xs[0, 0]).norm()) == pytest.approx(rest, rel=1e-14)
    m = G["R"]["mass"][0]
    assert float(((xs[0] - S["x"][0]) * m[:, None]).sum(0).abs().max()) < 1e-18


def test_inextensibility_residual_decreases_with_iterations():
    rng = np.random.default_rng(3)
    n = 20
    x = straight(n, 0.5)
    p, sim = make([x], x0=[x + rng.normal(scale=0.004, size=x.shape)], inextensible=True, E=1e4)
    G, S = sim.groups[0], sim.state[0]
    xs = S["x"]
    eb = G["R"]["ebar"][0]
    res = []
    for it in range(8):
        res.append(float(((edges_of(xs, False)[0].norm(dim=-1) - eb).abs() / eb).max()))
        for col in G["colors"]:
            xs = sim.inext_sweep(G, xs, col)
    assert all(b < a for a, b in zip(res, res[1:])), res
    m = G["R"]["mass"][0]
    assert float(((xs[0] - S["x"][0]) * m[:, None]).sum(0).abs().max()) < 1e-16


# ---------------------------------------------------------------------- P7 momentum in contact

@pytest.mark.parametrize("inclined", [False, True])
def test_momentum_conserved_through_self_contact(inclined):
    """The paper reports a total momentum error of 1e-13 .. 1e-14 in 'parallel' and
    'inclined' contact (App. C, tests/golden/momentum_contact.txt); an inverse-mass-weighted
    projection conserves it to rounding."""
    n = 30
    l = 0.01
    # hairpin: two arms joined by a half-turn; arms 3.5 mm apart (r = 2 mm, so they overlap)
    arm = np.arange(12) * l
    gap = 0.0035
    a1 = np.stack([arm, np.zeros(12), np.zeros(12)], 1)
    turn_ang = np.linspace(-math.pi / 2, math.pi / 2, 8)[1:-1]
    rt = gap / 2
    turn = np.stack([arm[-1] + 0.003 + rt * np.cos(turn_ang) * 0 + 0.004 * np.cos(turn_ang),
                     rt + rt * np.sin(turn_ang), np.zeros(6)], 1)
    a2 = a1[::-1] + np.array([0, gap, 0])
    if inclined:
        a2 = a2 + np.stack([np.zeros(12), np.zeros(12), np.linspace(0.004, -0.004, 12)], 1)
    x = np.concatenate([a1, turn, a2])[:n]
    rng = np.random.default_rng(5)
    p = inputs.custom([x], frames=15, K=1e5, E=1e4, G=1e3, damping=0.0, gravity=0.0,
                      self_contact=True)
    p.v0 = rng.normal(scale=0.05, size=x.shape)
    sim = OracleSim(p)
    sim.set_state(p.x0, p.v0, p.theta0, p.omega0)
    P0 = sim.momentum()[0]
    pairs = sim.candidates(sim.groups[0], sim.state[0]["x"])
    assert pairs[0].shape[0] > 0
    errs = []
    for f in range(15):
        sim.step(p.actions[f:f + 1], 1)
        errs.append(np.abs(sim.momentum()[0] - P0).max())
    bound = float(open(GOLDEN / "momentum_contact.txt").read().split("max_total_momentum_error")[1].split()[0])
    assert max(errs) < bound, errs


# ---------------------------------------------------------------------- self-contact friction

@pytest.mark.parametrize("seed", range(6))
def test_self_contact_friction_obeys_coulomb(seed):
    """Self-contact friction (App. A.1: Coulomb friction whose normal impulse is approximated
    from the penetration depth d; reading O15 takes the normal velocity change as d/h).
    Physical checks on one crossing pair with random inverse masses and velocities:
    the impulse is tangential, so the normal relative velocity is unchanged; it opposes
    sliding and never reverses it; its size is the Coulomb bound mu d/h while sliding
    continues, and sliding stops exactly when that bound covers the tangential speed; it
    conserves linear momentum and does not add kinetic energy."""
    rng = np.random.default_rng(100 + seed)
    # edge 1 along x at z = 0; edge 6 crosses above it along y at a height below 2r, at
    # random points of both edges (so that the barycentric weights differ from 1/2)
    zc = rng.uniform(0.4, 0.95) * 2 * R_
    xc, ya = rng.uniform(0.003, 0.017), rng.uniform(0.003, 0.017)
    x = np.array([[-0.02, 0, 0], [0, 0, 0], [0.02, 0, 0], [0.03, 0.01, 0.01], [0.02, 0.03, 0.01],
                  [xc, ya + 0.01, zc], [xc, ya, zc], [xc + 0.001, ya - 0.02, zc], [xc + 0.001, ya - 0.04, zc]])
    p = inputs.custom([x], K=1e5, E=1e4, self_contact=True)
    sim = OracleSim(p)
    G = dict(sim.groups[0])
    R = dict(G["R"])
    R["w"] = torch.as_tensor(rng.uniform(0.5, 2.0, size=(1, len(x))) * 1e3, dtype=F64)
    G["R"] = R
    xs = torch.as_tensor(x, dtype=F64)[None]
    _, infos = sim.contact_sweep(G, xs, [torch.tensor([[1, 6]])])
    I = infos[0]
    assert bool(I["act"][0])
    s_, u_, n_, d = float(I["s"][0]), float(I["u"][0]), I["n"][0].numpy(), float(I["d"][0])
    h = 2e-4
    mu = p.mu_self
    idx = [1, 2, 6, 7]
    bary = np.array([1 - s_, s_, -(1 - u_), -u_])
    m = 1.0 / R["w"][0].numpy()

    def rel(v):
        return sum(b * v[i] for b, i in zip(bary, idx))

    for trial in range(8):
        v = rng.normal(size=(len(x), 3)) * 0.05
        # relative tangential speed well above or well below the Coulomb bound mu d / h
        vt_target = mu * d / h * (rng.uniform(1.5, 4.0) if trial % 2 == 0 else rng.uniform(0.1, 0.7))
        vr = rel(v)
        vt = vr - np.dot(vr, n_) * n_
        # rescale the tangential part of the relative velocity by moving vertex 2 (weight s)
        v[2] += (vt_target / np.linalg.norm(vt) - 1.0) * vt / s_
        vr = rel(v)
        vt = vr - np.dot(vr, n_) * n_
        assert np.linalg.norm(vt) == pytest.approx(vt_target, rel=1e-9)
        out = sim.self_friction(G, torch.as_tensor(v, dtype=F64)[None], infos, h)[0].numpy()
        vr2 = rel(out)
        vt2 = vr2 - np.dot(vr2, n_) * n_
        # tangential impulse: normal relative velocity unchanged
        assert np.dot(vr2, n_) == pytest.approx(np.dot(vr, n_), abs=1e-12)
        # opposes sliding without reversing it: vt2 = c vt with 0 <= c <= 1
        c = np.dot(vt2, vt) / np.dot(vt, vt)
        assert np.linalg.norm(vt2 - c * vt) < 1e-12 * np.linalg.norm(vt)
        assert -1e-12 <= c <= 1.0 + 1e-12
        dvt = np.linalg.norm(vt - vt2)
        if np.linalg.norm(vt) > mu * d / h:      # sliding: the Coulomb bound is reached
            assert dvt == pytest.approx(mu * d / h, rel=1e-9)
        else:                                     # sticking: the relative sliding stops
            assert np.linalg.norm(vt2) < 1e-12
        # momentum conserved, no kinetic energy added
        np.testing.assert_allclose((m[:, None] * (out - v)).sum(0), 0.0, atol=1e-15)
        assert (m * (out ** 2).sum(1)).sum() <= (m * (v ** 2).sum(1)).sum() * (1 + 1e-12)


# ---------------------------------------------------------------------- P8 plasticity

def test_plastic_return_reaches_yield_surface():
    n = 8
    p, sim = make([straight(n, 0.3)], E=1e4, plastic=True, yield_curv=2.0, creep_rate=1.0)
    G = sim.groups[0]
    rng = np.random.default_rng(2)
    kappa = torch.as_tensor(rng.normal(scale=0.07, size=(1, n - 2, 2)))
    kbar = torch.zeros_like(kappa)
    new = sim.plastic_update(G, kappa, kbar)
    thr = (G["R"]["sy"][:, None] * G["R"]["lbar"]).numpy()[0]
    el = (kappa - new).norm(dim=-1).numpy()[0]
    yielded = kappa.norm(dim=-1).numpy()[0] > thr
    assert yielded.any() and (~yielded).any()
    np.testing.assert_allclose(el[yielded], thr[yielded], rtol=1e-12)
    assert torch.equal(new[0, ~torch.as_tensor(yielded)], kbar[0, ~torch.as_tensor(yielded)])


@pytest.mark.slow
def test_bend_and_release_keeps_plastic_shape():
    """A clamped wire sagging under its own weight past yield keeps a bent rest shape after
    the load is removed (App. A.1: 'retain a new intrinsic shape'); an elastic one springs
    back straight."""
    n, L, F = 10, 0.3, 250
    pinned = np.zeros(n, bool)
    pinned[:2] = True
    res = {}
    for plastic in (False, True):
        p = inputs.custom([straight(n, L)], frames=F, K=1e7, E=1e8, G=0.0, plastic=plastic,
                          yield_curv=1.0, damping=20.0, pinned=pinned)
        sim = OracleSim(p)
        sim.set_state(p.x0, p.v0, p.theta0, p.omega0)
        sim.step(p.actions, F)              # sag under gravity
        loaded = 1.0 - sim.get_state()["x"][-1, 2]
        sim.p.gravity = 0.0
        sim.step(p.actions, F)              # remove the load, damp to rest
        st = sim.get_state()
        res[plastic] = (loaded, 1.0 - st["x"][-1, 2], np.abs(st["kbar"]).max())
        sim.p.gravity = 9.81
    assert res[False][2] == 0.0
    assert res[False][1] < 0.05 * res[False][0]     # elastic rod springs back
    assert res[True][1] > 0.3 * res[True][0]        # plastic rod keeps most of its sag
    assert res[True][2] > 0.0


# ---------------------------------------------------------------------- P9 loop holonomy

def tantrix_area(t):
    """Signed area of the spherical polygon t_0..t_{E-1} (fan triangulation, Van Oosterom &
    Strackee solid angle of each triangle)."""
    a = t[0]
    tot = 0.0
    for j in range(1, len(t) - 1):
        b, c = t[j], t[j + 1]
        num = a @ np.cross(b, c)
        den = 1 + a @ b + b @ c + c @ a
        tot += 2 * math.atan2(num, den)
    return tot


def test_planar_loop_has_no_holonomy():
    N = 24
    ang = np.arange(N) * 2 * math.pi / N
    x = np.stack([0.1 * np.cos(ang) + 0.03 * np.cos(3 * ang), 0.1 * np.sin(ang), np.zeros(N)], 1)
    _, _, psi = build_frames(torch.as_tensor(x)[None], True)
    assert abs(float(psi)) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_loop_holonomy_matches_tantrix_area_and_closes(seed):
    rng = np.random.default_rng(seed)
    N = 40
    s = np.arange(N) * 2 * math.pi / N
    c = rng.uniform(0.3, 1.0, 3)
    x = np.stack([np.cos(s) + c[0] * np.cos(2 * s), np.sin(s) + c[1] * np.sin(3 * s), c[2] * np.sin(2 * s + 1)], 1) * 0.1
    X = torch.as_tensor(x)[None]
    t, d1, psi = build_frames(X, True)
    area = tantrix_area(t[0].numpy())
    # discrete Gauss-Bonnet: transport around the tangent indicatrix rotates a vector
    # counter-clockwise by the (right-hand signed) area it encloses, modulo 2 pi
    diff = (float(psi) - area + math.pi) % (2 * math.pi) - math.pi
    assert abs(diff) < 1e-9, (float(psi), area)
    # after the correction every hinge carries the same reference twist -psi/N_e
    ta, tb = hinge_sides(t, True)
    ra, rb = hinge_sides(d1, True)
    ang = signed_angle(transport(ta, tb, ra), rb, tb)[0].numpy()
    np.testing.assert_allclose(ang, -float(psi) / N, atol=1e-12)


# ---------------------------------------------------------------------- P10 closest points

def test_closest_points_brute_force():
    rng = np.random.default_rng(4)
    g = np.linspace(0, 1, 2001)
    for trial in range(6):
        P = rng.normal(size=(4, 3))
        if trial == 5:                        # parallel segments
            P[3] = P[2] + (P[1] - P[0]) * 0.7
        p1, q1, p2, q2 = (torch.as_tensor(v) for v in P)
        s, u = closest_params(p1, q1, p2, q2)
        d = float(((p1 + s * (q1 - p1)) - (p2 + u * (q2 - p2))).norm())
        A = P[0][None] + g[:, None] * (P[1] - P[0])[None]
        Bp = P[2][None] + g[:, None] * (P[3] - P[2])[None]
        # coarse grid minimum, then exact minimisation of the quadratic along each clamp face
        D = np.linalg.norm(A[:, None] - Bp[None], axis=2)
        i, j = np.unravel_index(D.argmin(), D.shape)
        best = D[i, j]
        assert d <= best + 1e-12
        assert d == pytest.approx(best, abs=2e-6 * np.linalg.norm(P[1] - P[0]) + 2e-6 * np.linalg.norm(P[3] - P[2]))


# ---------------------------------------------------------------------- P12 SDF primitives

def test_box_and_capsule_sdf_against_sampling():
    rng = np.random.default_rng(6)
    c = np.array([0.1, -0.2, 0.05])
    hl = np.array([0.15, 0.1, 0.05])
    pts = c + rng.uniform(-2, 2, size=(200, 3)) * hl
    sdf, n = sdf_box(torch.as_tensor(pts), torch.as_tensor(c), torch.as_tensor(hl))
    # exact distance to the surface: nearest point on each of the six face rectangles
    best = np.full(len(pts), np.inf)
    for ax in range(3):
        for sgn in (-1, 1):
            q = np.clip(pts - c, -hl, hl)
            q[:, ax] = sgn * hl[ax]
            best = np.minimum(best, np.linalg.norm(pts - c - q, axis=1))
    inside = np.all(np.abs(pts - c) < hl, axis=1)
    np.testing.assert_allclose(np.abs(sdf.numpy()), best, atol=1e-14)
    assert np.array_equal(sdf.numpy() < 0, inside)
    # gradient = finite-difference gradient of the SDF
    h = 1e-7
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (sdf_box(torch.as_tensor(pts + e), torch.as_tensor(c), torch.as_tensor(hl))[0]
              - sdf_box(torch.as_tensor(pts - e), torch.as_tensor(c), torch.as_tensor(hl))[0]) / (2 * h)
        np.testing.assert_allclose(fd.numpy(), n[:, k].numpy(), atol=1e-6)
    # capsule against sampling of its axis
    a, b, rc = np.array([0.0, 0, 0]), np.array([0.0, 0, 0.04]), 0.01
    axis = a + np.linspace(0, 1, 4001)[:, None] * (b - a)
    q = rng.uniform(-0.05, 0.08, size=(100, 3))
    sd, nn = sdf_capsule(torch.as_tensor(q), torch.as_tensor(a), torch.as_tensor(b), rc)
    ref = np.linalg.norm(q[:, None] - axis[None], axis=2).min(1) - rc
    np.testing.assert_allclose(sd.numpy(), ref, atol=1e-7)


# ---------------------------------------------------------------------- rigid contact response

def test_rigid_contact_removes_approach_and_applies_coulomb_friction():
    """Vertex at the ground surface (d = 0, so f = 1) moving down and sideways: the normal
    approach velocity is removed (restitution 0) and the tangential speed drops by mu times
    the normal velocity change (Coulomb)."""
    x = straight(3, 0.02, z=R_)
    p = inputs.custom([x], K=1e5, E=1e4, planes=np.array([[0, 0, 1.0, 0.0]]))
    sim = OracleSim(p)
    sim.set_state(p.x0, p.v0, p.theta0, p.omega0)
    G, S = sim.groups[0], sim.state[0]
    v = torch.zeros(1, 3, 3, dtype=F64)
    v[0, :, 2] = -0.1
    v[0, :, 0] = 0.2
    out = sim.rigid_contact(G, S["x"], v, None, None, None, None)
    np.testing.assert_allclose(out[0, :, 2].numpy(), 0.0, atol=1e-15)
    np.testing.assert_allclose(out[0, :, 0].numpy(), 0.2 - 0.5 * 0.1, rtol=1e-12)
    # far above the plane (f below 0.1) nothing changes
    S2 = S["x"].clone()
    S2[..., 2] = 0.05
    out2 = sim.rigid_contact(G, S2, v, None, None, None, None)
    assert torch.equal(out2, v)


# ---------------------------------------------------------------------- substep count

@pytest.mark.parametrize("mat", [dict(K=1e8, E=1e8, G=4e7), dict(K=1e5, E=1e4, G=1e3),
                                 dict(K=1e4, E=1e8, G=4e3), dict(K=0.0, E=1e6, G=4e5, inextensible=True)])
def test_substep_count_keeps_symplectic_euler_stable(mat):
    """The per-rod substep count must put h * omega_max below the symplectic-Euler limit 2,
    where omega_max is the largest natural frequency of the linearised rod (generalised
    eigenvalues of the oracle energy's Hessian against the lumped masses and inertias)."""
    assert OracleSim(inputs.plain(2)).nsub == [5]
    n = 16
    p, sim = make([straight(n, 0.05)], substeps_min=1, **mat)
    G, S = sim.groups[0], sim.state[0]
    R = G["R"]

    def U(z):
        x = z[: 3 * n].reshape(1, n, 3)
        th = z[3 * n:].reshape(1, n - 1)
        return elastic_energy(x, th, S["tb"], S["d1b"], S["mprev"], S["kbar"], R, False).sum()

    z0 = torch.cat([S["x"].reshape(-1), S["theta"].reshape(-1)])
    H = torch.autograd.functional.hessian(U, z0).numpy()
    minv = np.concatenate([np.repeat(1.0 / R["mass"][0].numpy(), 3), 1.0 / R["inertia"][0].numpy()])
    lam = np.linalg.eigvals(np.sqrt(minv)[:, None] * H * np.sqrt(minv)[None]).real.max()
    h = 1e-3 / sim.nsub[0]
    w = math.sqrt(max(lam, 0.0))
    assert h * w < 2.0, (sim.nsub, h * w)
    assert h * w > 0.3, (sim.nsub, h * w)


# ---------------------------------------------------------------------- P14 rollout gradient

@pytest.mark.slow
def test_rollout_gradient_matches_central_differences():
    """Autograd through the whole oracle rollout (forces, plasticity, gripper kinematics,
    ground contact, inextensibility) against FP64 central differences, h = 1e-6."""
    rng = np.random.default_rng(9)
    n = 7
    rods = [straight(n, 0.18, z=0.03) + rng.normal(scale=0.004, size=(n, 3)) for _ in range(2)]
    acts = rng.normal(scale=0.002, size=(4, 2, 2, 6))
    gp = np.stack([np.stack([r[2], r[4]]) for r in rods])
    p = inputs.custom(rods, frames=4, actions=acts, n_grippers=[2, 2], grip_pos=gp,
                      K=[1e5, 0.0], E=[2e3, 1e3], G=[1e2, 0.0], inextensible=[False, True],
                      plastic=[True, False], yield_curv=[0.2, 0.0], damping=1.0,
                      planes=np.array([[0, 0, 1.0, 0.0]]), grip_radius=0.004, grip_half_len=0.006)
    target = rng.normal(size=(2 * n, 3))

    def loss(x0, v0, th0, act, E, sy):
        sim = OracleSim(p, params={"E": E, "yield_curv": sy})
        sim.set_state(x0, v0, th0, torch.zeros_like(th0))
        sim.step(act, 4, diff=True)
        st = sim.get_state(as_numpy=False)
        return (st["x"] * torch.as_tensor(target)).sum() + 0.1 * (st["theta"] ** 2).sum()

    args = [torch.as_tensor(p.x0), torch.as_tensor(p.v0) + 0.01, torch.as_tensor(p.theta0) + 0.05,
            torch.as_tensor(p.actions), torch.as_tensor(p.E), torch.as_tensor(p.yield_curv)]
    leaves = [a.clone().requires_grad_(True) for a in args]
    L = loss(*leaves)
    grads = torch.autograd.grad(L, leaves)
    h = 1e-6
    picks = [(0, (3, 2)), (0, (9, 0)), (1, (4, 1)), (2, (2,)), (3, (1, 0, 1, 0)), (3, (2, 1, 0, 4)),
             (4, (0,)), (5, (0,))]
    scale = {4: 1e3, 5: 0.2}
    for ai, idx in picks:
        hh = h * scale.get(ai, 1.0)
        ap = [a.clone() for a in args]
        am = [a.clone() for a in args]
        ap[ai][idx] += hh
        am[ai][idx] -= hh
        fd = (float(loss(*ap).detach()) - float(loss(*am).detach())) / (2 * hh)
        g = float(grads[ai][idx])
        assert g == pytest.approx(fd, rel=2e-4, abs=1e-8 * max(1.0, abs(fd))), (ai, idx, g, fd)


# ---------------------------------------------------------------------- self-contact projection

def crossing_pair(rng):
    """Nine vertices: edge 1 (vertices 1-2) along x at z = 0, edge 6 (vertices 6-7) crossing
    it along y at a random height below the contact distance 2r, above random points of both
    edges (so that the barycentric weights differ from 1/2)."""
    zc = rng.uniform(0.2, 0.95) * 2 * R_
    xc, ya = rng.uniform(0.003, 0.017), rng.uniform(0.003, 0.017)
    return np.array([[-0.02, 0, 0], [0, 0, 0], [0.02, 0, 0], [0.03, 0.01, 0.01], [0.02, 0.03, 0.01],
                     [xc, ya + 0.01, zc], [xc, ya, zc], [xc + 0.001, ya - 0.02, zc],
                     [xc + 0.001, ya - 0.04, zc]])


@pytest.mark.parametrize("seed", range(6))
def test_self_contact_projection_single_pair(seed):
    """One self-collision projection (App. A.1) of a single crossing pair with random inverse
    masses.  With the closest-point parameters (t, u) held at their pre-projection values the
    separation of the two segment points is linear in the correction, so after one projection
    they sit exactly r_a + r_b = 2r apart, along the line they were on.  The correction is
    also the smallest one, in the mass-weighted norm, that moves the two points apart to 2r
    along that line: the minimum-norm solution of one linear equation, found here by a
    library least-squares solve.  One vertex held fixed (w = 0) leaves the others to do all
    of it; a pair already 2r apart does not move."""
    rng = np.random.default_rng(300 + seed)
    x = crossing_pair(rng)
    p = inputs.custom([x], K=1e5, E=1e4, self_contact=True)
    sim = OracleSim(p)
    G = dict(sim.groups[0])
    R = dict(G["R"])
    w = rng.uniform(0.5, 2.0, size=len(x)) * 1e3
    if seed % 3 == 2:
        w[7] = 0.0                                  # a pinned vertex on the b side
    R["w"] = torch.as_tensor(w[None], dtype=F64)
    G["R"] = R
    idx = [1, 2, 6, 7]
    t_, u_ = (float(a) for a in closest_params(*(torch.as_tensor(x[i], dtype=F64) for i in idx)))
    beta = np.array([1 - t_, t_, -(1 - u_), -u_])
    sep0 = sum(b * x[i] for b, i in zip(beta, idx))
    assert np.linalg.norm(sep0) < 2 * R_
    out = sim.contact_sweep(G, torch.as_tensor(x, dtype=F64)[None], [torch.tensor([[1, 6]])])[0][0].numpy()
    dx = out - x
    # only the pair's four vertices move
    others = [i for i in range(len(x)) if i not in idx]
    assert np.abs(dx[others]).max() == 0.0
    # the two points at the fixed (t, u) are exactly 2r apart, on the line they were on
    sep1 = sum(b * out[i] for b, i in zip(beta, idx))
    assert np.linalg.norm(sep1) == pytest.approx(2 * R_, rel=1e-12)
    n0 = sep0 / np.linalg.norm(sep0)
    np.testing.assert_allclose(sep1 / np.linalg.norm(sep1), n0, atol=1e-12)
    # minimum mass-weighted correction: y = sqrt(m) dx minimises |y| subject to
    # n0 . sum_i beta_i dx_i = 2r - |sep0|  (w = 0 vertices: fixed, left out of the solve)
    free = [k for k, i in enumerate(idx) if w[i] > 0]
    row = np.concatenate([beta[k] * n0 / math.sqrt(1.0 / w[idx[k]]) for k in free])[None]
    y = np.linalg.lstsq(row, np.array([2 * R_ - np.linalg.norm(sep0)]), rcond=None)[0]
    want = np.zeros((4, 3))
    for j, k in enumerate(free):
        want[k] = y[3 * j:3 * j + 3] / math.sqrt(1.0 / w[idx[k]])
    np.testing.assert_allclose(dx[idx], want, rtol=1e-10, atol=1e-16)
    # a pair that is already 2r apart stays where it is
    x2 = x.copy()
    x2[5:] += (2 * R_ - np.linalg.norm(sep0) + 1e-6) * n0 * np.sign(n0[2])
    out2 = sim.contact_sweep(G, torch.as_tensor(x2, dtype=F64)[None], [torch.tensor([[1, 6]])])[0][0].numpy()
    assert np.array_equal(out2, x2)


# ---------------------------------------------------------------------- gripper kinematics

def rotvec_matrix(phi):
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(np.asarray(phi, np.float64)).as_matrix()


@pytest.mark.parametrize("motion", ["translation", "rotation", "both"])
def test_gripper_kinematics_closed_form(motion):
    """Grasped vertices are kinematic and follow their gripper rigidly (Sec. 3.2).  Under a
    constant per-frame action (dp, dphi) the gripper pose after f frames (and at the end of
    substep s of frame f, c = f + (s + 1)/n) is p0 + c dp and exp(c dphi) R0: repeated
    rotations about one axis add up.  A grasped vertex therefore sits at
    p0 + c dp + Rot(c dphi) (x_rest - p0), with Rot from a library rotation-vector map.
    R0 is a random rotation, so body and world frames differ."""
    rng = np.random.default_rng({"translation": 1, "rotation": 2, "both": 3}[motion])
    n = 8
    x = straight(n, 0.35, z=0.3)                 # 5 cm edges: one vertex per gripper grasped
    R0 = np.stack([rotvec_matrix(rng.normal(size=3)) for _ in range(2)])
    # gripper centres 1 cm from the grasped vertices (inside the 1 cm capsule's reach), so the
    # grasp offsets are not zero and the rotation moves the vertices
    off = rng.normal(size=(2, 3))
    gp = np.stack([x[2], x[5]]) + 0.01 * off / np.linalg.norm(off, axis=1, keepdims=True)
    dp = rng.normal(scale=0.002, size=(2, 3)) * (motion != "rotation")
    dphi = rng.normal(scale=0.02, size=(2, 3)) * (motion != "translation")
    frames = 4
    acts = np.zeros((frames, 1, 2, 6))
    acts[:, 0, :, :3] = dp
    acts[:, 0, :, 3:] = dphi
    p = inputs.custom([x], frames=frames, actions=acts, n_grippers=[2], grip_pos=gp[None], grip_rot=R0[None],
                      K=1e5, E=1e4, G=1e3, gravity=0.0)
    # inputs are rounded to float32: take the rounded values as the closed form's data
    # (the rounded R0 is orthogonal only to ~1e-7, so the offset R0^T (x - p0) maps back with
    # R0 R0^T, which the closed form carries explicitly)
    dp, dphi, gp, R0, x = p.actions[0, 0, :, :3], p.actions[0, 0, :, 3:], p.grip_pos[0], p.grip_rot[0], p.x_rest
    RRt = R0 @ np.transpose(R0, (0, 2, 1))
    sim = OracleSim(p)
    sim.set_state(p.x0, p.v0, p.theta0, p.omega0)
    G, S = sim.groups[0], sim.state[0]
    kind = G["kind"][0].numpy()
    assert [int(i) for i in np.nonzero(kind)[0]] == [2, 5] and kind[2] == 2 and kind[5] == 3
    n_sub = G["nsub"]
    act = torch.as_tensor(p.actions[0], dtype=F64)[None]
    for f in range(frames):
        for s in range(n_sub):
            S = sim.substep(G, S, act[0], s)
            c = f + (s + 1) / n_sub
            for g, vi in enumerate((2, 5)):
                want = gp[g] + c * dp[g] + rotvec_matrix(c * dphi[g]) @ RRt[g] @ (x[vi] - gp[g])
                np.testing.assert_allclose(S["x"][0, vi].numpy(), want, rtol=0, atol=1e-13)
        S = dict(S)
        S["gp"] = S["gp"] + act[0, ..., :3]
        from oracle.dlo import expmap
        S["gR"] = expmap(act[0, ..., 3:]) @ S["gR"]
    # the frame-level pose update (OracleSim.frame) gives the same closed form
    sim2 = OracleSim(p)
    sim2.set_state(p.x0, p.v0, p.theta0, p.omega0)
    sim2.step(p.actions, frames)
    st = sim2.get_state()
    for g, vi in enumerate((2, 5)):
        np.testing.assert_allclose(st["gp"][0, g], gp[g] + frames * dp[g], rtol=0, atol=1e-14)
        np.testing.assert_allclose(st["gR"][0, g], rotvec_matrix(frames * dphi[g]) @ R0[g], rtol=0, atol=1e-13)
        want = gp[g] + frames * dp[g] + rotvec_matrix(frames * dphi[g]) @ RRt[g] @ (x[vi] - gp[g])
        np.testing.assert_allclose(st["x"][vi], want, rtol=0, atol=1e-13)


# ---------------------------------------------------------------------- damping

def test_damping_decays_velocity_and_twist_rate_geometrically():
    """Mass-proportional damping (reading O8: force -c_d m v, torque -c_d I omega) under
    symplectic Euler.  A straight free rod with no gravity and no contact, moving as a rigid
    translation with a uniform twist rate, feels no elastic force or torque, so each substep
    multiplies v and omega by exactly (1 - h c_d): after n substeps they are
    (1 - h c_d)^n times their start values, and the positions have moved by the geometric sum
    h v0 sum_{k=1..n} (1 - h c_d)^k."""
    n = 12
    x = straight(n, 0.4, z=0.5)
    cd = 7.0
    p = inputs.custom([x], frames=6, K=1e5, E=1e4, G=1e3, damping=cd, gravity=0.0)
    v0 = np.array([0.12, -0.05, 0.08])
    p.v0 = np.tile(v0, (n, 1))
    p.omega0 = np.full(n - 1, 3.0)
    sim = OracleSim(p)
    sim.set_state(p.x0, p.v0, p.theta0, p.omega0)
    h = p.dt / sim.nsub[0]
    q = 1.0 - h * float(p.damping[0])
    for f in range(1, 7):
        sim.step(p.actions[f - 1:f], 1)
        k = f * sim.nsub[0]
        st = sim.get_state()
        np.testing.assert_allclose(st["v"], np.tile(q ** k * v0, (n, 1)), rtol=1e-9)
        np.testing.assert_allclose(st["omega"], np.full(n - 1, q ** k * 3.0), rtol=1e-12)
        moved = h * v0 * q * (1.0 - q ** k) / (1.0 - q)
        np.testing.assert_allclose(st["x"] - p.x0, np.tile(moved, (n, 1)), rtol=1e-9, atol=1e-15)


def test_no_twist_stiffness_means_no_twist_dynamics():
    """Reading O41: a rod with G = 0 (the parameter table's "Twisting -" rows) has no twist
    dynamics; its twist angles and rates keep their start values (here zero) while the rod
    bends and swings in 3D.  With a twist modulus that is tiny but positive, the same rod's
    twist angles move under the bending-twist coupling alone, so the pin is not trivially
    satisfied by the frames."""
    n = 16
    s = np.linspace(0.0, 1.0, n)
    x = np.stack([0.3 * s, 0.1 * np.sin(3 * s), 0.5 + 0.05 * np.cos(4 * s)], 1)   # curved, non-planar
    out = {}
    for G in (0.0, 1e-9):
        p = inputs.custom([x], frames=20, K=1e5, E=1e4, G=G)
        sim = OracleSim(p)
        sim.set_state(p.x0, p.v0, p.theta0, p.omega0)
        sim.step(p.actions, 20)
        out[G] = sim.get_state()
    assert np.all(out[0.0]["theta"] == 0.0) and np.all(out[0.0]["omega"] == 0.0)
    assert np.abs(out[1e-9]["theta"]).max() > 1e-12      # exactly zero only without dynamics
    assert np.abs(out[0.0]["x"] - x).max() > 1e-3        # the rod did move
