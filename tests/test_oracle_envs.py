"""Pins of the oracle's environments of several DLOs (Sec. 4: Separation's two ropes; the
self-collision projection and friction of App. A.1 applied between DLOs).

An environment is one record whose vertices are its DLOs ("strands") back to back.  The pins:

* strands far apart step exactly like the same DLOs stepped as separate rods (masses,
  frames, energies, plasticity and length projections stay within a strand);
* the elastic energy of a record is the sum of its strands' energies at any configuration,
  also one where two strands' ends coincide (the edge between them has length 0);
* segments of different strands collide even when their indices are adjacent, and the
  edge between two strands is no segment;
* one projection of a pair of segments of different strands puts them exactly 2r apart;
* total momentum of two colliding ropes is conserved to rounding (the paper's momentum
  check, App. C), while each rope's own momentum changes.
"""
import math
from pathlib import Path

import numpy as np
import pytest
import torch

from oracle import OracleSim, closest_params
from oracle.dlo import F64
from paper_2606_04206_gb300 import inputs

GOLDEN = Path(__file__).parent / "golden"


def strand_record(parts, **kw):
    """One record holding the vertex arrays ``parts`` as strands, as a one-record workload."""
    x = np.concatenate(parts)
    start = np.zeros(len(x), bool)
    start[np.cumsum([len(q) for q in parts])[:-1]] = True
    return inputs.custom([x], strand_start=start, **kw)


def curve(n, l, origin, heading, bend):
    """An open planar polyline of n vertices, edge length l, turning by ``bend`` rad per hinge."""
    ang = heading + bend * np.arange(n - 1)
    steps = l * np.stack([np.cos(ang), np.sin(ang), 0.02 * np.sin(3 * ang)], 1)
    return np.asarray(origin, float) + np.concatenate([np.zeros((1, 3)), np.cumsum(steps, 0)])


MAT = dict(K=1e5, E=1e4, G=1e3, damping=0.5)


def run(prob, frames):
    sim = OracleSim(prob)
    sim.set_state(prob.x0, prob.v0, prob.theta0, prob.omega0)
    for f in range(frames):
        sim.step(prob.actions[f:f + 1], 1)
    return sim.get_state()


@pytest.mark.parametrize("kind", ["elastic", "plastic_inext", "strain_limit_contact"])
def test_far_apart_strands_step_like_separate_rods(kind):
    """Two strands 0.5 m apart (no contact between them) against the same two DLOs as two
    separate rods: positions, velocities, twist, frames, rest curvature and reference twist
    agree to rounding after 12 frames under gravity on the ground plane, one vertex pinned.
    The first strand has an even vertex count, so the second starts at an even edge index and
    the red-black sweeps take the same order in both layouts."""
    a = curve(10, 0.01, [0, 0, 0.004], 0.3, 0.25)
    b = curve(8, 0.01, [0.5, 0.1, 0.004], 2.0, -0.35)
    kw = dict(MAT, frames=12, planes=np.array([[0.0, 0.0, 1.0, 0.0]]))
    if kind == "plastic_inext":
        kw.update(K=0.0, inextensible=True, plastic=True, yield_curv=2.0)
    if kind == "strain_limit_contact":
        kw.update(strain_limit=0.02, self_contact=True)
        a = curve(10, 0.01, [0, 0, 0.004], 0.3, 0.7)      # curls: self-contact candidates within a strand
    v0 = np.random.default_rng(3).normal(scale=0.2, size=(len(a) + len(b), 3))
    pin = np.zeros(len(a) + len(b), bool)
    pin[len(a) + 2] = True
    env = strand_record([a, b], pinned=pin, **kw)
    env.v0 = v0
    env.theta0 = np.random.default_rng(4).normal(scale=0.3, size=len(env.theta0))
    sep = inputs.custom([a, b], pinned=pin, **kw)
    sep.v0 = v0
    ne = len(a) - 1
    sep.theta0 = np.concatenate([env.theta0[:ne], env.theta0[ne + 1:]])
    E, S = run(env, 12), run(sep, 12)
    na = len(a)
    for k in ("x", "v"):
        assert np.allclose(E[k], S[k], rtol=0, atol=1e-13 * max(1.0, np.abs(S[k]).max())), k
    ed = np.r_[0:ne, ne + 1:len(env.theta0)]          # the real edges of the record
    for k in ("theta", "omega", "tb", "d1b"):
        assert np.allclose(E[k][ed], S[k], rtol=0, atol=1e-12), k
    # hinge arrays are stored per vertex; vertices na-1 and na are the break edge's ends
    for k in ("kbar", "mprev"):
        assert np.allclose(E[k], S[k], rtol=0, atol=1e-12), k
        assert np.all(E[k][[na - 1, na]] == 0)
    # the break edge keeps the frame it was given
    assert np.array_equal(E["tb"][ne], [0.0, 0.0, 1.0]) and np.array_equal(E["d1b"][ne], [1.0, 0.0, 0.0])
    if kind == "plastic_inext":
        assert np.abs(E["kbar"]).max() > 0      # plasticity acted


def test_record_energy_is_the_sum_of_its_strands_energies():
    """At a random configuration (strands overlapping, the second strand's first vertex on the
    first strand's last vertex, so the edge between them has length 0) the record's elastic
    energy and its gradient are the sums over the separate DLOs; the energy is finite."""
    rng = np.random.default_rng(11)
    a = curve(9, 0.01, [0, 0, 0.01], 0.0, 0.3)
    b = curve(7, 0.012, a[-1], 1.0, -0.2)
    env = strand_record([a, b], **MAT)
    sep = inputs.custom([a, b], **MAT)
    se, ss = OracleSim(env), OracleSim(sep)
    se.set_state(env.x0, env.v0, env.theta0, env.omega0)
    ss.set_state(sep.x0, sep.v0, sep.theta0, sep.omega0)
    # move the vertices without touching the frames' state (a non-rest configuration)
    d = rng.normal(scale=2e-3, size=env.x0.shape)
    d[len(a)] = d[len(a) - 1]                       # the two strand ends stay together
    xe = torch.as_tensor(env.x0 + d, dtype=F64)[None].requires_grad_(True)
    G, S = se.groups[0], se.state[0]
    from oracle.dlo import elastic_energy
    Ue = elastic_energy(xe, S["theta"], S["tb"], S["d1b"], S["mprev"], S["kbar"], G["R"], False, G["strands"])
    ge, = torch.autograd.grad(Ue.sum(), xe)
    tot, gs = 0.0, []
    for G2, S2 in zip(ss.groups, ss.state):
        rods = G2["ids"]
        for i, b_ in enumerate(rods):
            lo = 0 if b_ == 0 else len(a)
            xs = torch.as_tensor((env.x0 + d)[lo:lo + G2["N"]], dtype=F64)[None].requires_grad_(True)
            R = {k: (v[i:i + 1] if torch.is_tensor(v) and v.dim() > 0 and v.shape[0] == len(rods) else v)
                 for k, v in G2["R"].items()}
            U = elastic_energy(xs, S2["theta"][i:i + 1], S2["tb"][i:i + 1], S2["d1b"][i:i + 1],
                               S2["mprev"][i:i + 1], S2["kbar"][i:i + 1], R, False)
            g, = torch.autograd.grad(U.sum(), xs)
            tot += float(U)
            gs.append((lo, g[0].numpy()))
    assert math.isfinite(float(Ue))
    assert float(Ue) == pytest.approx(tot, rel=1e-12)
    gsum = np.zeros_like(env.x0)
    for lo, g in gs:
        gsum[lo:lo + len(g)] += g
    assert np.allclose(ge[0].numpy(), gsum, rtol=0, atol=1e-12 * np.abs(gsum).max())


def adjacent_crossing(seed):
    """Strands of 4 and 5 vertices (edge 1 cm, r = 6 mm, so the exclusion window is 2 edges):
    the first strand's last edge (2) crosses the second strand's first edge (4) 0.4-1.9 r
    above it; the edge between the strands is 3.  Edge indices 2 and 4 are two apart, inside
    the window, but they belong to different DLOs."""
    rng = np.random.default_rng(seed)
    r = 0.006
    zc = rng.uniform(0.2, 0.95) * 2 * r
    a = np.array([[-0.03, 0, 0], [-0.02, 0, 0], [-0.01, 0, 0], [0.0, 0, 0]])
    xb = rng.uniform(-0.008, -0.002)
    b = np.array([[xb, -0.005, zc], [xb, 0.005, zc], [xb, 0.015, zc], [xb, 0.025, zc], [xb, 0.035, zc]])
    return a, b, r


@pytest.mark.parametrize("seed", range(4))
def test_adjacent_segments_of_different_strands_collide(seed):
    """The candidate set of the record holds the pair (2, 4) and no pair of one strand inside
    the window: the window excludes neighbours along one DLO only.  Then one projection of
    that pair puts its two closest points at exactly 2r, and its vertices move by the
    App. A.1 weights."""
    a, b, r = adjacent_crossing(seed)
    env = strand_record([a, b], radius=r, K=1e5, E=1e4, self_contact=True)
    r = float(env.radius[0])                        # the workload's radius (rounded to float32)
    sim = OracleSim(env)
    sim.set_state(env.x0, env.v0, env.theta0, env.omega0)
    G = sim.groups[0]
    assert G["R"]["excl"][0] == 2
    found = sim.candidates(G, sim.state[0]["x"])[0].tolist()
    assert [2, 4] in found
    assert all(c - a_ > 2 for a_, c in found if (a_ < 3) == (c < 3)), found
    pairs = torch.tensor([[2, 4]])
    x = np.concatenate([a, b])
    idx = [2, 3, 4, 5]
    t_, u_ = (float(q) for q in closest_params(*(torch.as_tensor(x[i], dtype=F64) for i in idx)))
    beta = np.array([1 - t_, t_, -(1 - u_), -u_])
    out = sim.contact_sweep(G, torch.as_tensor(x, dtype=F64)[None], [pairs])[0][0].numpy()
    sep1 = sum(bb * out[i] for bb, i in zip(beta, idx))
    assert np.linalg.norm(sep1) == pytest.approx(2 * r, rel=1e-12)
    w = G["R"]["w"][0].numpy()
    W = sum(w[i] * bb * bb for i, bb in zip(idx, beta))
    sep0 = sum(bb * x[i] for bb, i in zip(beta, idx))
    n = sep0 / np.linalg.norm(sep0)
    dpen = 2 * r - np.linalg.norm(sep0)
    for i, bb in zip(idx, beta):
        assert np.allclose(out[i] - x[i], dpen * w[i] * bb / W * n, rtol=0, atol=1e-15)
    others = [i for i in range(len(x)) if i not in idx]
    assert np.abs(out[others] - x[others]).max() == 0.0


def test_the_edge_between_strands_is_no_segment():
    """Two strands whose ends are 6 cm apart with a third segment lying on the straight line
    between those ends: the line is the break edge, not rope, so no pair involves it (edge 2
    here) although its segment would pass within 2r of edge 0 of the second strand's far
    part; the same vertices as one rod do give that pair."""
    r = 0.002
    a = np.array([[0.0, 0, 0], [0.01, 0, 0], [0.02, 0, 0]])
    # second strand: starts at x = 0.08, comes back under the gap at x = 0.05
    b = np.array([[0.08, 0, 0], [0.08, 0.01, 0], [0.065, 0.015, 0], [0.05, 0.01, 0], [0.05, 0.0, -0.001],
                  [0.05, -0.01, -0.001]])
    env = strand_record([a, b], radius=r, K=1e5, E=1e4, self_contact=True)
    sim = OracleSim(env)
    sim.set_state(env.x0, env.v0, env.theta0, env.omega0)
    pairs = sim.candidates(sim.groups[0], sim.state[0]["x"])[0].tolist()
    assert all(2 not in pr for pr in pairs), pairs
    one = inputs.custom([np.concatenate([a, b])], radius=r, K=1e5, E=1e4, self_contact=True)
    s1 = OracleSim(one)
    s1.set_state(one.x0, one.v0, one.theta0, one.omega0)
    assert any(2 in pr for pr in s1.candidates(s1.groups[0], s1.state[0]["x"])[0].tolist())


def two_ropes_colliding():
    """Two straight inextensible ropes of 12 vertices crossing at right angles, 3 mm apart
    vertically (r = 2 mm: they overlap), moving towards each other at 0.3 m/s plus random
    vertex velocities; no gravity, no ground, no grippers."""
    n, l = 12, 0.01
    s = (np.arange(n) - (n - 1) / 2) * l
    a = np.stack([s, np.zeros(n), np.zeros(n)], 1)
    b = np.stack([np.zeros(n) + 0.0013, s + 0.0021, np.full(n, 0.003)], 1)
    rng = np.random.default_rng(21)
    v = rng.normal(scale=0.05, size=(2 * n, 3))
    v[:n, 2] += 0.15
    v[n:, 2] -= 0.15
    return a, b, v


def test_momentum_conserved_between_two_ropes():
    """The total momentum of the two ropes stays at its initial value to rounding (below the
    paper's 1e-13 .. 1e-14 momentum error of its contact check, tests/golden/
    momentum_contact.txt) through 15 frames of contact with friction, while each rope's own
    momentum changes: the contact moves momentum from one DLO to the other."""
    a, b, v = two_ropes_colliding()
    env = strand_record([a, b], frames=15, K=0.0, E=1e4, G=1e3, inextensible=True, damping=0.0,
                        gravity=0.0, self_contact=True)
    env.v0 = v
    sim = OracleSim(env)
    sim.set_state(env.x0, env.v0, env.theta0, env.omega0)
    G = sim.groups[0]
    pairs = sim.candidates(G, sim.state[0]["x"])[0]
    assert (G["sid"][pairs[:, 0]] != G["sid"][pairs[:, 1]]).all() and len(pairs) > 0
    m = G["R"]["mass"][0].numpy()
    n = len(a)

    def rope_momenta():
        vv = sim.get_state()["v"]
        return (m[:n, None] * vv[:n]).sum(0), (m[n:, None] * vv[n:]).sum(0)

    P0 = sim.momentum()[0]
    pa0, _ = rope_momenta()
    errs = []
    for f in range(15):
        sim.step(env.actions[f:f + 1], 1)
        errs.append(np.abs(sim.momentum()[0] - P0).max())
    bound = float(open(GOLDEN / "momentum_contact.txt").read().split("max_total_momentum_error")[1].split()[0])
    assert max(errs) < bound, errs
    pa1, _ = rope_momenta()
    assert np.abs(pa1 - pa0).max() > 1e3 * bound      # momentum went from one rope to the other
