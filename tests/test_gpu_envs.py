"""Environments of several DLOs on the GPU (the strands of one record, dlo_scene.strand_start;
Sec. 4's Separation ropes coupled by App. A.1's self-collision projection and friction),
through the C ABI, against the FP64 oracle.

Tolerances are those of the single-rod tests: a per-frame relative position error <= 1e-5
from the same float32 state, velocities <= 2e-3, twist angles 1e-4; the device's candidate
pair sets equal the oracle's exactly; gradients within relative L2 1e-3 and cosine 0.999 of
the oracle's reverse mode.  DLOs far apart step bit for bit like the same DLOs as separate
rods, since every phase does the same float arithmetic on each strand.
"""
import numpy as np
import pytest
import torch

from oracle import OracleSim
from paper_2606_04206_gb300 import inputs
from gpu_util import (sim_for, oracle_from_device_state, actions_dev, rel_inf, oracle_gradients,
                      device_gradients, grad_agreement)
import test_oracle_envs as V

pytestmark = pytest.mark.gpu


def strand_of_edges(prob, b):
    """Strand index of every edge of record b (-1 on the break edges)."""
    vo = prob.vert_off
    st = prob.strand_start[vo[b]:vo[b + 1]]
    sid = np.cumsum(st)
    e = np.where(st[1:], -1, sid[:-1])
    return e


def cross_pairs(prob, sets):
    """Number of candidate pairs between two different strands, over all records."""
    n = 0
    for b, s in enumerate(sets):
        sid = strand_of_edges(prob, b)
        n += sum(1 for a, c in s if sid[a] != sid[c])
    return n


def test_strand_records_start_like_the_oracle():
    """Initial frames (each strand starts its own), reference twists, substeps, masses and
    kinematic kinds of Separation records equal the oracle's."""
    p = inputs.small_case("separation", n_rods=3, n=14, frames=2)
    sim = sim_for(p)
    sim.reset()
    o = OracleSim(p)
    o.set_state(p.x0, p.v0, p.theta0, p.omega0)
    ds, os_ = sim.full_state_numpy(), o.get_state()
    for k, tol in (("tb", 1e-6), ("d1b", 1e-6), ("mprev", 2e-6), ("kbar", 1e-6), ("x", 0.0)):
        assert np.abs(ds[k] - os_[k]).max() <= tol, k
    oc = o.rod_constants()
    assert np.array_equal(sim.query(1), np.asarray(oc["nsub"]))
    m = sim.query(8)
    np.testing.assert_allclose(m[:, 0], oc["mass"], rtol=1e-6)
    np.testing.assert_allclose(m[:, 1], oc["w"], rtol=1e-6)
    assert np.array_equal(m[:, 2].astype(int), oc["kind"])


def separation_in_contact(broad_phase=0, plain=False, n_rods=4, n=16):
    """Separation records stepped until their ropes touch (candidate pairs between strands)."""
    p = inputs.small_case("separation", n_rods=n_rods, n=n, frames=200)
    sim = sim_for(p, broad_phase=broad_phase)
    sim.reset()
    acts = actions_dev(p)
    f = 0
    while f < 160:
        (sim.step_plain if plain else sim.step)(acts[f:f + 10].contiguous(), 10)
        f += 10
        if not plain and cross_pairs(p, sim.pair_sets()) > 0:
            break
    return p, sim, acts, f


@pytest.mark.parametrize("broad_phase", [0, 1], ids=["all-pairs", "spatial-hash"])
def test_candidates_between_strands_match_oracle(broad_phase):
    """Once the ropes touch, the device's candidate set of a frame equals the oracle's from
    the same state, record by record, pairs between the two ropes included; the frame then
    agrees with the oracle's."""
    p, sim, acts, f = separation_in_contact(broad_phase)
    o = oracle_from_device_state(p, sim)
    sim.step(acts[f:f + 1].contiguous(), 1)
    got = sim.pair_sets()
    n_cross = 0
    for G, S in zip(o.groups, o.state):
        cand = o.candidates(G, S["x"])
        for i, b in enumerate(G["ids"]):
            want = {(int(a), int(c)) for a, c in cand[i].tolist()}
            assert got[b] == want, (b, got[b] ^ want)
    n_cross = cross_pairs(p, got)
    assert n_cross > 0
    o.step(p.actions[f:f + 1], 1)
    fg, fo = sim.full_state_numpy(), o.get_state()
    assert rel_inf(fg["x"], fo["x"]) <= 1e-5
    assert rel_inf(fg["v"], fo["v"]) <= 2e-3
    assert np.abs(fg["theta"] - fo["theta"]).max() <= 1e-4


@pytest.mark.parametrize("plain", [False, True], ids=["persistent", "plain"])
def test_separation_frames_match_oracle(plain):
    """Three frames of tangled ropes in contact, from the same state: the persistent kernel
    and the plain per-phase comparator against the oracle."""
    p, sim, acts, f = separation_in_contact(plain=plain)
    o = oracle_from_device_state(p, sim)
    (sim.step_plain if plain else sim.step)(acts[f:f + 3].contiguous(), 3)
    o.step(p.actions[f:f + 3], 3)
    fg, fo = sim.full_state_numpy(), o.get_state()
    assert rel_inf(fg["x"], fo["x"]) <= 1e-5
    assert rel_inf(fg["v"], fo["v"]) <= 2e-3
    assert np.abs(fg["theta"] - fo["theta"]).max() <= 1e-4
    assert not (sim.query(2) & 3).any()      # DLO_Q_STATUS: finite, no pair overflow


@pytest.mark.parametrize("kind", ["elastic", "plastic_inext", "strain_limit_contact"])
def test_far_apart_strands_step_like_separate_rods(kind):
    """The two DLOs of the oracle pin (one curled into self-contact in the last case), 0.5 m
    apart, as one record of two strands and as two rods: after 12 frames every position,
    velocity and twist angle is bit for bit the same."""
    a = V.curve(10, 0.01, [0, 0, 0.004], 0.3, 0.7 if kind == "strain_limit_contact" else 0.25)
    b = V.curve(8, 0.01, [0.5, 0.1, 0.004], 2.0, -0.35)
    kw = dict(V.MAT, frames=12, planes=np.array([[0.0, 0.0, 1.0, 0.0]]))
    if kind == "plastic_inext":
        kw.update(K=0.0, inextensible=True, plastic=True, yield_curv=2.0)
    if kind == "strain_limit_contact":
        kw.update(strain_limit=0.02, self_contact=True)
    v0 = np.random.default_rng(3).normal(scale=0.2, size=(len(a) + len(b), 3))
    env = V.strand_record([a, b], **kw)
    sep = inputs.custom([a, b], **kw)
    env.v0 = sep.v0 = v0
    out = []
    for prob in (env, sep):
        sim = sim_for(prob)
        sim.reset()
        sim.step(actions_dev(prob), 12)
        out.append(sim.full_state_numpy())
        sim.close()
    E, S = out
    ne = len(a) - 1
    ed = np.r_[0:ne, ne + 1:len(E["theta"])]
    assert np.array_equal(E["x"], S["x"]) and np.array_equal(E["v"], S["v"])
    assert np.array_equal(E["theta"][ed], S["theta"])
    assert np.array_equal(E["tb"][ne], [0.0, 0.0, 1.0]) and np.array_equal(E["d1b"][ne], [1.0, 0.0, 0.0])


def colliding_ropes(frames):
    """The oracle pin's two crossing ropes, overlapping and moving into each other, each held
    by a gripper near one end, both moved by small smooth random actions; gravity on."""
    a, b, v = V.two_ropes_colliding()
    rng = np.random.default_rng(8)
    gp = np.stack([a[2], b[9]])[None]
    unit = lambda t: t / np.linalg.norm(t)
    gr = np.stack([inputs._gripper_frame(unit(a[3] - a[1])), inputs._gripper_frame(unit(b[10] - b[8]))])[None]
    acts = inputs._smooth_actions(rng, frames, 1, 1e-3, amp_pos=0.02, amp_rot=0.1)
    p = V.strand_record([a, b], frames=frames, K=0.0, E=5e3, G=1e3, inextensible=True, self_contact=True,
                        actions=acts, n_grippers=np.array([2]), grip_pos=gp, grip_rot=gr)
    p.v0 = inputs.f32(v)
    return p


@pytest.mark.parametrize("plain", [False, True], ids=["fused", "plain"])
def test_backward_through_contact_between_strands(plain):
    """Three frames of two ropes colliding (pairs between the strands active from the first
    projection) differentiated by the fused adjoint and by the plain comparator's: every
    gradient group (initial state, actions, material sensitivities) against the oracle's
    reverse mode."""
    from test_gpu_backward import weights, log_sens, GROUPS
    from test_gpu_plain import plain_gradients
    p = colliding_ropes(3)
    wx, wv, wth = weights(p, 5)
    ref, _ = oracle_gradients(p, 3, wx, wv, wth)
    sim = sim_for(p)
    got = (plain_gradients(sim, p, 3, wx, wv, wth) if plain else device_gradients(sim, p, 3, wx, wv, wth))
    o = OracleSim(p)
    o.set_state(p.x0, p.v0, p.theta0, p.omega0)
    first = o.candidates(o.groups[0], o.state[0]["x"])[0].tolist()
    assert cross_pairs(p, [{tuple(q) for q in first}]) > 0      # the ropes touch from the start
    got["material"], ref["material"] = log_sens(p, got["material"]), log_sens(p, ref["material"])
    report = {k: grad_agreement(got[k], ref[k]) for k in GROUPS}
    print("strands, gradient agreement (rel L2, cosine):",
          {k: (f"{r:.2e}", f"{c:.6f}") for k, (r, c) in report.items()})
    assert all(r <= 1e-3 and c >= 0.999 for k, (r, c) in report.items() if np.linalg.norm(ref[k]) > 0), report


def pushed_together(n_rods, n, frames, speed=0.6):
    """Separation records whose ropes start moving into each other (every vertex towards the
    nearest vertex of the other rope at ``speed`` m/s), so that they touch within a few frames."""
    p = inputs.small_case("separation", n_rods=n_rods, n=n, frames=frames)
    v = np.zeros_like(p.x0)
    for b in range(p.batch):
        x = p.x0[p.vert_off[b]:p.vert_off[b + 1]]
        A, B = x[:n], x[n:]
        for src, dst, off in ((A, B, 0), (B, A, n)):
            d = dst[np.argmin(np.linalg.norm(src[:, None] - dst[None], axis=2), axis=1)] - src
            v[p.vert_off[b] + off:p.vert_off[b] + off + n] = speed * d / np.linalg.norm(d, axis=1)[:, None]
    p.v0 = inputs.f32(v)
    return p


def test_plain_backward_equals_the_fused_adjoint_on_separation():
    """Six frames of Separation records whose ropes collide, checkpoints every 3 frames: the
    plain comparator's adjoint equals the fused one to float rounding."""
    from test_gpu_backward import weights, GROUPS
    from test_gpu_plain import plain_gradients
    q = pushed_together(3, 14, 6)
    wx, wv, wth = weights(q, 2)
    sim = sim_for(q, checkpoint_every=3)
    fused = plain_gradients(sim, q, 6, wx, wv, wth, record_plain=False, plain_bwd=False)
    assert sim.query(6).min() > 0          # DLO_Q_PAIRS: every record had candidates in some frame
    plain = plain_gradients(sim, q, 6, wx, wv, wth, record_plain=True, plain_bwd=True)
    for k in GROUPS:
        rel, cos = grad_agreement(plain[k], fused[k])
        assert rel <= 1e-4 and cos >= 0.999999, (k, rel, cos)


def test_momentum_conserved_between_two_ropes_on_device():
    """The oracle pin's colliding ropes without grippers or gravity: the contact moves momentum
    from one rope to the other, and the total is kept to within 1e-4 of the momentum moved.
    The projection conserves momentum exactly; what the device loses is rounding: float32
    arithmetic and the fixed-point sums of the position corrections (2^-30 m quanta, each
    worth m 2^-30 / h of momentum), about 1e-6 of the momentum moved here."""
    a, b, v = V.two_ropes_colliding()
    p = V.strand_record([a, b], frames=15, K=0.0, E=1e4, G=1e3, inextensible=True, damping=0.0,
                        gravity=0.0, self_contact=True)
    p.v0 = inputs.f32(v)
    sim = sim_for(p)
    sim.reset()
    m = sim.query(8)[:, 0]
    n = len(a)

    def momenta():
        vv = sim.full_state_numpy()["v"][:, :3]
        return (m[:n, None] * vv[:n]).sum(0), (m[n:, None] * vv[n:]).sum(0)

    pa0, pb0 = momenta()
    sim.step(actions_dev(p), 15)
    pa1, pb1 = momenta()
    moved = np.abs(pa1 - pa0).max()
    assert moved > 1e-2 * np.abs(m[:, None] * p.v0).sum()
    assert np.abs((pa1 + pb1) - (pa0 + pb0)).max() <= 1e-4 * moved


def test_invalid_strands_are_rejected():
    """A strand of one vertex, and strands in a closed loop, are argument errors of dlo_create."""
    from paper_2606_04206_gb300.dlo import DloError
    x = V.curve(8, 0.01, [0, 0, 0.01], 0.0, 0.2)
    bad = np.zeros(8, bool)
    bad[7] = True                                       # the last strand would be one vertex
    with pytest.raises(DloError):
        sim_for(inputs.custom([x], strand_start=bad, K=1e5, E=1e4))
    ring = np.stack([np.cos(np.linspace(0, 2 * np.pi, 9)[:-1]), np.sin(np.linspace(0, 2 * np.pi, 9)[:-1]),
                     np.zeros(8)], 1) * 0.05
    two = np.zeros(8, bool)
    two[4] = True
    with pytest.raises(DloError):
        sim_for(inputs.custom([ring], closed=[True], strand_start=two, K=1e5, E=1e4))
