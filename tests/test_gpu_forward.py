"""GPU forward path against the FP64 oracle, through the C ABI.

Tolerances: vertex positions within 1e-5 m after 100 and 200 contact-free frames of the
plain workload; with contact, the per-frame relative error ||x_gpu - x_oracle||_inf /
||x_oracle||_inf <= 1e-5 from the same float32 state.
"""
import numpy as np
import pytest
import torch

from oracle import OracleSim
from paper_2606_04206_gb300 import inputs
from gpu_util import sim_for, oracle_from_device_state, actions_dev, rel_inf

pytestmark = pytest.mark.gpu


def test_plain_config_against_oracle_100_and_200_frames():
    p = inputs.plain(200)
    sim = sim_for(p)
    sim.reset()
    o = OracleSim(p)
    o.set_state(p.x0, p.v0, p.theta0, p.omega0)
    acts = actions_dev(p)
    for f0, f1 in ((0, 100), (100, 200)):
        sim.step(acts[f0:f1].contiguous(), f1 - f0)
        o.step(p.actions[f0:f1], f1 - f0)
        x = sim.get_state()[0][:, :3].double().cpu().numpy()
        err = np.abs(x - o.get_state()["x"]).max()
        assert err <= 1e-5, (f1, err)


@pytest.mark.parametrize("kind", ["batching", "selfcontact", "trajopt", "diff"])
def test_initial_frames_constants_match_oracle(kind):
    p = inputs.small_case(kind, n_rods=5, n=40, frames=2)
    sim = sim_for(p)
    sim.reset()
    o = OracleSim(p)
    o.set_state(p.x0, p.v0, p.theta0, p.omega0)
    ds, os_ = sim.full_state_numpy(), o.get_state()
    for k, tol in (("tb", 1e-6), ("d1b", 1e-6), ("mprev", 2e-6), ("kbar", 1e-6), ("x", 0.0)):
        assert np.abs(ds[k] - os_[k]).max() <= tol, k
    oc = o.rod_constants()
    assert np.array_equal(sim.query(1), np.asarray(oc["nsub"]))          # DLO_Q_SUBSTEPS
    m = sim.query(8)
    np.testing.assert_allclose(m[:, 0], oc["mass"], rtol=1e-6)
    np.testing.assert_allclose(m[:, 1], oc["w"], rtol=1e-6)
    assert np.array_equal(m[:, 2].astype(int), oc["kind"])


@pytest.mark.parametrize("kind,warm", [("batching", 5), ("selfcontact", 5), ("trajopt", 20), ("diff", 5)])
def test_one_frame_from_same_state_with_contact(kind, warm):
    p = inputs.small_case(kind, n_rods=4, n=40, frames=warm + 1)
    sim = sim_for(p)
    sim.reset()
    acts = actions_dev(p)
    sim.step(acts[:warm].contiguous(), warm)
    o = oracle_from_device_state(p, sim)
    sim.step(acts[warm:warm + 1].contiguous(), 1)
    o.step(p.actions[warm:warm + 1], 1)
    fo = o.get_state()
    fg = sim.full_state_numpy()
    assert rel_inf(fg["x"], fo["x"]) <= 1e-5
    # the frame's motion itself (a far stricter check than positions): velocities
    assert rel_inf(fg["v"], fo["v"]) <= 2e-3
    assert np.abs(fg["theta"] - fo["theta"]).max() <= 1e-4
    assert np.abs(fg["kbar"] - fo["kbar"]).max() <= 1e-4


def test_creep_below_full_return_one_frame():
    """r_c = 0.3 creep of the rest curvature (App. A.1) against the oracle, from the same state."""
    p = inputs.small_case("batching", n_rods=4, n=40, frames=6)
    p.creep_rate[:] = 0.3
    p.yield_curv[:] = inputs.f32(np.full(4, 1.0))
    sim = sim_for(p)
    sim.reset()
    acts = actions_dev(p)
    sim.step(acts[:5].contiguous(), 5)
    o = oracle_from_device_state(p, sim)
    sim.step(acts[5:6].contiguous(), 1)
    o.step(p.actions[5:6], 1)
    fo, fg = o.get_state(), sim.full_state_numpy()
    assert np.abs(fo["kbar"]).max() > 0                     # yield was exceeded
    assert rel_inf(fg["x"], fo["x"]) <= 1e-5
    assert np.abs(fg["kbar"] - fo["kbar"]).max() <= 1e-4


def test_ragged_batch_all_size_classes():
    p = inputs.batching(n_rods=8, frames=3, seed=11, vmin=16, vmax=256)
    p.E[:] = inputs.f32(np.full(8, 2e4))          # keep substep counts small for the oracle
    p.K[:] = p.E
    p.G[:] = inputs.f32(0.4 * p.E)
    sim = sim_for(p)
    sim.reset()
    acts = actions_dev(p)
    sim.step(acts[:1].contiguous(), 1)
    o = oracle_from_device_state(p, sim)
    sim.step(acts[1:2].contiguous(), 1)
    o.step(p.actions[1:2], 1)
    assert rel_inf(sim.get_state()[0][:, :3].double().cpu().numpy(), o.get_state()["x"]) <= 1e-5


def coils(n_rods=3, frames=3, n=48):
    """Open rods wound 1.2 turns round a helix whose pitch (3.5 mm) is less than the contact
    distance 2r = 4 mm, so the overlapping part of the coil is in self-contact."""
    rods = []
    for k in range(n_rods):
        s = np.linspace(0.0, 2.4 * np.pi, n)
        R = 0.05 + 0.005 * k
        rods.append(np.stack([R * np.cos(s), R * np.sin(s), 0.05 + 0.0035 * s / (2 * np.pi)], 1))
    return inputs.custom(rods, frames=frames, K=1e5, E=1e4, G=1e3, self_contact=True,
                         planes=np.array([[0, 0, 1.0, 0.0]]))


def pair_set(cand):
    """The oracle's candidates of one rod ([n, 2] edge pairs, a < b) as a set."""
    return {(int(a), int(b)) for a, b in cand.tolist()}


@pytest.mark.parametrize("broad_phase", [0, 1], ids=["all-pairs", "spatial-hash"])
def test_self_contact_candidates_and_projection_match_oracle(broad_phase):
    p = coils()
    sim = sim_for(p, broad_phase=broad_phase)
    sim.reset()
    acts = actions_dev(p)
    o = oracle_from_device_state(p, sim)
    sim.step(acts[:1].contiguous(), 1)
    got = sim.pair_sets()                         # pairs found by the broad phase at that frame start
    for G, S in zip(o.groups, o.state):
        cand = o.candidates(G, S["x"])
        for i, b in enumerate(G["ids"]):
            assert got[b] == pair_set(cand[i]), (b, got[b] ^ pair_set(cand[i]))
    assert min(len(s) for s in got) > 0
    assert np.array_equal(sim.query(6), [len(s) for s in got])
    o.step(p.actions[:1], 1)
    fg, fo = sim.full_state_numpy(), o.get_state()
    assert rel_inf(fg["x"], fo["x"]) <= 1e-5
    assert rel_inf(fg["v"], fo["v"]) <= 2e-3


@pytest.mark.parametrize("broad_phase", [0, 1], ids=["all-pairs", "spatial-hash"])
def test_self_contact_candidates_match_brute_force_on_knots(broad_phase):
    """Knotted bands falling onto the box and the ground: once their crossings come within the
    candidate distance, the device's candidate set of a frame equals the oracle's brute-force
    set from the same state (P11), rod by rod, with either broad phase."""
    p = inputs.small_case("selfcontact", n_rods=6, n=60, frames=400)
    sim = sim_for(p, broad_phase=broad_phase)
    sim.reset()
    acts = actions_dev(p)
    f = 0
    while f < 380 and sim.query(6).sum() == 0:       # DLO_Q_PAIRS of the last dlo_step
        sim.step(acts[f:f + 20].contiguous(), 20)
        f += 20
    assert sim.query(6).sum() > 0, "the knots never came into self-contact"
    o = oracle_from_device_state(p, sim)
    sim.step(acts[f:f + 1].contiguous(), 1)
    got = sim.pair_sets()
    n = 0
    for G, S in zip(o.groups, o.state):
        cand = o.candidates(G, S["x"])
        for i, b in enumerate(G["ids"]):
            assert got[b] == pair_set(cand[i]), (b, got[b] ^ pair_set(cand[i]))
            n += len(got[b])
    assert n > 0


def test_bitwise_deterministic():
    p = inputs.small_case("selfcontact", n_rods=4, n=40, frames=4)
    outs = []
    for _ in range(2):
        sim = sim_for(p)
        sim.reset()
        sim.step(actions_dev(p), 4)
        outs.append(sim.get_state()[0].cpu().numpy())
        sim.close()
    assert np.array_equal(outs[0], outs[1])


def test_edge_cases_two_vertex_rod_and_triangle_loop():
    x2 = np.array([[0.0, 0, 0.5], [0.05, 0, 0.5]])
    tri = np.array([[0.0, 0, 0.5], [0.05, 0, 0.5], [0.025, 0.04, 0.5]])
    p = inputs.custom([x2, tri], closed=[False, True], frames=5, K=1e5, E=1e4, G=1e3,
                      planes=np.array([[0, 0, 1.0, 0.0]]))
    sim = sim_for(p)
    sim.reset()
    o = OracleSim(p)
    o.set_state(p.x0, p.v0, p.theta0, p.omega0)
    sim.step(actions_dev(p), 5)
    o.step(p.actions, 5)
    assert np.abs(sim.get_state()[0][:, :3].double().cpu().numpy() - o.get_state()["x"]).max() <= 1e-6


def test_zero_frames_and_nonfinite_detection():
    from paper_2606_04206_gb300.dlo import DloError
    p = inputs.small_case("trajopt", n_rods=3, n=24, frames=2)
    sim = sim_for(p)
    sim.reset()
    x0 = sim.get_state()[0].clone()
    sim.step(None, 0)
    assert torch.equal(sim.get_state()[0], x0)
    x, v, th = sim.tensors_from_problem()
    v[5, 0] = float("nan")
    sim.set_state(x, v, th)
    sim.step(None, 1)
    with pytest.raises(DloError) as ei:
        sim.get_state()
    assert ei.value.status == 4 and "rod 0" in str(ei.value)


def test_fp64_inextensibility_residual():
    """The inextensibility residual sum_j |C_j| = sum_j | |x_{j+1} - x_j| - |ebar_j| | after the
    last frame (App. A.1), accumulated on the device in FP64 (DLO_Q_RESIDUAL).  It equals the
    FP64 sum over the device's own float32 positions and float32 rest lengths to rounding of the
    sum, and it differs from the oracle's residual after the same frame from the same state by
    no more than the positions allow: each |C_j| moves by at most twice the largest position
    difference, plus the float32 rounding of the rest length."""
    from paper_2606_04206_gb300.dlo import Q_RESIDUAL
    p = inputs.small_case("trajopt", n_rods=6, n=64, frames=4)
    assert p.inextensible.any() and not p.inextensible.all()
    sim = sim_for(p)
    sim.reset()
    acts = actions_dev(p)
    sim.step(acts[:3].contiguous(), 3)
    o = oracle_from_device_state(p, sim)
    sim.step(acts[3:4].contiguous(), 1)
    o.step(p.actions[3:4], 1)
    res = sim.query(Q_RESIDUAL)
    x = sim.get_state()[0][:, :3].double().cpu().numpy()
    xo = o.get_state()["x"]
    vo = p.vert_off
    for b in range(p.batch):
        if not p.inextensible[b]:
            assert res[b] == 0.0
            continue
        eb = o.ebar[b]
        eb32 = eb.astype(np.float32).astype(np.float64)
        xb, xob = x[vo[b]:vo[b + 1]], xo[vo[b]:vo[b + 1]]
        own = np.abs(np.linalg.norm(np.diff(xb, axis=0), axis=1) - eb32).sum()
        assert res[b] == pytest.approx(own, rel=1e-12), (b, res[b], own)
        ora = np.abs(np.linalg.norm(np.diff(xob, axis=0), axis=1) - eb).sum()
        ne = len(eb)
        bound = 2 * ne * np.abs(xb - xob).max() + ne * 2.0 ** -24 * eb.max()
        assert abs(res[b] - ora) <= bound, (b, res[b], ora, bound)
        assert res[b] > 0.0


def test_status_flags_motion_past_the_candidate_margin():
    """Candidates are found once per frame with a margin of contact_margin x r beyond the contact
    distance 2r.  A rod whose vertices move half of that margin or more within one frame gets the
    warning bit 4 in DLO_Q_STATUS; a slow rod does not, and neither is an error."""
    from paper_2606_04206_gb300.dlo import Q_STATUS, STATUS_MOVED_PAST_MARGIN
    xs = [np.stack([np.linspace(0.0, 0.3, 20), np.full(20, y), np.full(20, 0.5)], 1) for y in (0.0, 0.5)]
    p = inputs.custom(xs, frames=2, K=1e5, E=1e4, G=1e3, gravity=0.0, damping=0.0, self_contact=True)
    p.v0 = np.concatenate([np.tile([0.1, 0.0, 0.0], (20, 1)), np.tile([4.0, 0.0, 0.0], (20, 1))])
    sim = sim_for(p)
    sim.reset()
    sim.step(None, 2)
    sim.get_state()                               # a warning, not an error
    st = sim.query(Q_STATUS)
    assert not (st[0] & STATUS_MOVED_PAST_MARGIN) and (st[1] & STATUS_MOVED_PAST_MARGIN), st


def test_rods_without_twist_stiffness_keep_their_twist_and_stay_finite():
    """Reading O41 on the device: a rope with G = 0 has no twist dynamics, so its twist angles
    and rates stay exactly zero.  The candidate checked is one of the CMA-ES population's
    knotted ropes (the bench's Unknotting generation) that, with a dynamic twist angle of so
    small an axial inertia, spun up its twist and became non-finite within 650 frames."""
    p = inputs.cmaes(pop=400, frames=2000, seed=5000, n=128).subset([0, 220])
    sim = sim_for(p)
    sim.reset()
    sim.step(actions_dev(p), 2000)
    x, v, th = (t.cpu().numpy() for t in sim.get_state())
    assert np.isfinite(x).all() and np.isfinite(v).all()
    assert np.all(th == 0.0) and np.all(v[:, 3] == 0.0)
