"""Planted mistakes in the oracle must fail its pins.

Each case edits one expression of one oracle function (a flipped sign, a dropped square, a
swapped operand, a wrong index or weight), installs the edited copy in place of the original
for the duration of the test, and runs the pin that is meant to catch that mistake: the pin
must fail with an assertion.  This shows that the pins of the self-collision projection, the
gripper kinematics, damping, self-contact friction and environments of several DLOs
constrain the oracle's arithmetic and not only its shape.  Nothing here touches the device
code.
"""
import inspect
import textwrap

import pytest

import oracle.dlo as O
import test_oracle_envs as V
import test_oracle_pins as P


def install_mutant(monkeypatch, owner, name, old, new):
    """Replace owner.name by a copy of its source with `old` replaced by `new` (exactly one
    occurrence), compiled in the oracle module's namespace."""
    fn = getattr(owner, name)
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, (name, old)
    ns = dict(vars(O))
    exec(compile(src.replace(old, new), f"<mutant of {name}>", "exec"), ns)
    monkeypatch.setattr(owner, name, ns[name])


def run_pin(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


PROJECTION = [
    ("normal flipped", "nrm = dv / torch.where(act, dist", "nrm = -dv / torch.where(act, dist"),
    ("W without squared weights", "W = w[a0] * (1 - s) ** 2 + w[a1] * s ** 2", "W = w[a0] * (1 - s) + w[a1] * s"),
    ("wrong barycentric weight", "(k * w[a1] * s)[:, None] * nrm", "(k * w[a1] * (1 - s))[:, None] * nrm"),
    ("b side weight of the wrong vertex", "-(k * w[c0] * (1 - u))", "-(k * w[c1] * (1 - u))"),
]


@pytest.mark.parametrize("what,old,new", PROJECTION, ids=[c[0] for c in PROJECTION])
def test_projection_pin_catches(what, old, new, monkeypatch):
    install_mutant(monkeypatch, O.OracleSim, "contact_sweep", old, new)
    run_pin(P.test_self_contact_projection_single_pair, 0)


GRIPPER = [
    ("substep rotation composed on the wrong side", "R1 = expmap(((s + 1) / n) * dphi) @ S[\"gR\"]",
     "R1 = S[\"gR\"] @ expmap(((s + 1) / n) * dphi)", "substep"),
    ("target at the substep start", "p1 = S[\"gp\"] + ((s + 1) / n) * dp", "p1 = S[\"gp\"] + (s / n) * dp",
     "substep"),
    ("grasped vertex rotated by the start pose", "tgt = p1[:, g, None, :] + (R1[:, g, None]",
     "tgt = p1[:, g, None, :] + (R0[:, g, None]", "substep"),
    ("rotation increment with the wrong sign", "R1 = expmap(((s + 1) / n) * dphi)", "R1 = expmap(-((s + 1) / n) * dphi)",
     "substep"),
    ("frame-end rotation composed on the wrong side", "S[\"gR\"] = expmap(act[..., 3:]) @ S[\"gR\"]",
     "S[\"gR\"] = S[\"gR\"] @ expmap(act[..., 3:])", "frame"),
    ("grasp offset kept in world axes", "off[i, grab] = (xr[grab] - pg) @ Rg", "off[i, grab] = (xr[grab] - pg)",
     "_group"),
]


@pytest.mark.parametrize("what,old,new,fn", GRIPPER, ids=[c[0] for c in GRIPPER])
def test_gripper_pin_catches(what, old, new, fn, monkeypatch):
    install_mutant(monkeypatch, O.OracleSim, fn, old, new)
    run_pin(P.test_gripper_kinematics_closed_form, "both")


DAMPING = [
    ("damping force with the wrong sign", "acc = -w * gx + grav - R[\"cd\"][:, None, None] * v",
     "acc = -w * gx + grav + R[\"cd\"][:, None, None] * v"),
    ("twist rate not damped", "om1 = om + h * (-gth / R[\"inertia\"] - R[\"cd\"][:, None] * om)",
     "om1 = om + h * (-gth / R[\"inertia\"])"),
    ("damping halved", "acc = -w * gx + grav - R[\"cd\"][:, None, None] * v",
     "acc = -w * gx + grav - 0.5 * R[\"cd\"][:, None, None] * v"),
    ("damping scaled by the inverse mass", "acc = -w * gx + grav - R[\"cd\"][:, None, None] * v",
     "acc = -w * gx + grav - R[\"cd\"][:, None, None] * v * w * R[\"mass\"][..., None] * 1.01"),
]


@pytest.mark.parametrize("what,old,new", DAMPING, ids=[c[0] for c in DAMPING])
def test_damping_pin_catches(what, old, new, monkeypatch):
    install_mutant(monkeypatch, O.OracleSim, "substep", old, new)
    run_pin(P.test_damping_decays_velocity_and_twist_rate_geometrically)


FRICTION = [
    ("wrong barycentric weight", "(w[I[\"a1\"]] * s)[:, None] * dv", "(w[I[\"a1\"]] * (1 - s))[:, None] * dv"),
    ("wrong vertex weight", "-(w[I[\"c0\"]] * (1 - u))", "-(w[I[\"c1\"]] * (1 - u))"),
    ("sign flipped", "dv = -(coef / Ws)[:, None] * vt", "dv = (coef / Ws)[:, None] * vt"),
    ("Coulomb bound doubled", "self.p.mu_self * I[\"d\"] / (h * vts)", "2.0 * self.p.mu_self * I[\"d\"] / (h * vts)"),
]


@pytest.mark.parametrize("what,old,new", FRICTION, ids=[c[0] for c in FRICTION])
def test_friction_pin_catches(what, old, new, monkeypatch):
    install_mutant(monkeypatch, O.OracleSim, "self_friction", old, new)
    run_pin(P.test_self_contact_friction_obeys_coulomb, 0)


ENVIRONMENT = [
    ("window applied across strands", "keep = real & ((sep > k) | other)", "keep = real & (sep > k)",
     O.OracleSim, "candidates", V.test_adjacent_segments_of_different_strands_collide, (0,)),
    ("break edge taken as a segment", "keep = real & ((sep > k) | other)", "keep = (sep > k) | other",
     O.OracleSim, "candidates", V.test_the_edge_between_strands_is_no_segment, ()),
    ("break edge projected to its length", "colors = [ev, [j for j in range(1, E, 2) if sid[j] >= 0]]",
     "colors = [ev, list(range(1, E, 2))]", O.OracleSim, "_group",
     V.test_far_apart_strands_step_like_separate_rods, ("plastic_inext",)),
    ("break edge counted in the Voronoi masses", "eb[v1 - 1] = 0.0", "eb[v1 - 1] = eb[v1 - 1]",
     O.OracleSim, "__init__", V.test_far_apart_strands_step_like_separate_rods, ("elastic",)),
    ("energy taken over the whole record", "st = G[\"strands\"]\n", "st = None\n",
     O.OracleSim, "substep", V.test_far_apart_strands_step_like_separate_rods, ("elastic",)),
    ("frames transported across the break", "    if strands is None:\n        return build_frames(x, closed)",
     "    if True:\n        return build_frames(x, closed)", O, "build_frames_of",
     V.test_far_apart_strands_step_like_separate_rods, ("elastic",)),
    ("contact moves one strand only", "delta = delta.index_add(0, c0, -(k * w[c0] * (1 - u))[:, None] * nrm)",
     "delta = delta.index_add(0, c0, 0.0 * (k * w[c0] * (1 - u))[:, None] * nrm)", O.OracleSim, "contact_sweep",
     V.test_momentum_conserved_between_two_ropes, ()),
]


@pytest.mark.parametrize("what,old,new,owner,fn,pin,args", ENVIRONMENT, ids=[c[0] for c in ENVIRONMENT])
def test_environment_pins_catch(what, old, new, owner, fn, pin, args, monkeypatch):
    install_mutant(monkeypatch, owner, fn, old, new)
    run_pin(pin, *args)


def test_unmutated_pins_pass():
    """The same pins with the oracle as it is (the baseline of the cases above)."""
    P.test_self_contact_projection_single_pair(0)
    P.test_gripper_kinematics_closed_form("both")
    P.test_damping_decays_velocity_and_twist_rate_geometrically()
    P.test_self_contact_friction_obeys_coulomb(0)
    V.test_adjacent_segments_of_different_strands_collide(0)
    V.test_the_edge_between_strands_is_no_segment()
    V.test_far_apart_strands_step_like_separate_rods("plastic_inext")
    V.test_far_apart_strands_step_like_separate_rods("elastic")
    V.test_momentum_conserved_between_two_ropes()
