"""Central differences of FP64 oracle rollouts, one coordinate per worker process.

Used by the long-horizon gradient test.  Each worker runs the oracle twice (coordinate
+h and -h) with its branch trace on, and reports whether the two runs took the same branches
(rigid contact active, yield, strain-limit projection, candidate pairs) at every substep:
where they did not, the loss is not differentiable across the interval and the central
difference does not estimate the derivative, so the caller resamples that coordinate.
"""
import copy

import numpy as np


def perturbed(prob, name, idx, delta):
    q = copy.deepcopy(prob)
    arr = q.actions if name == "act" else getattr(q, name)
    arr[idx] += delta
    return q


def target_loss(prob, frames, n_total):
    """sum over the rod's vertices of |x_T - target|^2 / n_total (its share of the mean over all
    rods' vertices), with the branch trace of the rollout."""
    from oracle import OracleSim
    o = OracleSim(prob)
    o.trace = []
    o.set_state(prob.x0, prob.v0, prob.theta0, prob.omega0)
    o.step(prob.actions, frames)
    x = o.get_state()["x"]
    return float(((x - prob.target) ** 2).sum() / n_total), o.trace


def same_branches(ta, tb):
    return len(ta) == len(tb) and all(ka == kb and np.array_equal(a, b) for (ka, a), (kb, b) in zip(ta, tb))


def central_difference(args):
    """(d loss / d coordinate by central differences, whether both runs took the same branches)."""
    import torch
    torch.set_num_threads(1)
    prob, frames, n_total, name, idx, h = args
    lp, tp = target_loss(perturbed(prob, name, idx, +h), frames, n_total)
    lm, tm = target_loss(perturbed(prob, name, idx, -h), frames, n_total)
    return (lp - lm) / (2.0 * h), same_branches(tp, tm)
