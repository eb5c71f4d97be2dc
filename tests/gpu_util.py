"""Shared helpers of the GPU tests: build/load the library, run the oracle beside it."""
import numpy as np
import torch

from oracle import OracleSim


def sim_for(prob, **opt):
    from paper_2606_04206_gb300 import build, dlo
    build.build()
    return dlo.DloSim(prob, **opt)


def oracle_from_device_state(prob, sim):
    """An oracle loaded with the device's current (float32) state, every internal array included."""
    o = OracleSim(prob)
    o.set_full_state(sim.full_state_numpy())
    return o


def actions_dev(prob, f0=0, f1=None):
    f1 = prob.frames if f1 is None else f1
    return torch.as_tensor(np.ascontiguousarray(prob.actions[f0:f1], np.float32), device="cuda")


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))
