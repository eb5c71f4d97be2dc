"""The step loop captured in a CUDA graph: dlo_step only enqueues stream-ordered work (a
memset and one persistent launch per size class) on the context's stream and never
synchronises, so a graph captured on that stream replays the same rollout.  Replaying a
captured 4-frame step three times must give bit for bit the state of 12 directly stepped
frames (the kernels reduce in a fixed order)."""
import numpy as np
import pytest
import torch

from paper_2606_04206_gb300 import inputs
from gpu_util import sim_for, actions_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["trajopt", "batching"])
def test_step_loop_in_a_cuda_graph(kind):
    p = inputs.small_case(kind, n_rods=8, n=48, frames=12)
    acts = actions_dev(p)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = sim_for(p)                     # the context enqueues on `stream`
        sim.reset()
        sim.step(acts, 12)
        direct = [t.clone() for t in sim.get_state()]
        buf = acts[:4].clone()               # the graph's action input
        sim.reset()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
            sim.step(buf, 4)
        stream.synchronize()
        sim.reset()                          # capture does not run the work
        for k in range(3):
            buf.copy_(acts[4 * k:4 * k + 4])
            g.replay()
        stream.synchronize()
        graphed = sim.get_state()
    for a, b in zip(direct, graphed):
        assert torch.equal(a, b)
