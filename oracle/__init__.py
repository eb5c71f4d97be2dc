"""FP64 CPU oracle of the DLO-Lab rod stepper.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (the C-ABI library and its Python binding) never calls it and
shares no code with it.

The oracle restates the paper's discrete-elastic-rod model (Sec. 3.1 and
Appendix A.1) in plain PyTorch CPU ops in float64, one group of equally sized
rods at a time, with forces taken as the autograd gradient of the elastic
energy and gradients of whole rollouts taken by autograd through every step.
"""
from .dlo import OracleSim, build_frames, elastic_energy, closest_params, sdf_plane, sdf_box, sdf_capsule, substeps_for

__all__ = ["OracleSim", "build_frames", "elastic_energy", "closest_params", "sdf_plane",
           "sdf_box", "sdf_capsule", "substeps_for"]
