"""GB300-native batched differentiable discrete-elastic-rod stepper (DLO-Lab hot path).

The compute path is the C-ABI library ``libdlo.so`` (hand-written sm_103a CUDA); this
package holds its thin ctypes binding (``dlo``) and the seeded workload generator
(``inputs``).  Importing the package does not load the library; ``dlo.load()`` does, and
fails loudly when the library is missing.
"""
__all__ = ["inputs", "dlo"]
