"""B300-native batched quadrotor simulator (arXiv 2308.12698, Sec. III-B hot path).

The compute lives in libquadsim.so (hand-written sm_103a CUDA behind the C ABI
of include/quadsim.h); this package only marshals arguments to it.
"""
from . import workload  # noqa: F401
from ._lib import SimError  # noqa: F401

__all__ = ["Sim", "Graph", "QuadRollout", "planar", "unplanar", "workload", "SimError"]


def __getattr__(name):
    if name in ("Sim", "Graph", "QuadRollout", "planar", "unplanar", "theta_of", "with_theta"):
        from . import sim
        return getattr(sim, name)
    raise AttributeError(name)
