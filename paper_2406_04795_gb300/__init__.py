"""GB300-native manifold tracing and certification for motion-planning
infeasibility proofs (arXiv 2406.04795), behind the C ABI of include/mf.h.

``mf`` is the same-name ctypes binding of libmf.so; ``api.Context`` is a thin
torch-facing layer over it; ``workloads`` builds seeded synthetic inputs.
"""
from . import mf  # noqa: F401

__all__ = ["mf", "api", "workloads", "build"]
