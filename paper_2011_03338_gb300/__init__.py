"""GB300 implementation of the multi-level blended DG/FV right-hand side of
Markert, Gassner & Walch (arXiv 2011.03338): CUDA kernels behind the C ABI of
include/sesc.h, with a thin ctypes binding (sesc.Solver, sesc.Batch) and seeded workload
generators (inputs)."""
from .sesc import Batch, Solver, SescError, load  # noqa: F401
