"""GB300-native slab factor+solve (SlabLU hot path) for finite-difference elliptic PDEs.

The compute path is libslab.so (hand-written sm_103a CUDA kernels behind the C
ABI in include/slab.h).  This package holds its build script, the ctypes
binding, a thin torch-facing wrapper and the seeded input generators.  Nothing
is imported eagerly, so `import paper_2211_07572_gb300.inputs` needs no GPU.
"""
__all__ = ["SlabSolver", "SlabSolveFunction", "SlabError"]


def __getattr__(name):
    if name in ("SlabSolver", "SlabSolveFunction"):
        from . import solver
        return getattr(solver, name)
    if name == "SlabError":
        from ._lib import SlabError
        return SlabError
    raise AttributeError(name)
