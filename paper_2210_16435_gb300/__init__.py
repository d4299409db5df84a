"""GB300-native s-FairSC: fair spectral clustering via the k smallest eigenpairs of
P L_n P + sigma (I - P) (Wang, Lu, Davidson and Bai, AISTATS 2023, Algorithm 3).

The computation lives in libsfairsc.so (hand-written sm_103a CUDA behind a C
ABI, include/sfairsc.h).  `binding` exposes the C entry points by name;
`solver` wraps them for PyTorch tensors.  Importing this package does not load
the library; the first call does, and fails loudly if it is missing.
"""
from . import binding
from .buildlib import build, library_path

__all__ = ["binding", "build", "library_path", "FairSC", "FairEigenvalueSum", "kmeans"]


def __getattr__(name):
    if name in ("FairSC", "FairEigenvalueSum", "kmeans"):
        from . import solver

        return getattr(solver, name)
    raise AttributeError(name)
