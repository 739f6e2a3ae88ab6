"""tetmf: GB300-native matrix-free Laplace operators on tetrahedral meshes
(arxiv 2509.10226).  The compute path is the CUDA library libtetmf.so behind
the C ABI of include/tetmf.h; this package holds its build script and a thin
ctypes/PyTorch binding."""
from ._lib import FemError  # noqa: F401


def __getattr__(name):
    if name in ("FemSpace", "FemApply", "fem_apply"):
        from . import fem
        return getattr(fem, name)
    raise AttributeError(name)
