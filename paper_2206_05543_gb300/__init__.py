"""GB300 (sm_103a) geometric multigrid for the Dirichlet Poisson problem with
the SPAI smoothers of He, Liu and Wang, "Optimized sparse approximate inverse
smoothers for solving Laplacian linear systems" (arXiv:2206.05543).

The compute path is the CUDA library libmg.so (C ABI: include/mg.h); the
Python layer (binding.py) only marshals torch tensors and streams into it.

    from paper_2206_05543_gb300 import Solver, smoothers
    s = Solver(d=2, N=8192)                 # M9 smoother, V(1,1), FP64
    info = s.solve(b)                       # b: CUDA float64 tensor (N-1, N-1)
"""
from . import smoothers  # noqa: F401  (pure Python constants)

__all__ = ["Solver", "SolveInfo", "MGError", "smoothers", "binding"]


def __getattr__(name):
    # the CUDA binding is imported lazily so that the constants and the input
    # generators stay importable without a GPU
    if name in ("Solver", "SolveInfo", "MGError", "binding"):
        import importlib
        binding = importlib.import_module(__name__ + ".binding")
        return binding if name == "binding" else getattr(binding, name)
    raise AttributeError(name)
