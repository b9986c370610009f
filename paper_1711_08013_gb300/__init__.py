"""GB300-native (sm_103a) OSQP ADMM hot path: C-ABI CUDA library + thin binding.

Importing the package does not load the CUDA library; ``solver.Solver`` and
``_binding`` load it on first use and raise if it is missing.
"""
__all__ = ["problems", "build", "solver"]
