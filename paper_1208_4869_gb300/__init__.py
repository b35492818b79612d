"""GB300-native complex Krylov solvers (the hot path of Flatau's CCGPAK 2.0).

The solver library is ``libccg.so`` (CUDA for sm_103a behind a C ABI declared
in ``include/ccg.h``); ``paper_1208_4869_gb300.ccg`` is its Python binding.
The binding is imported on demand so that the input generators in
``workloads`` stay importable on machines without the built library.
"""
__all__ = ["ccg", "workloads"]
