"""EBIT interface step on GB300: C-ABI library (libebit.so) + thin binding.

Importing the package does not load the CUDA library; ``paper_2309_00338_gb300.ebit``
does, and fails loudly if it was not built.
"""
__all__ = ["build", "ebit", "workloads"]
