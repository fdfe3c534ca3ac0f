"""GB300-native magnified stochastic texture filtering with sample reuse.

The compute path lives in the CUDA library ``libstf.so`` (sources in ``csrc/``, C interface in
``include/stf.h``); ``stf`` is its thin ctypes binding. ``workloads`` makes the seeded synthetic
inputs. Importing the package loads nothing; the library is loaded on first use and a missing
library is an error (there is no CPU fallback).
"""
__all__ = ["stf", "workloads"]
