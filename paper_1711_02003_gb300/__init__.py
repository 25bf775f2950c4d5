"""GB300-native regularized colour-gradient lattice Boltzmann (arXiv:1711.02003).

The compute path is the CUDA library ``liblbcg.so`` (C ABI declared in
include/lbcg.h), loaded lazily by :mod:`paper_1711_02003_gb300.lbcg`.
"""
from . import workloads  # noqa: F401  (pure-python input generators)

__all__ = ["workloads"]
