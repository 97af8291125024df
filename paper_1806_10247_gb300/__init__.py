"""GB300 (sm_103a) cascaded lattice Boltzmann with Strang-split forcing and
sources (arXiv:1806.10247): a C-ABI CUDA library (``include/lbm.h``) and its
thin Python binding (:mod:`paper_1806_10247_gb300.lbm`)."""
from . import workloads  # noqa: F401

__all__ = ["lbm", "workloads", "build"]
