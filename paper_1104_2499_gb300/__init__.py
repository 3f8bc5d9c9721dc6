"""GB300-native ensemble integrator for active Brownian particles (arXiv 1104.2499).

The compute path is the C-ABI library ``libabp.so`` (hand-written sm_103a CUDA), reached
through :mod:`paper_1104_2499_gb300.abp`; importing this package does not load it, so the
input generators in :mod:`paper_1104_2499_gb300.workloads` stay usable without a GPU.
"""

__all__ = ["abp", "workloads"]
