"""FP64 CPU oracle of the active-Brownian-particle ensemble (arXiv 1104.2499, Sec. 2).

Test infrastructure only: used by ``tests/``, the smoke check and the benchmark's CPU
baseline leg.  It shares no code with the CUDA path.
"""
