"""FP64 CPU oracle of the harmonic-balance residual path.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg / reference arm of ``bench.py`` may import this package.
The product library never loads it, and it shares no code with the CUDA path.
"""
from .hb_oracle import Oracle, build, d_matrix, van_albada, roe_flux  # noqa: F401
