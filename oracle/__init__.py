"""FP64 CPU oracle of the TS2-GauSum split step (test infrastructure only).

This package is test infrastructure. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it. The CUDA library in
``paper_1512_03210_gb300`` shares no code with it and never calls it.

Every function follows the paper (Antoine, Tang & Zhang, "On the ground states
and dynamics of space fractional nonlinear Schroedinger/Gross-Pitaevskii
equations with rotation term and nonlocal nonlinearity", arXiv 1512.03210)
step by step, in float64, with numpy's FFT as the only library primitive.
Parity of every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, brute-force quadrature, invariants and special cases.
"""
from .fse_oracle import *  # noqa: F401,F403
from .fse_oracle import __all__  # noqa: F401
