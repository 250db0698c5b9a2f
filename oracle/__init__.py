"""Oracle for the BSS determinant QMC sweep (Rost & Bluemer, arXiv:1504.05090).

TEST INFRASTRUCTURE ONLY.  Plain, slow FP64 CPU code (numpy/scipy) that
restates the method so that the CUDA library can be checked against it.  Only
`tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference leg of
`bench.py` may import it.  The product path never calls it and it shares no
code with the CUDA library.
"""
from .dqmc import *  # noqa: F401,F403
