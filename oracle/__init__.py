"""CPU oracle for the batched constant-pressure reactor path (TEST INFRASTRUCTURE).

A plain FP64 C++ restatement of the method of Stone, Alferman & Niemeyer
(arXiv 1608.05794), wrapped with ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and reference
legs may import it (``oracle/make_*.py`` are the committed scripts that wrote
the stored inputs from it).
It shares no code with the CUDA library in ``paper_1608_05794_gb300``.
"""
from .oracle import Oracle, OracleMech, build_oracle, ORA_ROS4, ORA_RKF45  # noqa: F401
