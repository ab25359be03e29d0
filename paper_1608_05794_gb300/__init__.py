"""Batched constant-pressure chemical kinetics on GB300 (sm_103a).

The compute path is the CUDA library ``libck.so`` (C ABI in ``include/ck.h``);
``paper_1608_05794_gb300.ck`` is its Python binding.
"""
__all__ = ["ck", "build"]
