"""GB300 (sm_103a) EM-PIC step with the damped-current PML of arXiv:2201.09084.

The compute path is libpicpml.so (CUDA kernels behind the C ABI of
include/picpml.h); ``api.Sim`` is a thin binding over it.  Build it with
``paper_2201_09084_gb300.build.build()``.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "api", "build"]
