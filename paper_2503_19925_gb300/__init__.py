"""EXACT (extragradient algorithm for computed tomography) on GB300.

The computation lives in ``libexact.so`` (CUDA kernels for sm_103a behind the C
ABI of ``include/exact.h``); :mod:`.exact` is its thin Python binding.
"""
from .exact import (Geometry, Plan, SolveInfo, ExactError, Job, Batch, TvInfo, load, library_path,  # noqa: F401
                    tv_options, tv_project)
from ._build import build  # noqa: F401
