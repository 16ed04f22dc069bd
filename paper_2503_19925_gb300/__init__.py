"""EXACT (extragradient algorithm for computed tomography) on GB300.

The computation lives in ``libexact.so`` (CUDA kernels for sm_103a behind the C
ABI of ``include/exact.h``); :mod:`.exact` is its thin Python binding.
"""
from .exact import (Geometry, Plan, SolveInfo, ExactError, Job, Batch, Dense, TvInfo, load,  # noqa: F401
                    library_path, tv_options, tv_project, tv_prox, gather_ceiling)
from ._build import build  # noqa: F401
