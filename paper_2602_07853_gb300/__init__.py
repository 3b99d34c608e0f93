"""GB300 (sm_103a) MPM Lite hot path: C-ABI library ``libmpml.so`` and its thin binding.

``paper_2602_07853_gb300.mpml`` exposes the C entry points by their C names;
``paper_2602_07853_gb300.scenes`` generates seeded synthetic inputs.
"""
from . import build  # noqa: F401
