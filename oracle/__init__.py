"""FP64 CPU oracle for the MeCuCo fast mean-curvature estimator (arXiv 2606.06329).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only code that may import this package.
It shares no code with the CUDA library under ``paper_2606_06329_gb300/``.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import __all__  # noqa: F401
