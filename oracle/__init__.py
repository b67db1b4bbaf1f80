"""FP64 CPU oracle for vortex-field smoothing (arXiv:2203.09764).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
and reference legs of the benchmark are the only callers.  The product path never imports
this package.  See ``vs_oracle.c`` for the arithmetic and its citations.
"""

from .oracle import *  # noqa: F401,F403
from .oracle import __all__  # noqa: F401
from .cooled import cooled_labels  # noqa: F401
