"""FP64 CPU oracle of the 3DSS renderer -- test infrastructure only.

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference arm
of ``bench.py`` may import this package.  It shares no code with the CUDA
path and never imports it.
"""
from . import density, model, optim  # noqa: F401
