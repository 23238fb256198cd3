"""Plain FP64 CPU oracle for MBE(3)-OSV-MP2 (arXiv 2106.06149).  Test infrastructure only: imported by tests/,
the smoke check in __graft_entry__ and bench.py's CPU-baseline leg, never by the product path."""
from .osvmp2 import *  # noqa: F401,F403
from .osvmp2 import __all__  # noqa: F401
