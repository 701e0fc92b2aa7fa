"""FP64 CPU oracle of the dimension-weighted FMM -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs import this package.  The library never does.
"""
from . import dwfmm_oracle  # noqa: F401
