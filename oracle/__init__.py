"""CPU FP64 oracle of hQR (arXiv:1809.10585, Alg. 1 and Alg. 2).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs.  The product path never imports it.
"""
from .core import *  # noqa: F401,F403
