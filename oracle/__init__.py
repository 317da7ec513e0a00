"""FP64 CPU oracle of the diffractive-storage forward model and its gradient.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.
"""
from .dos_oracle import *  # noqa: F401,F403
