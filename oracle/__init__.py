"""FP64 CPU oracle for the quaternion T-product (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs import this package; the product path never does.
"""
from .qtp_oracle import *  # noqa: F401,F403
