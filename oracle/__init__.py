"""CPU oracle of the fast matrix multiply -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline legs
import this package; the library's product path never does.
"""
from .fmm_oracle import *  # noqa: F401,F403
