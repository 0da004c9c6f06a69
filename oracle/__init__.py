"""FP64 CPU oracle of the iterative FSA method — test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package; the product path never does.
"""
from .fsa_oracle import *  # noqa: F401,F403
