"""FP64 CPU oracle of SamBaTen (arxiv 1709.00668) -- test infrastructure only.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA path.
Every function follows the paper's steps in order; see `oracle/sambaten.py`
for the section map and the readings taken where the paper is silent.
"""
from . import csampling, sambaten  # noqa: F401
from .csampling import build  # noqa: F401
