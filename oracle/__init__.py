"""CPU oracle for ABC rejection sampling of the paper's compartmental model.

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library in
``paper_2012_14332_gb300`` never imports it and shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build, lib  # noqa: F401
