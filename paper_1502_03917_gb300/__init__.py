"""All-at-once multigrid for the Poisson control problem on GB300 (sm_103a).

The compute path is the CUDA library ``libaaomg.so`` behind the C ABI declared
in ``include/aaomg.h``; ``paper_1502_03917_gb300.aaomg`` is its thin ctypes
binding.  Importing this package loads nothing: the library is loaded on first
use and a missing library is an error, never a fallback.
"""
