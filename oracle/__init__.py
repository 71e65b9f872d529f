"""CPU oracle for the SimpleX2 DCT sweep (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: its C sources live here, are compiled here with gcc and are called
through ctypes.
"""
from .oracle import *  # noqa: F401,F403
