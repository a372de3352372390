"""FP64 CPU oracle for the HSE Fock-like exchange path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may
import this package.  The CUDA library and its Python binding never do.
"""
from .hse_oracle import *  # noqa: F401,F403
from . import ortho  # noqa: F401
