"""Plain, slow FP64 CPU oracle for TR-ALS-Sampled (Malik & Becker, ICML 2021).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import it. The CUDA library never
calls it, and it shares no code with the CUDA path: it is written from the paper's
definitions and algorithms in NumPy FP64, one step per stated operation.
"""

from .trals_oracle import *  # noqa: F401,F403
