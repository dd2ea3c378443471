"""Plain FP64 CPU oracle (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference`` arm) may import this package.
It shares no code with the CUDA library in ``paper_2506_09743_gb300``.
"""
from . import philox, qmc_oracle  # noqa: F401
