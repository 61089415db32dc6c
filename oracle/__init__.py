"""Plain FP64 CPU oracle of the lattice Boltzmann squirmer method.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path
(``paper_1903_04799_gb300``) never imports it.
"""
from .oracle import OracleSim, build_oracle, load_oracle  # noqa: F401
