"""FP64 CPU oracle for the probabilistic bond-based peridynamic hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the CPU-baseline leg of ``bench.py``; never by the product package. It shares
no code with the CUDA path (the two meet only in the seeded input recipes of
``pd_workloads``).

* ``pd_oracle.c`` (through ``core``): neighbour lists, boundary sets, bond laws,
  the explicit step and the peak-load quantity of interest, in plain FP64.
* ``field``: truncated Karhunen-Loeve random fields (Section 5), the Philox
  counter-based generator and the marginal transforms.
* ``mlmc``: the Monte Carlo / multilevel estimators (Section 4) and the
  multilevel inverse CDF (Section 7).

Parity status of every function is stated in its module docstring.
"""
from . import core, field, mlmc  # noqa: F401
from .core import build  # noqa: F401
