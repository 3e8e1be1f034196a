"""FP64 CPU oracle of the dynamic-OT primal-dual method (arXiv 1501.04840).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check in
__graft_entry__.py and by the CPU-baseline leg of bench.py.  The CUDA product
path never imports, links or runs anything in this directory.

Parity pins of every function: tests/test_oracle_operators.py,
tests/test_oracle_projection.py, tests/test_oracle_prox.py and
tests/test_oracle_solve.py.
"""
from .dynot import *  # noqa: F401,F403
from .dynot import Grid, State, rgb_grid, hue_grid, NEUMANN, PERIODIC  # noqa: F401
