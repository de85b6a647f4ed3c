"""FP64 CPU oracle of arXiv 2404.18034's SCP + CTCS + PIPG path.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
CPU-baseline leg of the benchmark, never by the solver itself.
"""
from .pdg_oracle import *  # noqa: F401,F403
from .pdg_oracle import build, lib  # noqa: F401
