"""FP64 CPU oracle for the 3DGS render hot path -- test infrastructure only.

Importable by tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg;
never by the product package.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build, lib  # noqa: F401
