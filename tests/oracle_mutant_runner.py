"""Run every oracle pin against a compiled oracle variant; exit 0 iff all hold.

Invoked in a subprocess by ``tests/test_oracle_mutants.py`` so that a planted
mistake that crashes or loops cannot take the test session down with it.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import ctypes  # noqa: E402

import oracle  # noqa: E402
from tests import oracle_pins  # noqa: E402

if __name__ == "__main__":
    lib = oracle._bind(ctypes.CDLL(sys.argv[1]))
    failed = oracle_pins.run_all(lib)
    for f in failed:
        print(f)
    sys.exit(1 if failed else 0)
