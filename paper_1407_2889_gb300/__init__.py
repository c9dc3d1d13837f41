"""GB300-native multi-pattern scan: Aho-Corasick DFA and Wu-Manber over a text.

The compute path lives in ``libpmscan.so`` (C-ABI, hand-written sm_103a
kernels); :mod:`paper_1407_2889_gb300.pmscan` is the thin binding over it.
Importing this package does not load the library; using the binding does,
and it raises if the library has not been built.
"""
__all__ = ["pmscan", "synth"]
