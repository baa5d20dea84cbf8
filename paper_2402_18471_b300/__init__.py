"""B300-native coagulation-fragmentation step (cuDisc Sec. 5) behind a C ABI.

The compute path is the CUDA shared library built from ``csrc/``; the Python
binding in :mod:`paper_2402_18471_b300.coag` only marshals arguments.
"""
__all__ = ["synth"]
