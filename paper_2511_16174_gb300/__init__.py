"""GB300-native two-stage symmetric eigensolver (successive band reduction pipelined
with bulge chasing, on-device divide and conquer, blocked back-transformation).

The compute path is the C-ABI library ``libevd`` built from ``csrc/``; the Python
module :mod:`paper_2511_16174_gb300.evd` marshals arguments to it and nothing else.
"""
__all__ = ["evd", "inputs"]
