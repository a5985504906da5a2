"""ORACLE — test infrastructure, not part of the product.

A plain, slow, obviously correct CPU implementation of what the sparse-tiled DG elastic-wave
path computes: the untiled loop chain in FP64 (dg.py, exact rational reference element in
refelem.py), the sparse-tiling inspector of Algorithms 1-3 run sequentially (inspector.py over
inspector.c) and a brute-force schedule-legality checker (checker.py).  It shares no code with
the CUDA library; only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may use it.
"""
