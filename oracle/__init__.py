"""FP64 CPU oracle of the SRHD per-patch update (test infrastructure only).

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
may import this package; the product package never does.
"""
