"""CPU oracle for the IFMM hot path: plain NumPy, FP64, written from the paper.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import, call or run anything in this package; the product
path (paper_1905_10602_gb300) never imports it and shares no code with it.
"""
