"""CPU FP64 oracle of arXiv 2201.04560's coupled LBM + energy step.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the CPU
baseline of bench.py, never by the product package.
"""
