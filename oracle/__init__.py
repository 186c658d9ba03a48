"""FP64 CPU oracle of the Green's-function pixel-by-pixel optimizer.

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / --impl reference legs.  The CUDA product path never imports it.
"""
