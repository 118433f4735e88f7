"""Brute-force FP64 reference renderer (the oracle): test infrastructure only.

Only tests/, the smoke check and the CPU-baseline leg of the benchmark import
this package.  The CUDA product path never does.
"""
