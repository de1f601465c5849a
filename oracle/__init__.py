"""Plain FP64 CPU oracle of the D3Q27 cumulant LBM step (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg
import this package; the product library never does.
"""
