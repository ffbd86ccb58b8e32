"""Plain FP64 CPU oracle of the Walk-on-Interfaces estimator.

Test infrastructure only: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the product path never imports it.
"""
