"""CPU oracle for the HGKS hot path (test infrastructure only).

Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
may import this package.  The product path never does.
"""
