"""Independent plain-FP64 CPU oracle of the per-time-step test-particle update.

Test infrastructure: only the test suite, the smoke check and the CPU
baseline leg of the benchmark import this package.  It shares no code with
the CUDA library it checks.
"""
