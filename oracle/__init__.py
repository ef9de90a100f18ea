"""CPU oracle for sliced tensor-network contraction — TEST INFRASTRUCTURE ONLY.

Plain complex128 C (``tn_oracle.c``) written from the paper's definitions, loaded through
``oracle.oracle``.  Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may use it; the GPU product path never imports it.
"""
