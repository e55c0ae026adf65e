"""Plain FP64 CPU oracle for the explicit phase-field step (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it.
"""
