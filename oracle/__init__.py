"""CPU FP64 oracle for the distance threshold search (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package; the CUDA library is independent of it.
"""
