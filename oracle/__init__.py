"""FP64 CPU oracle (test infrastructure only).

Imported by the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` and nothing else.  It shares no code with the CUDA path.
"""
