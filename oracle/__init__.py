"""CPU fp64 oracle for the RSF Gaussian-process likelihood path.

ORACLE -- test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import anything in this package;
the product path never does.  It shares no code with the CUDA path.
"""
