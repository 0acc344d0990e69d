"""ORACLE -- test infrastructure only.

CPU reference of the QQMC estimator (complex128, naive Keldysh sum with a
pivoted LU per configuration).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product package
never does, and this package imports nothing from the product.
"""
