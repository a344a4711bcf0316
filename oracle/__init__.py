"""CPU oracle of the BP RI-OEDG stage (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.
"""
