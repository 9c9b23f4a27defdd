"""CPU oracle of the semi-coherent F-statistic path (test infrastructure only).

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import anything from this package; the product package never does.
"""
