"""FP64 reference oracle for the creeping-wave field evaluator.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (``paper_2310_10578_gb300``) never imports, links or runs
anything here, and nothing here imports the product package. The two share
only the seeded input generators in ``paper_2310_10578_gb300.scenes``, which
hold none of the method's arithmetic.
"""
