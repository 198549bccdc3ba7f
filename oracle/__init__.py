"""FP64 CPU oracle of the GCP-CROWN bound: test infrastructure only.

Imported by the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py``; never by the library itself.
"""
