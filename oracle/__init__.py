"""CPU oracle for the AMS-sort hot path (test infrastructure only).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The product path (the
CUDA library and its Python binding) never imports, links or calls anything here,
and this package imports nothing from the product path; the two share only the
seeded input generators, which hold none of the method's arithmetic.

Everything here is plain, single-threaded numpy / Python written from
Axtmann, Bingmann, Sanders, Schulz, "Practical Massively Parallel Sorting"
(SPAA'15): Section 1 (output definition), Section 2 and Appendix D (tie
breaking), Section 4.2 (fast work-inefficient sorting by all-pairs ranking),
Section 6 (AMS-sort: sampling, splitters, partitioning, bucket grouping, Lemma on
the scanning algorithm, recursion, base case) and Appendix C (bucket grouping).

Two layers:

* ``sort_keys`` / ``sort_pairs`` / ``sort_segmented`` -- the *definition*: the
  unique permutation ordered by (transformed key, original index).  The method
  reaches exactly this result, so this is the parity reference for every output.
* ``sample`` / ``rank_sort`` / ``splitters`` / ``classify`` / ``bin_pack`` /
  ``pieces`` / ``ams_sort`` -- the algorithm's steps in the paper's order, used to
  pin the intermediates of each kernel (same seeds, same parameters).

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
against brute force, closed forms, library routines or the paper's lemmas.
"""
from .ams_oracle import *  # noqa: F401,F403
from .ams_oracle import __all__  # noqa: F401
