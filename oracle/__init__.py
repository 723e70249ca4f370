"""Plain FP64 CPU oracle for the HDG static-condensation hot path (arXiv 1807.00086).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may import it. It shares no
code with the CUDA library under ``paper_1807_00086_gb300/`` and never imports it; the
two meet only through the seeded input generators in ``paper_1807_00086_gb300.inputs``
(which hold none of the method's arithmetic) and through plain arrays.

Everything here is written for readability against the paper, not for speed:
element blocks are formed by quadrature in physical coordinates, each element is
factorised with partial-pivot LU, the condensed trace system is assembled as a sparse
matrix and solved directly.

Module map
  reference.py  quadrature rules and orthonormal simplex bases (Sec. 2.2 spaces)
  acoustic.py   acoustic HDG scheme: skeleton (Sec. 2.1), local blocks, static
                condensation (Sec. 2.4, Eq. LS), recovery, BDF / DIRK marching
                (Sec. 2.3, Eqs. 9b and 10), monolithic brute force, energy identity.

Parity status: every function is pinned by a test in tests/test_oracle_*.py against
closed forms, brute force or invariants. The workload conventions (Ricker wavelet, point-source
element, the elastic Gaussian-bump initial data) are stated in acoustic.py and elastic.py;
the first two are pinned too.
"""
