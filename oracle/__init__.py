"""Plain, slow FP64 CPU oracle for the partitioned network expansion (PNE).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path; its only common dependency is the seeded
input module ``paper_2512_10910_gb300.inputs`` (geometry and tensors, none of
the method's arithmetic).

Contents (each function cites the passage it follows):
  bp.py         message passing, boundary reflection, rank-1 projectors
                (Eq. A7, Sec. II.B, Sec. III.D, App. B)
  enumerate.py  cluster enumeration (bitmask scan; per-anchor level growth in
                ``enum_oracle.c``) and vertex-disjoint term tuples (Eq. A4)
  expansion.py  cluster/term values in the ORIGINAL basis with explicit P and
                Q = I - P matrices, per-order Neumaier sums, the full PNE
                pipeline, open-index output (Eq. A2-A4, Sec. III.A, III.D)
  exact.py      exact contractions used as truth (Eq. A1, Eq. B1, Eq. B2):
                whole-network einsum, site-by-site sweep with log scaling,
                literal Ising spin sums, the Ising high-temperature closed form
                and Onsager's free energy.
  combinatorial.py  multi-index partitions with factorised rank-1 projectors
                and the combinatorial form (Eq. A6, A8-A10): every sub-network
                contracted as written, the residue with the non-factorising
                complements inserted directly, and the linear form over
                partitions (Eq. A4).
  weights.py    weight passing (App. C) and expansions with rank-r projectors
                onto the largest weights (Sec. V), linear and combinatorial.
  recursive.py  recursive partitioning (Sec. IV.A): the combinatorial form
                whose too-large sub-networks are expanded again over the
                second-level partitions that fit inside them.
  strips.py     the infinite-lattice strip expansion (Sec. IV.C): uniform BP,
                strip transfer-matrix eigenvalues (LAPACK / ARPACK), capped
                patches by einsum and by row sweeps, and the per-cell sums over
                the 2L strip partitions (1D and 2D forms).

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (closed forms, brute force, exact identities).
"""
