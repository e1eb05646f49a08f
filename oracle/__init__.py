"""Plain, slow FP64 CPU oracle for BlockBP (test infrastructure only).

This package restates the BlockBP method of the thesis (Ch. 2, Eq. of the
BlockBP update, Alg. 1) in NumPy complex128, step by step and without any
blocking, fusion or reordering beyond what the method states.  It is the
reference the CUDA path is checked against.  It shares no code with the CUDA
path: only the seeded input generators in ``synthetic`` serve both.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything from here.

Modules
-------
geometry  lattices, blocks, faces, regions (Sec. 2.2.2, Sec. 2.3.1, App. A)
tn        double-layer fusion, MPS helpers, boundary-MPS sweep (Sec. 1.1.3)
blockbp   the BlockBP iteration and local observables (Sec. 2.2, Alg. 1)
bp        site-level BP (Eq. of BP) used as a pin: 1x1 blocks reduce to it
exact     brute-force exact contraction of small finite lattices
core      core extraction: two opposing bubbles, the zipper into a pMPS, the
          Edge TN of a bond (Sec. 2.3, "Core", "Edge")
ite       imaginary time evolution: two-site gate, ALS on the Edge TN, full
          ITE over a block (Ch. 3, Alg. 2)
hexagonal hexagonal Kagome blocks of face-length N: geometry, the six
          contraction orders, BlockBP on them (Sec. 2.3.1, Sec. 2.3)

Parity status: every function is pinned by ``tests/test_oracle_*.py`` except
the loopy configurations themselves, which have no closed form: the BlockBP
fixed point of a loopy network ("parity unpinned" for that value as such;
its ingredients are pinned, and tree-of-blocks cases are exact).
"""
