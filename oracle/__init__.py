"""Plain FP64 CPU oracle of the paper's edge-matrix AMG (Kogler & Schoeberl).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with
the CUDA library; the only common dependency is the seeded input generator
(``workloads``), which holds none of the method's arithmetic.

Modules, each following the paper's section noted in its header:

* ``topology``    Sec. 3-4: Skew, kernel transfer Q, auxiliary matrix,
                  finest edge matrices (Thm. deng_elast), coarse edge/vertex
                  matrices (Thm. cemats).
* ``criteria``    Sec. 5: mu_D, mu_s, mu_p (Lemma mu2), mu_g (Thm. mu1).
* ``coarsening``  Sec. 5.2: Algorithm 1 (successive matching).
* ``prolongation`` Sec. 3 Def. pwp / pwp_el, Sec. 6 Def. aux_sp.
* ``solve``       Sec. 3 Algorithm tg (two-grid / V-cycle), the block-l1
                  smoother of Sec. 7, the coarsest-level regularisation of
                  Sec. 3 after Lemma eet_is_diag, Galerkin products, PCG.
* ``hierarchy``   multi-level setup driver.
* ``learned``     FP64 reference of the per-vertex learned smoother (MLP
                  forward/backward, patch-inverse targets).

Parity unpinned: the exact hierarchy (agglomerates, coarse sizes, iteration
counts) cannot be pinned to the paper, whose meshes and parameters sigma /
omega are not given; every function the GPU path is compared against is
pinned by the tests in ``tests/test_oracle_*.py``.
"""
