"""CPU FP64 oracle for the fast multitask Gaussian process hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls, links or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA library; both sides consume the same seeded inputs.

Modules
  design    design points (Def. 2.1 lattices, Def. 2.2 digital sequences) and the
            univariate SI / DSI kernels (Eq. 2.4 product form, Eq. 2.5, Eq. 2.6).
  dense     the plain definition: dense Gram matrix (Eq. 3.1, Sec. 3.1), dense
            Cholesky, optimal means (Eq. 3.4), MLE loss (Eq. 3.3), its analytic
            gradient and the posterior (Eq. 3.2).
  spectral  the fast-MTGP structure (Thm. 3.1 / Thm. FMTGP_computations), the
            inverse / log-determinant of Lambda-tilde by Algorithm 1 in the paper's
            step order, and per-frequency / per-residue-class dense solves for sizes
            the dense oracle cannot hold.
  exact     exact rational determinant (fraction-free Bareiss elimination) for N <= 64.

Parity unpinned: nothing here; every function is pinned by a ``-m "not gpu"`` test
(see tests/test_oracle_*.py).
"""
