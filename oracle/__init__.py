"""CPU oracle for the typicality + block-Lanczos estimator of rho*_s and H*.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it. It shares no code with the CUDA
library (no kernels, headers, helpers, tables or constants); the two meet only in
the seeded input specifications of the ``workloads`` module.

Everything here is plain float64 NumPy written from the paper (Chen & Cheng,
arXiv:2204.08147):

  ``spin_ops``     eq. Ht and the Kronecker convention of Sec. 2.2 (dense and
                   tensor-leg matrix-free forms of H_t, H_s, H_b, H_sb);
  ``exact``        the naive method of Sec. 2.4: exact diagonalisation plus an
                   explicit partial trace (the definition of rho*, eq. 4/5);
  ``rng``          the counter-based bath-vector generator (SplitMix64 on a
                   counter) shared by definition, not by code, with the library;
  ``lanczos``      Algorithm 1 (block Lanczos), eq. fT / trB_est / rho_est and the
                   E0 shift of Sec. 3.2, plus the Gram (function-application) form;
  ``closed_form``  App. C (isotropic XY chain, N_s = 2);
  ``post``         H* through eigenvalues (Sec. 3.2 end) and the von Neumann
                   entropy (Sec. 5.3.1).

Pins (tests marked "not gpu") tie each function to something other than itself:
the App. C closed form, textbook two-site spectra, brute-force matrix elements,
symmetry and limit cases (Sec. 2.3), polynomial exactness of the quadrature
(Sec. 4.2) and exhaustive-basis exactness of the estimator (Sec. 2.1).
"""
