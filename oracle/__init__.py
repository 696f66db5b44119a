"""FP64 CPU oracle for MUFFIN (Ammanouil et al. 2019) -- TEST INFRASTRUCTURE.

A plain, slow, obviously-correct NumPy restatement of the paper's method used
only to check the CUDA library: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
nothing in the product path does.  It shares no code with the CUDA side.

Modules (each function cites the passage it follows):

* ``daubechies`` -- Daubechies scaling filters by spectral factorisation
  (the spatial dictionary of Sec. 4.2.1: union of the first 8 Daubechies bases);
* ``wavelets``   -- periodised orthonormal 2D DWT (Mallat layout), the union
  W_s and its adjoint;
* ``iuwt``       -- the isotropic undecimated wavelet transform (starlet), the
  alternative spatial dictionary named in Sec. 2.1;
* ``spectral``   -- the orthonormal DCT-II W_lambda (Sec. 4.2.1);
* ``convolution``-- H_l, H_l^T as circular convolutions (Eq. model), the
  Lipschitz constant beta;
* ``muffin``     -- step sizes (Sec. 2.2 step condition), the objective
  (Eqs. probopt, RegAll), Algorithm 2 (parallel MUFFIN update);
* ``sure``       -- Algorithms 3 and 4 (derivative iterates), PSURE-FDMC
  (Eq. PSURE0), SUGAR-FDMC (Eq. SUGAR), ADA-PT (Algorithm 5, Eq. adaptgrad);
* ``weights``    -- weights alpha_n, beta_l from an initial cube (Eq. 2regpar)
  and the global SUGAR gradient descent (Eq. globalgrad);
* ``metrics``    -- SNR and WMSE (Sec. 4.1).

Parity pins: every function is checked by ``tests/test_oracle_*.py`` against
closed forms, dense brute force, library special cases, finite differences
and Monte-Carlo expectations.  The values the paper prints for its own
datasets (tuned parameters, SNR, WMSE, Sec. 4.2.1) need data that is not
available, so no pin uses a printed number.
"""
