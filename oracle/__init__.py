"""FP64 CPU oracle for the InFo-ESRF perturbation and mean updates.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA library and never reads a value produced by it.

Everything here is plain, slow, dense NumPy/SciPy in float64, written from
the paper (Armstrong & Grooms, "Data Assimilation With An Integral-Form
Ensemble Square-Root Filter"):

* ``localization``  Gaspari-Cohn localization and grid distances (Sec. 2.3,
  Sec. 5.2; GC function from Gaspari & Cohn 1999, Eq. 4.10).
* ``quadrature``    the elliptic quadrature rule (App. D,
  Eq. elliptic_quadrature_rule), the Gauss-Legendre rule
  (Eq. gaussian_quadrature_rule) and the rule choosing ell.
* ``filter``        ensemble anomalies (Eq. normalized_perturbations), the
  localized covariances (Eq. localized_state_covar, Sec. 2.3), the mean
  update (Eq. info_esrf_mean_solve), the perturbation update
  (Eq. info_esrf_perturbation_solve, solved densely) and the GETKF limit
  (Eq. modified_gain / Eq. getkf).
* ``pcg``           PCG (Golub & Van Loan Alg. 11.5.1 as cited in App. E),
  the limited-memory preconditioner and the randomized Ritz pairs (App. E).
* ``philox``        Philox4x32-10 (Salmon et al., SC'11) and Box-Muller, the
  counter-based generator the randomized eigensolver draws from.
* ``learned``       forward/backward of the learned preconditioner correction
  (gradient checks only).

Readings of garbled or silent passages are listed at the top of each module.
"""
