"""Plain FP64 CPU oracle for the randomised primal-dual (PD-R) RI imaging path.

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously correct reference
against which the CUDA path is checked. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (the C-ABI library and its Python binding) never imports, links
or calls anything in here, and this package never imports the product path.

Modules (each function cites the passage of arXiv:1610.08895 it follows):

* ``measurement`` -- Phi = G F Z and its adjoint (Sec. 2, measurement model;
  Sec. 3, data split eq. (data-split)).
* ``wavelets``    -- the SARA collection Psi of b orthonormal bases (Sec. 3).
* ``prox``        -- P_B (eq. proj-L2), S_alpha (eq. prox-L1), P_C (eq. proj-plus).
* ``philox``      -- counter-based draws for the active sets (Alg. 1 step 3).
* ``adaptive``    -- adaptive selection probabilities (Sec. 4, eq. prob-choice).
* ``pd``          -- Algorithm 1 (PD-R) step by step, and the power method (Sec. 5).
* ``experiment``  -- noise level and the chi-square bounds epsilon_i (Sec. 5).

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except the multi-iteration PD-R trajectory itself,
whose components are pinned but whose sequence has no printed values in the
paper; the converged point is pinned against an independent solver instead.
"""
