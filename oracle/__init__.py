"""Plain, slow FP64 CPU oracle for the purified quantics Lindblad step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library and
its Python binding) imports, calls or links anything in this package.  Only the
test suite, the smoke check in ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path.

Modules
-------
dense  -- dense density-matrix integrator of the Lindblad equation (Eq. 1) with
          the first-order Kraus scheme of Sec. V.B (H_eff, U_1, K = U + h L) and
          the trace renormalisation; observables; the vectorised superoperator
          (brute force) and the continuous Lindbladian used as pins.
qtt    -- quantics encoding (Sec. II.A), plain TT-SVD of vectors and operators
          (Eq. MPS, Sec. II.B) and MPO ranks (Table I).
mps    -- the purified MPS algorithm itself written out in numpy: stacked Kraus
          MPO applied site by site (Sec. V.B with the matrix addition of
          Sec. V.A), bond compression by SVD, purification-rank truncation
          (Sec. IV.A) and renormalisation.  Used to check the truncated form.

Every function cites the passage of the paper it follows.  Where the paper is
silent or garbled the reading taken is stated in the docstring.
"""
