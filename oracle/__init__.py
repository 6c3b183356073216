"""CPU oracle for the machine-learned finite-temperature SP2 (MLSP2) hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It is
plain, slow and written to be checked against the paper by eye: FP64 NumPy,
library primitives (``eigh``, ``matmul``, ``solve``) used as single steps, no
blocking, fusion or algebraic re-arrangement beyond what the paper states.  It
shares no code, header, table or constant generator with the CUDA path.

Modules and the passages they follow (arXiv 2605.08523):

* ``fermi``    -- Fermi function (Eq. FD_Func), entropy function (Eqs. entropy,
                  entropy-matrix), D and S by eigendecomposition, the chemical
                  potential at a given filling, a pure-Python Jacobi eigensolver
                  for tiny cross-checks.
* ``tables``   -- the 26-layer MLSP2 coefficients printed in Appendix A
                  (beta0 = 1500, mu0 = 1/3).
* ``mlsp2``    -- the scalar and matrix MLSP2 recursions (Eq. mlsp2,
                  Eq. mlsp2-output, Alg. 1 without its inner flip), the entropy
                  recursion (Eqs. entropy expansion, entropy expansion-s) and the
                  alpha-rescaled ansatz (Sec. II B).
* ``rescale``  -- Gershgorin bounds (Appendix A), the normalisation
                  (Eqs. H', mu', beta'), the flip (Eq. flip), validity
                  (Eq. conditions), H0 (Eq. H0) and model choice (Sec. III,
                  workflow step 4).
* ``pipeline`` -- Alg. 2: density matrix and entropy of one Hamiltonian, plus
                  the method-exact references D_rec / S_rec on eigenvalues.
* ``sp2``      -- SP2 with known mu (Eq. sp2-mu), its MLSP2 embedding
                  (Appendix C), the layer-count estimate (Eq. layer count) and
                  the golden-ratio fixed point (Sec. IV B).
* ``lanczos``  -- spectral bounds tightened by a few Lanczos steps (counter-
                  based start vector, splitmix64), intersected with Gershgorin.
* ``newton``   -- the chemical potential for a prescribed electron count by
                  Newton-Raphson (Sec. III A 4, Eqs. g, dg, delta_mu; sign of
                  Eq. drho taken from the definition of D).
* ``train``    -- training: eigenvalue sampling (Sec. II C 1), residuals,
                  reverse-mode Jacobian, Levenberg-Marquardt with optional
                  geodesic acceleration (Sec. II C 2).
* ``altform``  -- the one-term form of the recursion (Eq. mlsp2_alt and its
                  output), its embedding into Eq. mlsp2 (Appendix on model
                  embeddings), the SP2 sequence in that form, the chain-rule
                  Jacobian, LM fit and method-exact references.
* ``skipsp2``  -- Skip-SP2 with one stored layer and one accumulator
                  (Sec. II A 3), the Appendix embedding of Eq. mlsp2, the
                  reverse-mode Jacobian, LM fit and method-exact references.

Readings of passages that are silent, garbled or inconsistent are stated in
the docstring of the function that takes them.

Pins (checked by ``tests/test_oracle_*.py`` against values the paper prints,
closed forms, invariants and brute force):  every function above is pinned;
the one exception is the accuracy of tables trained by ``train``,
``altform.lm_fit`` and ``skipsp2.lm_fit`` beyond the paper's printed targets,
which is "parity unpinned" (the paper prints no trained entropy table, no
Fig. 2 weights and no coefficients of the one-term form or of Skip-SP2); the
LM loops themselves are pinned by their acceptance property and their
Jacobians by central differences.
"""
