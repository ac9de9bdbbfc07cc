"""CPU oracle for the smallest eigenpairs of a graph Laplacian (FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
CUDA library never calls it and shares no code with it; the only shared module
is ``graphgen`` (seeded inputs, no eigensolver arithmetic).

Contents, each following the paper (Bergamaschi, Bozzo, Franceschet,
"Computing the smallest eigenpairs of the graph Laplacian", arXiv 1311.1695):

* ``laplacian`` -- L = D - A (Section 2), its action, the quadratic form
  (Eq. 1) and the 1-norm used to normalise residuals.
* ``dense``     -- the definition: the k smallest eigenpairs of L restricted
  to the complement of the constant vector, by dense symmetric eigensolve.
* ``jd``        -- Jacobi-Davidson, Algorithm 2 with deflation (Eq. 5),
  restart (m_min, m_max) and the projected PCG correction (Section 3.2).
* ``dacg``      -- Deflation-accelerated conjugate gradient, Algorithm 3.
* ``irlm``      -- Lanczos on the pseudo-inverse with implicit restarts,
  Algorithm 1 (right) and Section 3.1.1.
* ``blockops``  -- the per-step definitions the GPU kernels are compared with
  (Laplacian SpMM, projection, Gram products, CGS2, Rayleigh-Ritz, residuals,
  projected PCG correction).
* ``rng``       -- SplitMix64, the counter-based generator both sides
  implement for start vectors.
* ``gnn``       -- forward and backward of the warm-start message-passing
  network and its subspace loss, in FP64.
"""
