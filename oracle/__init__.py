"""FP64 CPU oracle for the unbalanced Beckmann-OT proximal path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and it shares no code, table or
helper with the CUDA path: the two meet only at the seeded inputs of ``synth``.

Plain, slow, obviously correct NumPy in float64, following the paper
(Lee, Bertrand, Rozell, "Parallel Unbalanced Optimal Transport Regularization
for Large-scale Imaging Problems", arXiv:1909.00149):

* ``grid``        -- divergence D and its adjoint D* (Sec. III-A), the l_{2,1}
                      norm, the Neumann Laplacian spectrum (Theorem 1).
* ``prox``        -- Algorithm 1 (Sec. III-B), its stopping rule and the
                      duality-gap certificate of eq. (Prox_UOT).
* ``dct``         -- the orthonormal DCT-II by its defining sums and the
                      Neumann-Laplacian solve it diagonalises.
* ``projection``  -- the same prox (eq. Prox_UOT) by ADMM with an exact
                      projection onto the constraint set, using ``dct``.
* ``svt``         -- one-sided Jacobi SVD and singular-value thresholding
                      (Sec. IV-B.1).
* ``rpca``        -- Algorithm 3 (RPCA+UOT-DF) with Phi_t = I.
* ``unet``        -- direct-sum 3x3 convolution, pooling, upsampling and
                      their gradients (FP64) for the learned warm start.

Parity pins: every function is checked by ``tests/test_oracle_*.py`` against
closed forms, brute force and library routines, never against itself.
"""
