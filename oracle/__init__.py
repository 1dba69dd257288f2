"""FP64 CPU oracle for polynomially preconditioned f(A)b, f(z) = z^{-1/2} or z^{1/2}.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library; the only module both sides use is
``synth`` (seeded input generators, no arithmetic of the method).

Layout
  operators  sparse test matrices (2D/3D Dirichlet Laplacians, 3D upwind
             convection-diffusion) built as Kronecker sums, plus their
             closed-form 1D eigen-decompositions.
  exact      x* = A^{-1/2} b / A^{1/2} b by plain definitions: dense
             eigendecomposition or Schur square root (tiny n), the sine-basis
             closed form (Laplacians and, by diagonal similarity, the 1D-
             separable convection-diffusion operator), diagonal A.
  chebyshev  the Chebyshev preconditioning polynomial q ~ z^{-1/2} on [a,b]
             (Sec. 5.1) and the quantities of Prop. 3.2 / Example in Sec. 3.2.
  krylov     Algorithm 1 (left) and Algorithm 2 (right) polynomially
             preconditioned Arnoldi / Lanczos, the stopping rule of Sec. 6,
             and plain unpreconditioned Arnoldi as a large-n reference.
  ritz       interpolation at Ritz / harmonic Ritz values in Newton form at
             Leja-ordered nodes (Sec. 5.2).
  lsq        least-squares polynomials on a contour (Sec. 5.3).
  wilson     the Wilson-type lattice operator D (with chemical potential),
             A = D^H D, Q = Gamma_5 D and free-field closed forms.
  sign       sign(Q) b = Q (Q^2)^{-1/2} b and the overlap operator (Sec. 6,
             Example 2).

Every function is FP64 (complex128 where the data is complex) and follows
the paper passage named in its docstring.  Pins for all of it live in
tests/test_oracle_*.py.
"""
