"""FP64 CPU oracle for the minimal-rank H^2 VIE matrix-vector product.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it. It shares no code with the CUDA library; both sides only
share the seeded inputs of the ``synth`` module.

Contents (each function cites the passage of Omar & Jiao, "O(N) iterative and
O(N log N) fast direct volume integral equation solvers with a minimal-rank
H^2-representation", that it follows):

  vie      pulse-basis E-field VIE operator Z = I - K diag(chi)   (Sec. II.A)
  tree     cluster tree by balanced bisection, strong admissibility
           partition                                              (Sec. III.A)
  h2build  truncated-SVD minimal-rank nested H^2 build            (Sec. III.C)
  h2mv     dense and H^2 matrix-vector products                   (Sec. IV.B)
  krylov   restarted GMRES(m) with modified Gram-Schmidt
  conv     direct 3-D convolution forward/backward (learned preconditioner)

Every function is written for clarity, not speed, in float64/complex128.
Parity status of each function is stated in its module header.
"""
