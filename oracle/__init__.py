"""Plain, slow, FP64 CPU oracle for the Laplace-domain elastodynamic BEM frequency solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its Python
binding) imports, calls or links anything in this package.  Only the tests, the smoke check of
the entry module and the CPU-baseline leg of the benchmark use it.  It shares no code with the
CUDA path: every formula here is written out independently from the paper (Xiao, Rong, Ye,
Zhang, "An efficient adaptive frequency sampling scheme for large-scale transient boundary
element analysis") and from textbook mathematics where the paper omits it.

Modules
  kernels     Laplace-domain fundamental solutions U*, T* (Sec. 2.1, Eq. (bie); the paper omits
              the formulas and points to textbooks: the Laplace-transformed Stokes solution)
  quadrature  triangle rules (4-pt degree 3, 7-pt degree 5), Gauss-Legendre, Duffy map
  bem         element geometry, near lists, element integrals, dense assembly of A(s) a = b(s)
              (Sec. 2.1, Eq. (Aa_b)) and its LU solution
  closed_form pressurised spherical cavity in a full space (pin, exact Laplace-domain solution)
  fsm         Fourier-series-method inverse Laplace transform (Sec. 2.2, Eqs. (invLap),
              (IDFT-MFT))
  vf          vector fitting (Sec. 2.3, Eqs. (vf-f), (vf-td))
  afs         adaptive frequency sampling driver (Sec. 3, Eqs. (snew)-(converge), Algorithm AFS)
  mlp         POD basis and the small MLP warm-start model, forward/backward/Adam in FP64
  hmatrix     hierarchical low-rank far field (the fast matrix-vector product's role, Sec. 2.1):
              the dense 4-point far field it approximates, cluster tree, block partition,
              adaptive cross approximation and the H-matrix product
"""
