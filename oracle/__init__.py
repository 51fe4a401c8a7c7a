"""CPU oracle for the local parallel two-grid finite element method (Algorithm 3) for the
transient triple-porosity Navier-Stokes model.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct FP64
implementation written from the paper (Sec. 2, Sec. 3.1, Algorithm 3 of Sec. 5) with
NumPy/SciPy.  It shares no code with the GPU library and must never be imported by the
product path: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.

Modules
  quad    quadrature rules (7-point degree-5 triangle rule, Gauss-Legendre on edges)
  mesh    structured right-triangle meshes, P2/P1 numbering, subdomains (Alg. 3 Step 2)
  fe      P2/P1 reference elements and element integrals of the weak forms (Sec. 3.1)
  mms     manufactured solutions and the data they induce (forcing, boundary, interface)
  scheme  Algorithm 3 (coarse step, local corrections, glue) and a global fine
          linearised solve used as a brute-force check
  mesh3d, fe3d, mms3d, scheme3d
          the same in 3D: Kuhn tetrahedral meshes, P2/P1 tetrahedra with a collapsed
          Gauss-Jacobi rule, Gamma faces at z = 1, the 3D manufactured solutions, Algorithm 3

Parity status: every routine is pinned by a CPU test (closed forms, invariants, exact
polynomial reproduction, brute force, convergence rates) except the paper's printed
error tables, which use different elements (MINI/P1) and are therefore "parity
unpinned" to digits; only rates are compared.
"""
