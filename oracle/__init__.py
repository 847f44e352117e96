"""FP64 CPU oracle for the lumped-mass metric-graph Gaussian random field sampler.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's CPU
baseline may import this package. The product path (the CUDA library and its
Python binding) never imports, links or runs anything here, and this package
never imports the product path. The two share only the seeded graph
generators in `grf_inputs`, which hold none of the method's arithmetic.

What it computes (Kovacs, Molnar, Szaraz, "Efficient generation of Gaussian
random fields on metric graphs via domain decomposition and mass matrix
lumping"):
  * mesh and DOF map (Sec. 3, Phase 1),
  * lumped mass M_L and P1 stiffness G, assembled element by element over the
    whole graph (Sec. 3, Phase 2),
  * white noise b = M_L^{1/2} xi with xi from Philox4x32-10 + Box-Muller
    (Eq. wh_def with the lumped factor of Sec. 2.5),
  * the sinc quadrature of the Balakrishnan integral (Eq. 3-4 and the
    quadrature limits of Sec. 4.1),
  * the sampled field U = sum_l (c_I^(l) M_L + c_L^(l) K)^{-1} b with
    K = kappa^2 M_L + G (Eq. spde_approx_fem), each shifted system solved by a
    global sparse direct factorisation (scipy's SuperLU) -- no domain
    decomposition, no Schur complement, no PCG.

Parity pins: every function is pinned by a `-m "not gpu"` test against a fact
that does not come from this package (closed forms, published known answers,
the paper's table values, dense eigen-decompositions, Monte-Carlo moments).
"""

