"""FP64 CPU oracle for the AD-PRD operator of arXiv 2505.20968 (Riva et al.).

Test infrastructure, not product code: only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline leg may import anything under oracle/.  The CUDA
library never calls into this package and shares no code with it; both read
their inputs from paper_2505_20968_gb300.inputs, which holds no arithmetic of
the method.

The oracle computes, plainly and slowly, the discrete operator the library
implements, module by module:
  * faddeeva      W(a,v) = w(v + i a)                 (Sect. 2.4)
  * spline        natural cubic spline, constant extension (Sect. 6.2)
  * geometry      angular grid, scattering angles, polarisation basis (Sect. 4.2)
  * atom          two-level / two-term atom with Paschen-Back levels (Sect. 2.2)
  * redistribution  F, G tiles against the spline basis; R_III profiles
                  (Eqs. RQIIKKp, G, RIIIQKKp; App. C)
  * preconditioner  P = Id - Lambda* Sigma* and its block inverse (Sect. 5.2, App. F)
  * problem       K, eps_th, DELO-linear Lambda, Sigma, Kirchhoff
                  normalisation, GMRES, emergent Stokes (Sects. 2.6-2.7, 3, 4, 5;
                  App. B, E)
                  and the transposed operator A^T = Id - Sigma^T Lambda^T
                  with its GMRES solve (not in the paper: the adjoint)
"""
