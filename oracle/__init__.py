"""CPU oracle for the multilevel linearized-buckling solver path (test infrastructure only).

This package is a plain, slow, FP64 restatement of what the paper computes, written to be checked
by eye against the paper (Ferrari & Sigmund, "Towards solving large-scale topology optimization
problems with buckling constraints at the cost of linear analyses"):

  elements.py     element matrices K_e0, G_e0[u_e] and the adjoint element vector (Sec. 2)
  grid.py         structured-grid numbering, element connectivity, level geometry
  assembly.py     sparse global K[x], G[x,u] with the SIMP interpolations (Sec. 2)
  transfer.py     explicit bi/trilinear interpolation I^j_{j+1} between nested grids (Sec. 2.1)
  lba.py          linear analysis, exact LBA (Algorithm 1), multilevel LBA (Sec. 2.1 steps 1-4)
  sensitivity.py  adjoint systems and buckling-load-factor sensitivities (Sec. 2)

It is test infrastructure: only the tests, the smoke check and the CPU-baseline leg of the benchmark
may import it.  The GPU library never imports, links or calls it, and it shares no code with the
GPU library.  Every function cites the passage of the paper it follows.
"""
