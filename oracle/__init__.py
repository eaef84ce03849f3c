"""FP64 CPU oracle for the Spectral Difference (SD) residual with BR1 and compact
viscous fluxes (Lodato & Tonicello, "A novel compact scheme for second-order fluxes
applied to the Spectral Difference method").

TEST INFRASTRUCTURE ONLY. This package is the slow, plain, obviously-correct
definition that the CUDA path is checked against. Only the test-suite, the smoke
check of the package entry point and the CPU-baseline leg of the benchmark may import
it. The product path (the C-ABI library and its Python binding) never imports,
links or calls anything here, and this package imports nothing from the product.

Every array is float64 (complex128 where a Bloch analysis needs it). Each function
cites the section / equation of the paper it follows.

Modules:
  operators  - solution/flux points, Lagrange extrapolation L and derivative M (Sec. 2.1)
  grid       - periodic uniform Cartesian element grid, J and S = adj(J) (Eqs. ns:mapped, adj:f)
  physics    - heat, porous-medium and compressible Navier-Stokes fluxes (Secs. 4.3, 4.4)
  residual   - the SD semi-discrete residual, BR1 (Sec. 2.1) and compact (Secs. 2.2, 2.3)
  curvilinear- periodic grids of trilinear hexahedra (Sec. 2 mapping, K = 8), per-point
               metric terms and the residual on them (Sec. 2.3 steps with [S]^{Fd}, [J^-1]^S)
  timestep   - RK4, SSPRK(5,4) and the 5-stage low-storage RK (Sec. 4.4 time integration)
  diagnostics- kinetic energy, enstrophy, conserved totals (Sec. 4.4)
  bloch      - the temporal-eigenanalysis operator B(theta) of Sec. 3 (used as a pin)
  mlp        - the per-element MLP closure forward/backward in FP64

Parity status per function is stated in each module header ("pinned by" lists the
tests that tie the function to something other than itself).
"""
