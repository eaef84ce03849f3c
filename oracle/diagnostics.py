"""Volume diagnostics (paper Sec. 4.4: kinetic energy and enstrophy) and the
conserved totals, by Gauss quadrature over every element.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

E_k = 1/2 int u.u dOmega (the paper's definition, without rho), plus the
density-weighted 1/2 int rho u.u; enstrophy = int omega.omega with omega = curl u and
the velocity gradient obtained from the conservative gradient at the solution points
(Eq. w:e, which is the same for the BR1 and compact schemes):
    d u_i / d x_k = (d(rho u_i)/d x_k - u_i d rho / d x_k) / rho.

Pinned by tests/test_oracle_diagnostics.py: the Taylor-Green initial field has
E_k/|Omega| = u0^2/8 and enstrophy/|Omega| = 3/4 u0^2/L^2 (to the spectral
discretisation error), mass/momentum/energy totals against closed forms.
"""
import numpy as np

from .residual import gradient


def ns_diagnostics(U, grid):
    W = grid.quadrature_weights()
    rho = U[0]
    vel = [U[1 + i] / rho for i in range(3)]
    ke_paper = 0.5 * np.sum(W * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
    ke_rho = 0.5 * np.sum(W * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
    g = gradient(U, grid, 5)                  # g[k][v] = d U_v / d x_k
    du = [[(g[k][1 + i] - vel[i] * g[k][0]) / rho for i in range(3)] for k in range(3)]
    om = [du[1][2] - du[2][1], du[2][0] - du[0][2], du[0][1] - du[1][0]]
    enst = np.sum(W * (om[0] ** 2 + om[1] ** 2 + om[2] ** 2))
    return dict(
        ke=float(ke_paper), ke_rho=float(ke_rho), enstrophy=float(enst),
        mass=float(np.sum(W * U[0])),
        mom=[float(np.sum(W * U[1 + i])) for i in range(3)],
        energy=float(np.sum(W * U[4])),
        volume=float(np.sum(W)),
        nonfinite=int(not np.all(np.isfinite(U))),
    )


def scalar_diagnostics(U, grid):
    W = grid.quadrature_weights()
    return dict(mass=float(np.sum(W * U[0])), l2sq=float(np.sum(W * U[0] ** 2)),
                volume=float(np.sum(W)), nonfinite=int(not np.all(np.isfinite(U))))


def l2_error(U, Uexact, grid, mask=None):
    """Gauss-quadrature L2 norm of U - Uexact (one variable), optionally restricted to
    the points where mask is true (the ZKB footnote of Sec. 4.3 restricts the error to
    |x|^2 < 0.9 H)."""
    W = grid.quadrature_weights()
    d2 = (U - Uexact) ** 2
    if mask is not None:
        W = W * mask
    return float(np.sqrt(np.sum(W * d2)))
