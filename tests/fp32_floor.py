"""The FP32 error floor of the SD divergence (test helper).

R_v = -J^-1 sum_d M_d G_d is a sum of terms J^-1 M_if G_f whose size is the flux's, while
the result is the flux's divergence: where the flow is nearly solenoidal (Taylor-Green at
Ma = 0.1) the terms cancel to a far smaller number. Rounding each flux-point value to FP32
(unit roundoff u = 2^-24) perturbs R_v by about u times the sum of the terms' magnitudes, so
no evaluation that forms the flux-point values in FP32 beats

    u kappa_v,   kappa_v = || sum_d J^-1 |M_d| |G_d| ||_2 / || R_v ||_2

(norms over the points considered). kappa_v grows like 1/h: the terms scale with the
element's derivative operator, the residual does not. The CUDA kernels carry the momentum
flux with p - p0 (the constant p0 has zero discrete divergence), so kappa is taken with
that flux; the energy flux (rho E + p) u keeps its full size in both."""
import numpy as np

from oracle.physics import NavierStokes
from oracle.residual import residual

U32 = 2.0 ** -24


def conditioning(U, grid, scheme, prm):
    """(R, C): the oracle residual and, per point, sum_d J^-1 |M_d| |G_d| for each variable."""
    R, parts = residual(U, grid, scheme, NavierStokes(prm), return_parts=True)
    absM = np.abs(grid.ops.M)
    C = np.zeros_like(R)
    for d in range(grid.dim):
        G = parts["G"][d].copy()
        G[1 + d] -= prm.p0 * grid.S[d, d]
        ax = grid.pt_axis(d)
        C += grid.Jinv * np.moveaxis(np.tensordot(absM, np.abs(G), axes=([1], [ax])), 0, ax)
    return R, C


def kappa(R, C):
    """kappa_v over all points of R, C (arrays [v][...])."""
    return np.array([np.linalg.norm(C[v]) / np.linalg.norm(R[v]) for v in range(R.shape[0])])
