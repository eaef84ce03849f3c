"""Periodic uniform Cartesian element grid and its metric terms (paper Sec. 2,
Eqs. ns:mapped and adj:f; the 1D case of Sec. 2.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Array layout used throughout the oracle (and, identically, by the C-ABI):
    U[var][E_{dim-1}]...[E_0][n]...[n]
i.e. variable-major, then the element grid with x fastest, then the n^dim points of
each element with the x point index fastest. In 3D: U[var][ez][ey][ex][k][j][i].

For a linear (affine) element x = x_lo + (h/2)(xi + 1) per axis, the Jacobian matrix is
diag(h_d/2), J = prod_d h_d/2 and S = adj(J_matrix) = diag(J / (h_d/2)). In 1D this gives
J = h/2 and S = 1, as stated in Sec. 2.1.
"""
import numpy as np

from .operators import operators


class Grid:
    def __init__(self, dim, ne, lo, hi, p, dtype=np.float64):
        if dim not in (1, 2, 3):
            raise ValueError("dim must be 1, 2 or 3")
        ne = tuple(int(v) for v in ne)
        if len(ne) != dim or min(ne) < 1:
            raise ValueError("ne must give dim positive element counts (x first)")
        self.dim = dim
        self.ne = ne                      # (E_x, E_y, E_z)
        self.lo = tuple(float(v) for v in lo)
        self.hi = tuple(float(v) for v in hi)
        self.p = int(p)
        self.n = self.p + 1
        self.dtype = np.dtype(dtype)
        self.ops = operators(self.n, dtype)
        T = self.dtype.type
        self.h = tuple((T(self.hi[d]) - T(self.lo[d])) / self.ne[d] for d in range(dim))
        # metric terms of the affine map (Eq. adj:f)
        self.J = T(1)
        for hd in self.h:
            self.J = self.J * (hd / 2)
        self.Jinv = 1 / self.J
        self.S = np.zeros((dim, dim), dtype=dtype)
        for d in range(dim):
            self.S[d, d] = self.J / (self.h[d] / 2)

    # ----- axis bookkeeping -------------------------------------------------------
    def elem_axis(self, d):
        """Axis of the element index along direction d (0 = x) in U[var, ...]."""
        return 1 + (self.dim - 1 - d)

    def pt_axis(self, d):
        """Axis of the point index along direction d in U[var, ...]."""
        return 1 + self.dim + (self.dim - 1 - d)

    def shape(self, nvar):
        return (nvar,) + tuple(reversed(self.ne)) + (self.n,) * self.dim

    @property
    def n_elements(self):
        return int(np.prod(self.ne))

    @property
    def n_points(self):
        return self.n_elements * self.n ** self.dim

    def coordinates(self):
        """Physical coordinates of every solution point: list over d of arrays with
        the shape of one variable of U."""
        xs = self.ops.xs
        out = []
        for d in range(self.dim):
            shp = [1] * (2 * self.dim)
            e = np.arange(self.ne[d])
            shp_e = list(shp)
            shp_e[self.elem_axis(d) - 1] = self.ne[d]
            shp_p = list(shp)
            shp_p[self.pt_axis(d) - 1] = self.n
            x = (self.lo[d] + self.h[d] * e).reshape(shp_e) + \
                (self.h[d] / 2.0) * (xs + 1.0).reshape(shp_p)
            out.append(np.broadcast_to(x, self.shape(1)[1:]).copy())
        return out

    def quadrature_weights(self):
        """J * prod_d w_{i_d} at every solution point (Gauss quadrature on each
        element), with the shape of one variable of U."""
        ws = self.ops.ws
        W = np.ones(self.shape(1)[1:])
        for d in range(self.dim):
            shp = [1] * (2 * self.dim)
            shp[self.pt_axis(d) - 1] = self.n
            W = W * ws.reshape(shp)
        return self.J * W

    def integrate(self, f):
        """Gauss-quadrature integral of point values f (shape of one variable)."""
        return float(np.sum(self.quadrature_weights() * f))
