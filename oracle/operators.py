"""Reference-element operators of the SD method (paper Sec. 2.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Pinned by tests/test_oracle_operators.py: polynomial exactness of L (degree <= p) and
M (degree <= p+1), row sums, Gauss exactness, and the closed forms of the compact
correction scalars alpha = c_L^T L M c_R = (-1)^p / 2 and beta = c_R^T L M c_L = -alpha.
"""
import numpy as np


def _gauss_legendre(n, dtype):
    """Gauss-Legendre nodes and weights; for extended precision the float64 rule is
    polished by Newton steps on the Legendre recurrence in that precision."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = np.asarray(x, dtype=dtype)
    if np.dtype(dtype) == np.float64:
        return x, np.asarray(w, dtype=dtype)
    one = dtype(1)
    for _ in range(3):
        p0, p1 = np.ones_like(x), x.copy()
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        if n == 1:
            p0, p1 = np.ones_like(x), x.copy()
        dp = n * (x * p1 - p0) / (x * x - one)
        x = x - p1 / dp
    p0, p1 = np.ones_like(x), x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    if n == 1:
        p0, p1 = np.ones_like(x), x.copy()
    dp = n * (x * p1 - p0) / (x * x - one)
    return x, 2 * one / ((one - x * x) * dp * dp)


def solution_points(n, dtype=np.float64):
    """n Gauss-Legendre points on [-1, 1] and their quadrature weights
    (Sec. 2: solution points follow the n-point Gauss-Legendre rule)."""
    return _gauss_legendre(n, dtype)


def flux_points(n, dtype=np.float64):
    """n+1 flux points: the Gauss-Legendre points of order n-1 plus the two end
    points -1 and +1 (Sec. 2). For n = 1 only the end points remain."""
    if n == 1:
        inner = np.zeros(0, dtype=dtype)
    else:
        inner, _ = _gauss_legendre(n - 1, dtype)
    return np.concatenate((np.array([-1], dtype=dtype), inner, np.array([1], dtype=dtype)))


def lagrange_values(nodes, x):
    """A[i, j] = l_j(x_i), l_j the Lagrange basis polynomial on `nodes` (Eq. lagr:poly)."""
    nodes = np.asarray(nodes)
    x = np.asarray(x)
    A = np.ones((len(x), len(nodes)), dtype=nodes.dtype)
    for j in range(len(nodes)):
        for k in range(len(nodes)):
            if k != j:
                A[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return A


def lagrange_derivatives(nodes, x):
    """D[i, j] = l_j'(x_i) by the product-rule identity of the footnote to Eq. Mmat:
    l_j'(x) = l_j(x) * sum_{k != j} 1/(x - x_k). Valid only where x is not a node,
    which holds for solution points against flux points (the zeros of consecutive
    Legendre polynomials interlace strictly)."""
    nodes = np.asarray(nodes)
    x = np.asarray(x)
    for xi in x:
        if np.min(np.abs(xi - nodes)) < 1e-14:
            raise ValueError("evaluation point coincides with a node")
    vals = lagrange_values(nodes, x)
    D = np.zeros_like(vals)
    for j in range(len(nodes)):
        s = np.zeros(len(x), dtype=nodes.dtype)
        for k in range(len(nodes)):
            if k != j:
                s += 1.0 / (x - nodes[k])
        D[:, j] = vals[:, j] * s
    return D


class Operators:
    """The 1D SD operators for n = p + 1 solution points (Sec. 2.1).

    L  (n+1, n): extrapolation solution -> flux points,  L_ij = l_j(xi_{i-1/2})  (Eq. Lmat)
    M  (n, n+1): derivative flux points -> solution pts, M_ij = l'_{j-1/2}(xi_i) (Eq. Mmat)
    cL, cR (n+1,): unit vectors selecting the interface flux points     (Eq. cl:cr)
    xs, ws: solution points and Gauss weights; xf: flux points.
    """

    def __init__(self, n, dtype=np.float64):
        if n < 1:
            raise ValueError("n must be >= 1")
        self.n = n
        self.p = n - 1
        self.dtype = np.dtype(dtype)
        self.xs, self.ws = solution_points(n, dtype)
        self.xf = flux_points(n, dtype)
        self.L = lagrange_values(self.xs, self.xf)
        self.M = lagrange_derivatives(self.xf, self.xs)
        self.cL = np.zeros(n + 1, dtype=dtype)
        self.cL[0] = 1
        self.cR = np.zeros(n + 1, dtype=dtype)
        self.cR[n] = 1

    @property
    def alpha(self):
        """c_L^T L M c_R: the left-face value of the derivative of the right
        correction (Sec. 2.2: first row of L times last column of M)."""
        return float(self.cL @ self.L @ self.M @ self.cR)

    @property
    def beta(self):
        """c_R^T L M c_L (Sec. 2.2: last row of L times first column of M)."""
        return float(self.cR @ self.L @ self.M @ self.cL)


_CACHE = {}


def operators(n, dtype=np.float64):
    """Cached operators; dtype float64 (default) or np.longdouble (x86 80-bit extended
    precision, used as a higher-precision evaluation of the same definition)."""
    key = (n, np.dtype(dtype).name)
    if key not in _CACHE:
        _CACHE[key] = Operators(n, dtype)
    return _CACHE[key]
