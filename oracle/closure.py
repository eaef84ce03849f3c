"""Reference definitions of the learned per-element sub-grid closure data: the box filter
(L2 projection of a fine SD field onto a coarser SD space), the sub-grid flux targets,
the 64 element features, and the injection of a per-element flux into the residual.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no closure (it notes that an explicit sub-grid model is "quite possibly
required" for under-resolved Taylor-Green runs, Sec. 4.4); the definitions below are the
reading this repository takes, written once here and once in the CUDA kernels:

* Filter: coarse element E holds r^3 fine elements (r = ne_fine / ne_coarse per axis).
  The coarse nodal values are the L2 projection onto Q_{p_c}(E):
  u_c(x_a) = (1 / (J_c w_a)) int_E u_f l_a dx, with the coarse Lagrange basis l_a on the
  Gauss points (orthogonal under Gauss quadrature) and the integral evaluated exactly by
  the fine Gauss rule (degree p_f + p_c <= 2 n_f - 1).
* Sub-grid flux target, per coarse element and direction d:
  tau_e[v][d] = mean_E F_d,v(u_f, grad u_f) - mean_E F_d,v(u_c, grad u_c),
  F = F_c - F_v the Navier-Stokes flux at solution points, gradients the SD auxiliary
  variable v^S of each grid, means by Gauss quadrature.
* Injection: the residual treats tau_e as an extra flux constant over element e: it is
  added to G at the interior flux points and the centred average (tau_e- + tau_e)/2 is
  added at each interface (conservative; inside an element its divergence vanishes, so it
  acts through the interface jumps).
* Features (64, scaled by rho0, u0 and the element half-width h/2):
   0-4   element means of (rho - rho0, rho u, rho v, rho w, rho E - rhoE0)
   5-19  linear Legendre moments 3 mean(U_v xi_d)
  20-34  means of the conservative gradients (h/2) dU_v/dx_d
  35-43  means of the velocity gradient (h/2) du_i/dx_k
  44-46  means of (h/2) de/dx_k
  47-51  fraction of each variable's modal energy (mean excluded) in modes of degree p
         (max index), E_top / (E_total + 1e-14)
  52-56  within-element variances of U_v
  57-62  within-element covariances of the velocity components (i <= j)
  63     1000 / Re

Pinned by tests/test_oracle_closure.py: the projection is exact on the coarse space and
conserves the integral; the sub-grid flux vanishes when the fine field has no content the
filter removes; the injection is conservative and acts only through interface jumps;
features of fields with closed-form moments.
"""
import numpy as np

from .grid import Grid
from .operators import operators
from .physics import NavierStokes
from .residual import gradient


# ------------------------------------------------------------------ projection
def projection_matrix(pf, pc, r):
    """P (n_c x r n_f): coarse value a from the fine values of the r fine elements along
    one direction (fine element s, point k)."""
    of, oc = operators(pf + 1), operators(pc + 1)
    nf, nc = pf + 1, pc + 1
    P = np.zeros((nc, r * nf))
    for s in range(r):
        xi = -1.0 + (2 * s + 1 + of.xs) / r           # fine points in coarse coordinates
        lv = np.ones((nc, nf))
        for a in range(nc):
            for b in range(nc):
                if b != a:
                    lv[a] *= (xi - oc.xs[b]) / (oc.xs[a] - oc.xs[b])
        for a in range(nc):
            P[a, s * nf:(s + 1) * nf] = of.ws * lv[a] / (r * oc.ws[a])
    return P


def project(Uf, gf: Grid, gc: Grid):
    """L2 projection of the fine 3D field Uf (nvar, Ezf, Eyf, Exf, nf, nf, nf) onto the
    coarse grid gc (nested: gf.ne = r * gc.ne)."""
    r = gf.ne[0] // gc.ne[0]
    assert all(gf.ne[d] == r * gc.ne[d] for d in range(3))
    P = projection_matrix(gf.p, gc.p, r)
    nv = Uf.shape[0]
    Ec = gc.ne
    nf = gf.n
    # (v, Ezc, sz, Eyc, sy, Exc, sx, k, j, i)
    A = Uf.reshape(nv, Ec[2], r, Ec[1], r, Ec[0], r, nf, nf, nf)
    # group (s, point) per axis: x: (sx, i), y: (sy, j), z: (sz, k)
    A = np.einsum("vZzYyXxkji,axi->vZzYyXkja", A, P.reshape(gc.n, r, nf))
    A = np.einsum("vZzYyXkja,byj->vZzYXkba", A, P.reshape(gc.n, r, nf))
    A = np.einsum("vZzYXkba,czk->vZYXcba", A, P.reshape(gc.n, r, nf))
    return np.ascontiguousarray(A)


# ------------------------------------------------------------------ fluxes and means
def point_fluxes(U, grid, phys: NavierStokes):
    """F_d = F_c,d - F_v,d at every solution point, d = 0..2, with the SD gradient v^S."""
    g = gradient(U, grid, 5)
    return [phys.flux(U, g, d) for d in range(3)]


def element_means(field, grid):
    """Gauss-quadrature mean over each element of a field shaped like one variable
    (...E dims..., n, n, n) -> (...E dims...)."""
    w = grid.ops.ws
    W = np.einsum("k,j,i->kji", w, w, w) / 8.0
    return np.einsum("...kji,kji->...", field, W)


def sgs_target(Uf, gf, gc, phys):
    """tau[v, Ezc, Eyc, Exc, d] (the sub-grid flux of the filtered field)."""
    r = gf.ne[0] // gc.ne[0]
    Uc = project(Uf, gf, gc)
    Ff = point_fluxes(Uf, gf, phys)
    Fc = point_fluxes(Uc, gc, phys)
    Ec = gc.ne
    tau = np.zeros((5,) + tuple(reversed(Ec)) + (3,))
    for d in range(3):
        mf = element_means(Ff[d], gf)          # (v, Ezf, Eyf, Exf)
        mf = mf.reshape(5, Ec[2], r, Ec[1], r, Ec[0], r).mean(axis=(2, 4, 6))
        mc = element_means(Fc[d], gc)
        tau[..., d] = mf - mc
    return tau, Uc


# ------------------------------------------------------------------ features
def features(U, grid, phys: NavierStokes):
    """(E, 64) features of every element of the 3D NS state U on grid (see module doc);
    rows in element order ez, ey, ex (x fastest)."""
    prm = phys.prm
    n, p = grid.n, grid.p
    o = grid.ops
    E = grid.n_elements
    w = o.ws
    W = np.einsum("k,j,i->kji", w, w, w) / 8.0           # sums to 1 over an element
    rho0, u0 = prm.rho0, prm.u0
    rhoE0 = prm.p0 / (prm.gamma - 1.0)
    scale = np.array([rho0, rho0 * u0, rho0 * u0, rho0 * u0, rho0 * u0 * u0])
    V = U.copy()
    V[0] -= rho0
    V[4] -= rhoE0
    V = V / scale[:, None, None, None, None, None, None]
    hh = grid.h[0] / 2.0                                    # cubic elements assumed
    mean = lambda f: np.einsum("...kji,kji->...", f, W).reshape(-1)     # noqa: E731
    F = np.zeros((E, 64))
    for v in range(5):
        F[:, v] = mean(V[v])
    xi = o.xs
    X = [np.broadcast_to(xi[None, None, :], (n, n, n)),
         np.broadcast_to(xi[None, :, None], (n, n, n)),
         np.broadcast_to(xi[:, None, None], (n, n, n))]
    for v in range(5):
        for d in range(3):
            F[:, 5 + 3 * v + d] = 3.0 * mean(V[v] * X[d])
    g = gradient(U, grid, 5)                                # g[k][v] = dU_v/dx_k
    for v in range(5):
        for d in range(3):
            F[:, 20 + 3 * v + d] = hh * mean(g[d][v]) / scale[v]
    rho = U[0]
    vel = [U[1 + i] / rho for i in range(3)]
    du = [[(g[k][1 + i] - vel[i] * g[k][0]) / rho for i in range(3)] for k in range(3)]
    for i in range(3):
        for k in range(3):
            F[:, 35 + 3 * i + k] = hh * mean(du[k][i]) / u0
    Et = U[4] / rho
    for k in range(3):
        dE = (g[k][4] - Et * g[k][0]) / rho
        de = dE - sum(vel[i] * du[k][i] for i in range(3))
        F[:, 44 + k] = hh * mean(de) / (u0 * u0)
    # modal energy fractions (Legendre coefficients by Gauss quadrature)
    Pm = np.stack([np.polynomial.legendre.Legendre.basis(m)(xi) for m in range(n)])   # (m, i)
    norm = 2.0 / (2.0 * np.arange(n) + 1.0)
    T = Pm * w[None, :] / norm[:, None]                    # c_m = sum_i T[m, i] u_i
    hi = np.zeros((n, n, n), dtype=bool)
    hi[p, :, :] = hi[:, p, :] = hi[:, :, p] = True
    nrm = np.einsum("a,b,c->abc", norm, norm, norm)
    for v in range(5):
        c = np.einsum("ck,bj,ai,...kji->...cba", T, T, T, V[v])
        e = c * c * nrm
        tot = e.reshape(e.shape[:-3] + (-1,)).sum(axis=-1) - e[..., 0, 0, 0]
        top = (e * hi).reshape(e.shape[:-3] + (-1,)).sum(axis=-1)
        F[:, 47 + v] = (top / (tot + 1e-14)).reshape(-1)     # content below 1e-14: none
    for v in range(5):
        m1 = mean(V[v])
        F[:, 52 + v] = mean(V[v] * V[v]) - m1 * m1
    k = 0
    for i in range(3):
        for j in range(i, 3):
            ui, uj = vel[i] / u0, vel[j] / u0
            F[:, 57 + k] = mean(ui * uj) - mean(ui) * mean(uj)
            k += 1
    F[:, 63] = 1000.0 / prm.Re
    return F
