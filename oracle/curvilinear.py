"""The SD residual on periodic grids of curved (trilinear) hexahedra: Sec. 2, the
mapping x_e = sum_i M_i(xi) x_{e,i} with K = 8 corner nodes, Eqs. ns:mapped and adj:f
(q = J u, G = S . F, H = S^T u, S = adj(dx/dxi)), and the steps of Sec. 2.3 with the
metric terms evaluated point by point: [S]^{Fd} at the flux points of family d and
[J^-1]^S at the solution points.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Grid input: the corner nodes, nodes[c][k][j][i] with shape (3, nz+1, ny+1, nx+1); element
(ex, ey, ez) has the corners (ex+a, ey+b, ez+c), a, b, c in {0, 1}, and the last node along
each axis is the periodic image of the first (it differs from it by one constant period
vector per axis).

Metric terms: the Jacobian matrix Jm[i][t] = d x_i / d xi_t comes from the derivatives of
the trilinear shape functions; S = adj(Jm) is formed entry by entry as the transposed
cofactor matrix and J = det(Jm) by cofactor expansion. Row d of S at the flux points of
family d is the (unnormalised) area vector of the constant-xi_d surface through them; on
an interface it depends only on the face's own nodes, so both elements see the same
vector (the continuity that Sec. 2.3 relies on).

Interface fluxes on a curved face: the common flux is the area-vector component of the
numerical flux, |S_d| F_riemann(u_L, u_R; n) - S_d . F_v(u_hat, v_hat), n = S_d / |S_d| the
unit normal at that flux point (option (a) of Sec. 2.1; option (b) averages the two
sides' viscous fluxes instead).

Interior penalty (Sec. 3, multi-dimensional case): tau = eta_IP (p+1)^2 / h with
1/h = |A_f| / min(V_{e-}, V_{e+}), A_f the integral of the area vector S_d over the face
(Gauss quadrature over the face's flux points) and V the element volumes (the integral of
J); the penalty tau (u_R - u_L) n is added to the interface average of the gradient. On
a uniform Cartesian grid this is eta_IP (p+1)^2 / h_d, the 1D value.

Pinned by tests/test_oracle_curvilinear.py: equality with the Cartesian oracle on an
undeformed lattice (both schemes, NS / heat / PME, interior penalty, options (a) and (b));
rotation equivariance (a rigidly rotated grid and field give the rotated residual);
free-stream preservation and the discrete metric identities on jittered grids; exactness
on quadratic polynomials for the heat equation on jittered grids (R = nu lap u, a
constant); conservation; the 3-versus-5 element stencil of the compact and BR1 schemes;
the domain volume; the Taylor-Green kinetic energy and enstrophy (ns_diagnostics).
"""
import numpy as np

from .operators import operators
from .residual import _ix, along


def shape_functions(ref, dtype=np.float64):
    """Values N (npts, 8) and derivatives dN (npts, 8, 3) of the trilinear shape functions
    at reference points ref (npts, 3) = (xi, eta, zeta); corner k = a + 2 b + 4 c sits at
    xi = 2a - 1, eta = 2b - 1, zeta = 2c - 1, and N_k = prod_t (1 + s_t r_t) / 2."""
    ref = np.asarray(ref, dtype=dtype)
    npts = ref.shape[0]
    N = np.ones((npts, 8), dtype=dtype)
    dN = np.ones((npts, 8, 3), dtype=dtype)
    one = dtype(1) if isinstance(dtype, type) else np.dtype(dtype).type(1)
    for k, (a, b, c) in enumerate((a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)):
        s = (2 * a - 1, 2 * b - 1, 2 * c - 1)
        f = [(one + s[t] * ref[:, t]) / 2 for t in range(3)]
        N[:, k] = f[0] * f[1] * f[2]
        for t in range(3):
            g = [f[u] for u in range(3)]
            g[t] = np.full(npts, s[t] / 2, dtype=dtype)
            dN[:, k, t] = g[0] * g[1] * g[2]
    return N, dN


def adjugate(A):
    """adj(A)[i][j] = (-1)^(i+j) det(A with row j and column i removed), over the last
    two axes of A (..., 3, 3)."""
    out = np.empty_like(A)
    for i in range(3):
        for j in range(3):
            r = [x for x in range(3) if x != j]
            c = [x for x in range(3) if x != i]
            minor = A[..., r[0], c[0]] * A[..., r[1], c[1]] - A[..., r[0], c[1]] * A[..., r[1], c[0]]
            out[..., i, j] = minor if (i + j) % 2 == 0 else -minor
    return out


def determinant(A, adjA):
    """det(A) by cofactor expansion along the first row: sum_j A[0][j] adj(A)[j][0]."""
    return A[..., 0, 0] * adjA[..., 0, 0] + A[..., 0, 1] * adjA[..., 1, 0] + A[..., 0, 2] * adjA[..., 2, 0]


class CurvGrid:
    """Periodic grid of trilinear hexahedra with its metric terms (3D only)."""

    dim = 3

    def __init__(self, nodes, p, dtype=np.float64):
        nodes = np.asarray(nodes)
        if nodes.ndim != 4 or nodes.shape[0] != 3 or min(nodes.shape[1:]) < 2:
            raise ValueError("nodes must have shape (3, nz+1, ny+1, nx+1)")
        self.dtype = np.dtype(dtype)
        T = self.dtype.type
        self.nodes = nodes.astype(self.dtype)
        self.ne = (nodes.shape[3] - 1, nodes.shape[2] - 1, nodes.shape[1] - 1)
        self.p = int(p)
        self.n = self.p + 1
        self.ops = operators(self.n, dtype)
        n = self.n
        nz, ny, nx = self.ne[2], self.ne[1], self.ne[0]
        # corner coordinates of every element: (ez, ey, ex, 8, 3)
        Xc = np.empty((nz, ny, nx, 8, 3), dtype=self.dtype)
        for k, (a, b, c) in enumerate((a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)):
            for comp in range(3):
                Xc[:, :, :, k, comp] = self.nodes[comp, c:c + nz, b:b + ny, a:a + nx]
        self.corners = Xc
        xs, xf = self.ops.xs, self.ops.xf

        def metric(rz, ry, rx):
            """S and J on the tensor grid of reference coordinates (zeta, eta, xi) given
            per axis; results shaped (ez, ey, ex, len(rz), len(ry), len(rx)) (+ (3, 3))."""
            pts = np.array([(x, y, z) for z in rz for y in ry for x in rx], dtype=self.dtype)
            _, dN = shape_functions(pts, self.dtype.type)
            Jm = np.einsum("zyxkc,pkt->zyxpct", Xc, dN)      # d x_c / d xi_t
            S = adjugate(Jm)
            J = determinant(Jm, S)
            shp = (nz, ny, nx, len(rz), len(ry), len(rx))
            return S.reshape(shp + (3, 3)), J.reshape(shp)

        # S_{d m} at the flux points of family d: Sf[d] has shape (3 [m], ez, ey, ex, pts)
        # with n+1 points along direction d
        self.Sf = []
        for d in range(3):
            r = [xs, xs, xs]                       # (xi, eta, zeta)
            r[d] = xf
            S, _ = metric(r[2], r[1], r[0])
            self.Sf.append(np.moveaxis(S[..., d, :], -1, 0).copy())
        S_sp, J_sp = metric(xs, xs, xs)
        if not np.all(J_sp > 0):
            raise ValueError("a mesh element has a non-positive Jacobian")
        self.J_sp = J_sp
        self.Jinv = T(1) / J_sp
        ws = self.ops.ws
        W = np.einsum("k,j,i->kji", ws, ws, ws)
        self.volume = np.sum(J_sp * W, axis=(3, 4, 5))                  # (ez, ey, ex)
        # interior-penalty scale 1/h of the left face of each element along d
        self.ip_inv_h = []
        for d in range(3):
            pa = 3 + (2 - d)                       # point axis of direction d in Sf[d][m]
            ea = 2 - d                             # element axis of direction d in volume
            face = [self.Sf[d][m][_ix(6, pa, 0)] for m in range(3)]     # (ez, ey, ex, q1, q2)
            A = [np.sum(face[m] * np.einsum("a,b->ab", ws, ws), axis=(3, 4)) for m in range(3)]
            area = np.sqrt(A[0] ** 2 + A[1] ** 2 + A[2] ** 2)
            vmin = np.minimum(self.volume, np.roll(self.volume, 1, axis=ea))
            self.ip_inv_h.append(area / vmin)

    # ----- axis bookkeeping (same layout as the Cartesian grid) -------------------
    def elem_axis(self, d):
        return 1 + (2 - d)

    def pt_axis(self, d):
        return 4 + (2 - d)

    def shape(self, nvar):
        return (nvar,) + tuple(reversed(self.ne)) + (self.n,) * 3

    @property
    def n_elements(self):
        return int(np.prod(self.ne))

    def quadrature_weights(self):
        """J w_i w_j w_k at every solution point."""
        ws = self.ops.ws
        return self.J_sp * np.einsum("k,j,i->kji", ws, ws, ws)

    def coordinates(self):
        """Physical coordinates of the solution points (list over d)."""
        xs = self.ops.xs
        pts = np.array([(x, y, z) for z in xs for y in xs for x in xs], dtype=self.dtype)
        N, _ = shape_functions(pts, self.dtype.type)
        X = np.einsum("zyxkc,pk->czyxp", self.corners, N)
        n = self.n
        return [X[c].reshape(self.ne[2], self.ne[1], self.ne[0], n, n, n) for c in range(3)]


def _common_flux(phys, uL, uR, uhat, vhat, sideL, sideR, Svec, viscous):
    """S . F_hat at interface flux points with area vector Svec (list of 3 arrays)."""
    if phys.kind == "ns":
        area = np.sqrt(Svec[0] ** 2 + Svec[1] ** 2 + Svec[2] ** 2)
        nvec = [Svec[m] / area for m in range(3)]
        G = area * phys.riemann_normal(uL, uR, nvec)
        for m in range(3):
            if viscous == "a":
                G = G - Svec[m] * phys.viscous_flux(uhat, vhat, m)
            else:
                G = G - Svec[m] * 0.5 * (phys.viscous_flux(uL, sideL, m) + phys.viscous_flux(uR, sideR, m))
        return G
    G = 0.0
    for m in range(3):
        if viscous == "a":
            G = G + Svec[m] * phys.flux(uhat, vhat, m)
        else:
            G = G + Svec[m] * 0.5 * (phys.flux(uL, sideL, m) + phys.flux(uR, sideR, m))
    return G


def gradient_parts(U, grid):
    """The steps 1-3 arrays shared by the residual and the diagnostics: u^{Fd}, the
    continuous and one-sided flux-point arrays, the corrections and traces."""
    n, nd = grid.n, U.ndim
    L = grid.ops.L
    uF = [along(L, U, grid.pt_axis(d)) for d in range(3)]
    out = dict(uF=uF, uFC=[], uFL=[], uFR=[], uhatL=[], uhatR=[], traceL=[], traceR=[])
    for d in range(3):
        ea, pa = grid.elem_axis(d), grid.pt_axis(d)
        tl = uF[d][_ix(nd, pa, 0)]
        tr = uF[d][_ix(nd, pa, n)]
        hl = 0.5 * (np.roll(tr, 1, axis=ea) + tl)
        hr = 0.5 * (tr + np.roll(tl, -1, axis=ea))
        C = uF[d].copy()
        C[_ix(nd, pa, 0)] += hl - tl
        C[_ix(nd, pa, n)] += hr - tr
        Lf = C.copy()
        Lf[_ix(nd, pa, n)] -= hr - tr
        Rf = C.copy()
        Rf[_ix(nd, pa, 0)] -= hl - tl
        for key, val in (("uFC", C), ("uFL", Lf), ("uFR", Rf), ("uhatL", hl), ("uhatR", hr),
                         ("traceL", tl), ("traceR", tr)):
            out[key].append(val)
    return out


def gradient_at_solution_points(grid, family):
    """v_m^S = [J^-1]^S (sum_d M_d (u^{Fd,*} [S_dm]^{Fd})) (Sec. 2.3 step 3 in 3D);
    family[d] is the flux-point solution array used along direction d."""
    M = grid.ops.M
    out = []
    for m in range(3):
        acc = 0.0
        for d in range(3):
            acc = acc + along(M, family[d] * grid.Sf[d][m], grid.pt_axis(d))
        out.append(grid.Jinv * acc)
    return out


def gradient(U, grid):
    """v^S (list over the physical direction m), identical for both schemes."""
    U = np.asarray(U).astype(grid.dtype)
    return gradient_at_solution_points(grid, gradient_parts(U, grid)["uFC"])


def residual(U, grid: CurvGrid, scheme, phys, eta_ip=0.0, viscous="a"):
    """du/dt at the solution points of a curvilinear grid (Sec. 2.3 steps 1-5; u = J^-1 q).

    scheme: "br1" or "compact"; viscous: interface viscous flux option "a" or "b"
    (Sec. 2.1 step 4); eta_ip: interior-penalty parameter (Sec. 3)."""
    if scheme not in ("br1", "compact"):
        raise ValueError(scheme)
    if viscous not in ("a", "b"):
        raise ValueError(viscous)
    if getattr(phys, "coef_at_solution_points", False):
        raise ValueError("the solution-point diffusivity variant is Cartesian only")
    U = np.asarray(U).astype(grid.dtype)
    if U.shape != grid.shape(phys.nvar):
        raise ValueError("U has shape %s, expected %s" % (U.shape, grid.shape(phys.nvar)))
    ops = grid.ops
    L, M = ops.L, ops.M
    n, nd = grid.n, U.ndim

    # Steps 1-2: discontinuous and continuous solution at the flux points, the
    # one-sided arrays of the compact scheme, the common solution and the traces.
    P = gradient_parts(U, grid)
    uFC, uFL, uFR = P["uFC"], P["uFL"], P["uFR"]
    uhatL, uhatR, traceL, traceR = P["uhatL"], P["uhatR"], P["traceL"], P["traceR"]

    # Step 3: v^S from the continuous fluxes H^{Fd,C}_m = u^{Fd,C} [S_dm]^{Fd}.
    vS = gradient_at_solution_points(grid, uFC)

    # interior flux points: v^{Fd} = L_d v^S with zero end columns
    vF = []
    for d in range(3):
        pa = grid.pt_axis(d)
        row = []
        for m in range(3):
            a = along(L, vS[m], pa)
            a[_ix(nd, pa, 0)] = 0.0
            a[_ix(nd, pa, n)] = 0.0
            row.append(a)
        vF.append(row)

    # own-side interface gradients: BR1 extrapolates v^S; the compact scheme
    # differentiates the one-sided fluxes along d (transverse fluxes continuous) and
    # extrapolates each to its own interface only
    faceL, faceR = [], []
    for d in range(3):
        pa = grid.pt_axis(d)
        if scheme == "compact":
            vSL = gradient_at_solution_points(grid, [uFL[d] if dd == d else uFC[dd] for dd in range(3)])
            vSR = gradient_at_solution_points(grid, [uFR[d] if dd == d else uFC[dd] for dd in range(3)])
        else:
            vSL = vSR = vS
        faceL.append([along(ops.cL[None, :] @ L, vSL[m], pa)[_ix(nd, pa, 0)] for m in range(3)])
        faceR.append([along(ops.cR[None, :] @ L, vSR[m], pa)[_ix(nd, pa, 0)] for m in range(3)])

    # Step 4: interface averages (+ interior penalty along the unit normal) and the
    # continuous auxiliary variable at the flux points
    vFC, vhatL_all, vhatR_all = [], [], []
    sides = []          # option (b): (left elem side, right elem side) at the left and right faces
    for d in range(3):
        ea, pa = grid.elem_axis(d), grid.pt_axis(d)
        SL = [grid.Sf[d][m][_ix(6, pa - 1, 0)] for m in range(3)]      # own left-face area vector
        SR = [grid.Sf[d][m][_ix(6, pa - 1, n)] for m in range(3)]      # own right-face area vector
        aL = np.sqrt(SL[0] ** 2 + SL[1] ** 2 + SL[2] ** 2)
        aR = np.sqrt(SR[0] ** 2 + SR[1] ** 2 + SR[2] ** 2)
        ih = grid.ip_inv_h[d]                                          # (ez, ey, ex), left faces
        ihL = ih[..., None, None]
        ihR = np.roll(ih, -1, axis=2 - d)[..., None, None]
        jl = traceL[d] - np.roll(traceR[d], 1, axis=ea)                # u_R - u_L at the left face
        jr = np.roll(traceL[d], -1, axis=ea) - traceR[d]               # at the right face
        row, vl_row, vr_row = [], [], []
        s_ll, s_rl, s_lr, s_rr = [], [], [], []
        for m in range(3):
            vl = 0.5 * (np.roll(faceR[d][m], 1, axis=ea) + faceL[d][m])
            vr = 0.5 * (faceR[d][m] + np.roll(faceL[d][m], -1, axis=ea))
            pen_l = pen_r = 0.0
            if eta_ip:
                pen_l = eta_ip * n ** 2 * ihL * jl * (SL[m] / aL)
                pen_r = eta_ip * n ** 2 * ihR * jr * (SR[m] / aR)
                vl = vl + pen_l
                vr = vr + pen_r
            s_ll.append(np.roll(faceR[d][m], 1, axis=ea) + pen_l)
            s_rl.append(faceL[d][m] + pen_l)
            s_lr.append(faceR[d][m] + pen_r)
            s_rr.append(np.roll(faceL[d][m], -1, axis=ea) + pen_r)
            a = vF[d][m].copy()
            a[_ix(nd, pa, 0)] += vl
            a[_ix(nd, pa, n)] += vr
            row.append(a)
            vl_row.append(vl)
            vr_row.append(vr)
        vFC.append(row)
        vhatL_all.append(vl_row)
        vhatR_all.append(vr_row)
        sides.append((s_ll, s_rl, s_lr, s_rr))

    # Step 4 (fluxes): G^{Fd} = [S . F]^{Fd} at the interior flux points, the common
    # area-vector flux at the interfaces
    G = []
    for d in range(3):
        ea, pa = grid.elem_axis(d), grid.pt_axis(d)
        Gd = 0.0
        for m in range(3):
            Gd = Gd + grid.Sf[d][m] * phys.flux(uFC[d], vFC[d], m)
        SL = [grid.Sf[d][m][_ix(6, pa - 1, 0)] for m in range(3)]
        SR = [grid.Sf[d][m][_ix(6, pa - 1, n)] for m in range(3)]
        s_ll, s_rl, s_lr, s_rr = sides[d]
        GL = _common_flux(phys, np.roll(traceR[d], 1, axis=ea), traceL[d], uhatL[d], vhatL_all[d],
                          s_ll, s_rl, SL, viscous)
        GR = _common_flux(phys, traceR[d], np.roll(traceL[d], -1, axis=ea), uhatR[d], vhatR_all[d],
                          s_lr, s_rr, SR, viscous)
        Gd[_ix(nd, pa, 0)] = GL
        Gd[_ix(nd, pa, n)] = GR
        G.append(Gd)

    # Step 5: dq/dt = -sum_d M_d G^{Fd}; u = J^-1 q.
    dq = 0.0
    for d in range(3):
        dq = dq - along(M, G[d], grid.pt_axis(d))
    return grid.Jinv * dq


def ns_diagnostics(U, grid):
    """Kinetic energy (1/2 int u.u and 1/2 int rho u.u), enstrophy, conserved totals and
    volume on a curvilinear grid (Sec. 4.4 volume diagnostics with the weights J w w w)."""
    W = grid.quadrature_weights()
    U = np.asarray(U).astype(grid.dtype)
    rho = U[0]
    vel = [U[1 + i] / rho for i in range(3)]
    g = gradient(U, grid)
    du = [[(g[k][1 + i] - vel[i] * g[k][0]) / rho for i in range(3)] for k in range(3)]
    om = [du[1][2] - du[2][1], du[2][0] - du[0][2], du[0][1] - du[1][0]]
    return dict(
        ke=float(0.5 * np.sum(W * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))),
        ke_rho=float(0.5 * np.sum(W * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))),
        enstrophy=float(np.sum(W * (om[0] ** 2 + om[1] ** 2 + om[2] ** 2))),
        mass=float(np.sum(W * U[0])),
        mom=[float(np.sum(W * U[1 + i])) for i in range(3)],
        energy=float(np.sum(W * U[4])),
        volume=float(np.sum(W)),
        nonfinite=int(not np.all(np.isfinite(U))),
    )
