"""The SD semi-discrete residual du/dt on a periodic Cartesian grid, with the viscous
terms built by the standard BR1 auxiliary-gradient scheme (paper Sec. 2.1) or by the
compact one-sided scheme (Secs. 2.2 and 2.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

This is the literal sequence of steps 1-5 of Sec. 2.3 (its 2D statement applied
direction by direction, which the paper says carries over to 3D), with every
intermediate of the paper held as an explicit full array:
  u^{Fd}, u^{Fd,C}, u^{Fd,L}, u^{Fd,R}, H^{Fd,*} = u^{Fd,*} S_{dm}, v^S, the one-sided
  v^{S,dL}, v^{S,dR} obtained by differentiating the one-sided H arrays, the interior
  flux-point gradient v^{Fd} (with zero end columns), the interface averages, v^{Fd,C},
  G^{Fd} and the divergence.
No closed form of the compact correction is used here; the CUDA path uses one.

Pinned by tests/test_oracle_residual.py (polynomial exactness, conservation, stencil
3 vs 5 per axis, separability, free-stream preservation, symmetries), by
tests/test_oracle_bloch.py (the eigenanalysis operator of Sec. 3) and by
tests/test_oracle_convergence.py (the rate table of Sec. 4.1).
"""
import numpy as np

from .grid import Grid


def _ix(ndim, axis, idx):
    s = [slice(None)] * ndim
    s[axis] = idx
    return tuple(s)


def along(A, X, axis):
    """Apply matrix A (out x in) along `axis` of X (Eqs. int:2d and the derivative
    rules that follow: operators act direction by direction)."""
    Y = np.tensordot(A, X, axes=([1], [axis]))
    return np.moveaxis(Y, 0, axis)


def residual(U, grid: Grid, scheme, phys, return_parts=False, tau=None, eta_ip=0.0, viscous="a"):
    """du/dt at the solution points.

    U: array of shape grid.shape(phys.nvar), any float/complex dtype (promoted to
       float64 / complex128).
    scheme: "br1" (Sec. 2.1) or "compact" (Secs. 2.2, 2.3).
    tau: optional per-element extra flux (nvar, E..., dim) of a learned closure (not part
       of the paper's method; see oracle/closure.py): added to F at the element's interior
       flux points, with the average of the two elements' values at each interface.
    eta_ip: interior-penalty parameter (Sec. 3, the Q_IP term): the interface average of
       the d-component of the gradient on a face normal to d gains tau_IP (u_R - u_L),
       tau_IP = eta_ip (p+1)^2 / h_d (the element size; the paper's 1/h = |S| / J with the
       integrated surface and Jacobian gives 1/h_d on Cartesian grids).
    viscous: the interface viscous flux of Sec. 2.1 step 4: "a" = G(u_hat, v_hat) with the
       averaged state and gradient; "b" = (G(u_L, v_L) + G(u_R, v_R)) / 2, each side's trace
       and own interface gradient (the interior penalty term, when on, is added to both
       sides' normal gradients).
    """
    if scheme not in ("br1", "compact"):
        raise ValueError(scheme)
    if viscous not in ("a", "b"):
        raise ValueError(viscous)
    U = np.asarray(U)
    if np.iscomplexobj(U):
        U = U.astype(np.complex128)
    else:
        U = U.astype(grid.dtype)
    if U.shape != grid.shape(phys.nvar):
        raise ValueError("U has shape %s, expected %s" % (U.shape, grid.shape(phys.nvar)))
    ops = grid.ops
    L, M = ops.L, ops.M
    n, dim, nd = grid.n, grid.dim, U.ndim
    S, Jinv = grid.S, grid.Jinv

    # Step 1 (Eq. int:2d): discontinuous solution at the flux points of each family.
    uF = [along(L, U, grid.pt_axis(d)) for d in range(dim)]

    # Step 2 (Eqs. c:sol:2d:xi, c:sol:2d:eta and the 1D Eq. c:flux): common solution
    # hat u = average of the two traces, continuous array u^{Fd,C} and the one-sided
    # arrays u^{Fd,L} (corrected only at the left interface) and u^{Fd,R}.
    uFC, uFL, uFR, uhatL, uhatR, traceL, traceR = [], [], [], [], [], [], []
    for d in range(dim):
        ea, pa = grid.elem_axis(d), grid.pt_axis(d)
        tl = uF[d][_ix(nd, pa, 0)]          # u_e(-1)
        tr = uF[d][_ix(nd, pa, n)]          # u_e(+1)
        hl = 0.5 * (np.roll(tr, 1, axis=ea) + tl)     # (u_{e-}(1) + u_e(-1)) / 2
        hr = 0.5 * (tr + np.roll(tl, -1, axis=ea))    # (u_e(1) + u_{e+}(-1)) / 2
        C = uF[d].copy()
        C[_ix(nd, pa, 0)] += hl - tl
        C[_ix(nd, pa, n)] += hr - tr
        Lf = C.copy()
        Lf[_ix(nd, pa, n)] -= hr - tr
        Rf = C.copy()
        Rf[_ix(nd, pa, 0)] -= hl - tl
        uFC.append(C)
        uFL.append(Lf)
        uFR.append(Rf)
        uhatL.append(hl)
        uhatR.append(hr)
        traceL.append(tl)
        traceR.append(tr)

    def gradient_at_solution_points(family):
        """v_m^S = J^-1 sum_d M_d (u^{Fd,*} S_{dm}) (Eq. w:e and its multi-D form);
        family[d] is the flux-point solution array used along direction d."""
        out = []
        for m in range(dim):
            acc = 0.0
            for d in range(dim):
                if S[d, m] != 0.0:
                    acc = acc + along(M, family[d] * S[d, m], grid.pt_axis(d))
            out.append(Jinv * acc)
        return out

    # Step 3 (Eq. w:e): gradient at the solution points from the continuous fluxes.
    vS = gradient_at_solution_points(uFC)

    # Interior flux points (Eq. aux:v:std:2d): v^{Fd} = L_d v^S with zero end columns.
    vF = []
    for d in range(dim):
        pa = grid.pt_axis(d)
        row = []
        for m in range(dim):
            a = along(L, vS[m], pa)
            a[_ix(nd, pa, 0)] = 0.0
            a[_ix(nd, pa, n)] = 0.0
            row.append(a)
        vF.append(row)

    # Interface values of the gradient, own side of each face.
    faceL, faceR = [], []
    for d in range(dim):
        pa = grid.pt_axis(d)
        if scheme == "compact":
            # Eqs. aux:v:cmp:l - aux:v:cmp:t: the direction-d fluxes are replaced by the
            # one-sided ones, the transverse ones stay continuous; Eqs. aux:cmp:lr:2d,
            # aux:cmp:bt:2d: each is extrapolated to its own interface only.
            famL = [uFL[d] if dd == d else uFC[dd] for dd in range(dim)]
            famR = [uFR[d] if dd == d else uFC[dd] for dd in range(dim)]
            vSL = gradient_at_solution_points(famL)
            vSR = gradient_at_solution_points(famR)
        else:
            # Sec. 2.1 Eq. v:e: BR1 extrapolates the single v^S to both interfaces.
            vSL = vS
            vSR = vS
        faceL.append([along(ops.cL[None, :] @ L, vSL[m], pa)[_ix(nd, pa, 0)] for m in range(dim)])
        faceR.append([along(ops.cR[None, :] @ L, vSR[m], pa)[_ix(nd, pa, 0)] for m in range(dim)])

    # Step 4 (Eq. c:aux:v:2d with the averages of Eq. aux:v:int / cmp:int:avg):
    # continuous auxiliary variable at the flux points of each family.
    vFC = []
    vhatL_all, vhatR_all = [], []
    # option (b): the two sides' own interface gradients (with the penalty term) at the
    # left interface (sideL_*: element e-1, sideR_*: element e) and at the right one
    sideL_l, sideR_l, sideL_r, sideR_r = [], [], [], []
    for d in range(dim):
        ea, pa = grid.elem_axis(d), grid.pt_axis(d)
        row, vl_row, vr_row = [], [], []
        sl_l, sr_l, sl_r, sr_r = [], [], [], []
        for m in range(dim):
            vl = 0.5 * (np.roll(faceR[d][m], 1, axis=ea) + faceL[d][m])
            vr = 0.5 * (faceR[d][m] + np.roll(faceL[d][m], -1, axis=ea))
            pen_l = pen_r = 0.0
            if eta_ip and m == d:
                tip = eta_ip * (grid.n ** 2) / grid.h[d]
                pen_l = tip * (traceL[d] - np.roll(traceR[d], 1, axis=ea))
                pen_r = tip * (np.roll(traceL[d], -1, axis=ea) - traceR[d])
                vl = vl + pen_l
                vr = vr + pen_r
            sl_l.append(np.roll(faceR[d][m], 1, axis=ea) + pen_l)
            sr_l.append(faceL[d][m] + pen_l)
            sl_r.append(faceR[d][m] + pen_r)
            sr_r.append(np.roll(faceL[d][m], -1, axis=ea) + pen_r)
            a = vF[d][m].copy()
            a[_ix(nd, pa, 0)] += vl
            a[_ix(nd, pa, n)] += vr
            row.append(a)
            vl_row.append(vl)
            vr_row.append(vr)
        vFC.append(row)
        vhatL_all.append(vl_row)
        vhatR_all.append(vr_row)
        sideL_l.append(sl_l)
        sideR_l.append(sr_l)
        sideL_r.append(sl_r)
        sideR_r.append(sr_r)

    # Fluxes at all flux points (Eq. above c:aux:v:2d's use: G^{Fd,C} = [S . F]^{Fd}).
    # Interior flux points use the physical flux; interface points use the common
    # flux of the physics (for NS: Riemann solver minus the centred viscous flux).
    # nonlinear diffusivity evaluated at the solution points and extrapolated (PME
    # variant of Sec. 4.3): a^{Fd} = L_d a^S, two-valued at interfaces like any trace
    aF = None
    if getattr(phys, "coef_at_solution_points", False):
        aS = phys.coef(U)
        aF = [along(L, aS, grid.pt_axis(d)) for d in range(dim)]

    G = []
    for d in range(dim):
        ea, pa = grid.elem_axis(d), grid.pt_axis(d)
        Gd = 0.0
        for m in range(dim):
            if S[d, m] == 0.0:
                continue
            if aF is not None:
                Fm = -aF[d] * vFC[d][m]
            else:
                Fm = phys.flux(uFC[d], vFC[d], m)
            # left interface of each element: left state = neighbour's right trace
            vl = [vhatL_all[d][k] for k in range(dim)]
            vr = [vhatR_all[d][k] for k in range(dim)]
            if dim < 3 and phys.nvar == 5:
                raise ValueError("Navier-Stokes needs dim = 3")
            if aF is not None:
                # the two sides' extrapolated diffusivities at each interface
                atl = aF[d][_ix(nd, pa, 0)]                   # a_e(-1)
                atr = aF[d][_ix(nd, pa, n)]                   # a_e(+1)
                aln, arn = np.roll(atr, 1, axis=ea), np.roll(atl, -1, axis=ea)
                if viscous == "a":
                    FL = -0.5 * (aln + atl) * vl[m]
                    FR = -0.5 * (atr + arn) * vr[m]
                else:
                    FL = -0.5 * (aln * sideL_l[d][m] + atl * sideR_l[d][m])
                    FR = -0.5 * (atr * sideL_r[d][m] + arn * sideR_r[d][m])
            elif viscous == "a":
                FL = phys.interface_flux(np.roll(traceR[d], 1, axis=ea), traceL[d],
                                         uhatL[d], vl, m)
                FR = phys.interface_flux(traceR[d], np.roll(traceL[d], -1, axis=ea),
                                         uhatR[d], vr, m)
            else:
                FL = phys.interface_flux_b(np.roll(traceR[d], 1, axis=ea), traceL[d],
                                           sideL_l[d], sideR_l[d], m)
                FR = phys.interface_flux_b(traceR[d], np.roll(traceL[d], -1, axis=ea),
                                           sideL_r[d], sideR_r[d], m)
            Fm[_ix(nd, pa, 0)] = FL
            Fm[_ix(nd, pa, n)] = FR
            if tau is not None:
                t = tau[..., m]
                Fm = Fm + t.reshape(t.shape + (1,) * dim)
                tl = 0.5 * (np.roll(t, 1, axis=ea) + t) - t
                tr = 0.5 * (t + np.roll(t, -1, axis=ea)) - t
                Fm[_ix(nd, pa, 0)] += tl.reshape(tl.shape + (1,) * (dim - 1))
                Fm[_ix(nd, pa, n)] += tr.reshape(tr.shape + (1,) * (dim - 1))
            Gd = Gd + S[d, m] * Fm
        G.append(Gd)

    # Step 5: dq/dt = -sum_d M_d G^{Fd}; u = J^-1 q.
    dq = 0.0
    for d in range(dim):
        dq = dq - along(M, G[d], grid.pt_axis(d))
    dU = Jinv * dq
    if return_parts:
        return dU, dict(vS=vS, uFC=uFC, faceL=faceL, faceR=faceR, G=G)
    return dU


def gradient(U, grid: Grid, nvar):
    """The auxiliary variable v^S at the solution points (Eq. w:e), identical for the
    BR1 and compact schemes (both use H^{F,C} there). Returns a list over the physical
    direction m of arrays shaped like U."""
    ops = grid.ops
    n, dim, nd = grid.n, grid.dim, U.ndim
    out = []
    uFC = []
    for d in range(dim):
        ea, pa = grid.elem_axis(d), grid.pt_axis(d)
        uF = along(ops.L, U, pa)
        tl = uF[_ix(nd, pa, 0)]
        tr = uF[_ix(nd, pa, n)]
        hl = 0.5 * (np.roll(tr, 1, axis=ea) + tl)
        hr = 0.5 * (tr + np.roll(tl, -1, axis=ea))
        uF[_ix(nd, pa, 0)] += hl - tl
        uF[_ix(nd, pa, n)] += hr - tr
        uFC.append(uF)
    for m in range(dim):
        acc = 0.0
        for d in range(dim):
            if grid.S[d, m] != 0.0:
                acc = acc + along(ops.M, uFC[d] * grid.S[d, m], grid.pt_axis(d))
        out.append(grid.Jinv * acc)
    return out
