"""Physical fluxes for the three model problems (paper Secs. 3, 4.3 and 4.4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions: u has shape (nvar, ...); grad is a list over the physical direction k of
arrays shaped like u, grad[k][v] = d u_v / d x_k (the auxiliary variable v of Eq. ns).
flux(u, grad, m) returns the m-th physical component of F(u, grad u) such that the
equation reads du/dt + div F = 0.

Readings of the paper used here (where it is silent or garbled):
  * Heat: F = -nu grad u (Eq. advection with nu = 1 in Sec. 3; nu free here).
  * PME (Eq. pme): F = -m |u|^(m-1) grad u, the nonlinear factor evaluated from the
    solution at the flux points (Sec. 4.3). |u| keeps the diffusivity non-negative for
    even m where round-off makes u slightly negative; for u >= 0 it is the paper's u^(m-1).
  * NS (Sec. 4.4): energy convective flux (rho E + P) u; viscous energy flux
    u . tau + kappa grad T (heat flows down the temperature gradient); lambda = 0;
    kappa grad T = (mu gamma / Pr) grad e with e = E - |u|^2 / 2 (c_p T = gamma e);
    Sutherland mu = mu0 (T/T0)^(3/2) (T0 + S)/(T + S) with T/T0 = e/e0 and S/T0 given
    (110.4 K / 300 K by default); Roe flux with a Harten entropy fix on the two acoustic
    eigenvalues, delta = harten * (Roe-averaged sound speed).

Pinned by tests/test_oracle_residual.py (free stream; the closed-form responses of a heat
conduction and an entropy wave; Roe's textbook properties: consistency, pure upwinding of
supersonic pairs, exact resolution of a stationary contact), tests/test_oracle_physics_pins.py
(Sutherland's law away from T0: the textbook air ratios and a closed-form heat conduction
with T/T0 in [0.77, 1.43]; the viscous stress with its transpose and lambda = 0: closed-form
viscous residuals of a compressive and a shear velocity field; Harten's fix: the exact Roe
flux of a pure near-sonic acoustic wave), tests/test_oracle_variants.py (options (a) and (b)
of the interface viscous flux) and tests/test_oracle_curvilinear.py (the Riemann flux along a
general normal: the axis-aligned case, rotation equivariance, consistency).
"""
from dataclasses import dataclass

import numpy as np


class Heat:
    """Linear diffusion u_t = nu lap u."""

    nvar = 1
    kind = "heat"

    def __init__(self, nu=1.0):
        self.nu = float(nu)

    def flux(self, u, grad, m):
        return -self.nu * grad[m]

    def interface_flux(self, uL, uR, uhat, vhat, m):
        # Sec. 2.1 step 4, option (a): G(u_hat, v_hat)
        return self.flux(uhat, vhat, m)

    def interface_flux_b(self, uL, uR, vL, vR, m):
        # Sec. 2.1 step 4, option (b): (G(u_L, v_L) + G(u_R, v_R)) / 2
        return 0.5 * (self.flux(uL, vL, m) + self.flux(uR, vR, m))


class PorousMedium:
    """u_t = lap(u^m) = div(m u^(m-1) grad u) (Eq. pme).

    coef: where the nonlinear diffusivity m |u|^(m-1) is evaluated (Sec. 4.3): "flux" at
    the flux points from the extrapolated solution (the paper's results), "solution" at
    the solution points and then extrapolated to the flux points like any other field
    (the variant the paper mentions; the residual handles it, see oracle/residual.py)."""

    nvar = 1
    kind = "pme"

    def __init__(self, m=2.0, coef="flux"):
        if coef not in ("flux", "solution"):
            raise ValueError(coef)
        self.m = float(m)
        self.coef_at_solution_points = coef == "solution"

    def coef(self, u):
        return self.m * np.abs(u) ** (self.m - 1.0)

    def flux(self, u, grad, m):
        return -self.coef(u) * grad[m]

    def interface_flux(self, uL, uR, uhat, vhat, m):
        return self.flux(uhat, vhat, m)

    def interface_flux_b(self, uL, uR, vL, vR, m):
        return 0.5 * (self.flux(uL, vL, m) + self.flux(uR, vR, m))


@dataclass
class NSParams:
    """Compressible Navier-Stokes parameters (Sec. 4.4). mu0 = rho0 u0 L / Re and
    p0 = rho0 (u0/Ma)^2 / gamma; e0 = p0 / ((gamma - 1) rho0) is the reference
    internal energy that stands for T0 in Sutherland's law."""

    gamma: float = 1.4
    Pr: float = 0.71
    Re: float = 1600.0
    Ma: float = 0.1
    rho0: float = 1.0
    u0: float = 1.0
    L: float = 1.0
    sutherland: bool = True
    suth_s: float = 110.4 / 300.0
    riemann: str = "roe"            # "roe" or "rusanov"
    harten: float = 0.1

    @property
    def mu0(self):
        return self.rho0 * self.u0 * self.L / self.Re

    @property
    def p0(self):
        return self.rho0 * (self.u0 / self.Ma) ** 2 / self.gamma

    @property
    def e0(self):
        return self.p0 / ((self.gamma - 1.0) * self.rho0)


class NavierStokes:
    """F = F_c(U) - F_v(U, grad U), U = (rho, rho u, rho v, rho w, rho E) (Sec. 4.4)."""

    nvar = 5
    kind = "ns"

    def __init__(self, prm=None):
        self.prm = prm if prm is not None else NSParams()

    # --- thermodynamics ----------------------------------------------------------
    def primitives(self, U):
        g = self.prm.gamma
        rho = U[0]
        vel = [U[1 + i] / rho for i in range(3)]
        E = U[4] / rho
        ke = 0.5 * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
        e = E - ke
        p = (g - 1.0) * rho * e
        return rho, vel, E, e, p

    def viscosity(self, e):
        prm = self.prm
        if not prm.sutherland:
            return prm.mu0 * np.ones_like(e)
        theta = e / prm.e0
        s = prm.suth_s
        return prm.mu0 * theta ** 1.5 * (1.0 + s) / (theta + s)

    # --- fluxes ----------------------------------------------------------------------
    def convective_flux(self, U, m):
        rho, vel, E, e, p = self.primitives(U)
        F = np.empty_like(U)
        F[0] = U[1 + m]
        for i in range(3):
            F[1 + i] = U[1 + i] * vel[m] + (p if i == m else 0.0)
        F[4] = (U[4] + p) * vel[m]
        return F

    def viscous_flux(self, U, grad, m):
        prm = self.prm
        rho, vel, E, e, p = self.primitives(U)
        # primitive gradients from the conservative ones (Sec. 4.4)
        du = [[(grad[k][1 + i] - vel[i] * grad[k][0]) / rho for i in range(3)]
              for k in range(3)]                       # du[k][i] = d u_i / d x_k
        dE = [(grad[k][4] - E * grad[k][0]) / rho for k in range(3)]
        de = [dE[k] - sum(vel[i] * du[k][i] for i in range(3)) for k in range(3)]
        mu = self.viscosity(e)
        tau_m = [mu * (du[m][i] + du[i][m]) for i in range(3)]   # tau_{m i}, lambda = 0
        Fv = np.empty_like(U)
        Fv[0] = 0.0
        for i in range(3):
            Fv[1 + i] = tau_m[i]
        Fv[4] = sum(vel[i] * tau_m[i] for i in range(3)) + mu * prm.gamma / prm.Pr * de[m]
        return Fv

    def flux(self, U, grad, m):
        return self.convective_flux(U, m) - self.viscous_flux(U, grad, m)

    def entropy_fix(self, lam, c):
        """Harten's entropy fix of an acoustic eigenvalue magnitude |lambda| (Sec. 4.4, reading
        R8): below delta = harten * c it is replaced by (lambda^2 + delta^2) / (2 delta)."""
        delta = self.prm.harten * c
        return np.where(lam < delta, (lam ** 2 + delta ** 2) / (2.0 * delta), lam)

    def riemann(self, UL, UR, m):
        if self.prm.riemann == "roe":
            return self.roe(UL, UR, m)
        if self.prm.riemann == "rusanov":
            return self.rusanov(UL, UR, m)
        raise ValueError(self.prm.riemann)

    def rusanov(self, UL, UR, m):
        g = self.prm.gamma
        rl, vl, El, el, pl = self.primitives(UL)
        rr, vr, Er, er, pr = self.primitives(UR)
        cl = np.sqrt(g * pl / rl)
        cr = np.sqrt(g * pr / rr)
        smax = np.maximum(np.abs(vl[m]) + cl, np.abs(vr[m]) + cr)
        return 0.5 * (self.convective_flux(UL, m) + self.convective_flux(UR, m)) \
            - 0.5 * smax * (UR - UL)

    def roe(self, UL, UR, m):
        """Roe's approximate Riemann flux with Harten's entropy fix (Sec. 4.4)."""
        g = self.prm.gamma
        rl, vl, El, el, pl = self.primitives(UL)
        rr, vr, Er, er, pr = self.primitives(UR)
        Hl = (UL[4] + pl) / rl
        Hr = (UR[4] + pr) / rr
        sl = np.sqrt(rl)
        sr = np.sqrt(rr)
        wsum = sl + sr
        ut = [(sl * vl[i] + sr * vr[i]) / wsum for i in range(3)]
        Ht = (sl * Hl + sr * Hr) / wsum
        rt = sl * sr
        q2 = ut[0] ** 2 + ut[1] ** 2 + ut[2] ** 2
        c2 = (g - 1.0) * (Ht - 0.5 * q2)
        c = np.sqrt(c2)
        qn = ut[m]
        drho = rr - rl
        dp = pr - pl
        dv = [vr[i] - vl[i] for i in range(3)]
        dvn = dv[m]
        lam1 = np.abs(qn - c)
        lam2 = np.abs(qn)
        lam5 = np.abs(qn + c)
        if self.prm.harten > 0.0:
            lam1 = self.entropy_fix(lam1, c)
            lam5 = self.entropy_fix(lam5, c)
        a1 = (dp - rt * c * dvn) / (2.0 * c2)
        a2 = drho - dp / c2
        a5 = (dp + rt * c * dvn) / (2.0 * c2)
        dvt = [dv[i] - (dvn if i == m else 0.0) for i in range(3)]
        diss = np.empty_like(UL)
        diss[0] = lam1 * a1 + lam2 * a2 + lam5 * a5
        for i in range(3):
            en = 1.0 if i == m else 0.0
            diss[1 + i] = (lam1 * a1 * (ut[i] - c * en) + lam2 * a2 * ut[i]
                           + lam5 * a5 * (ut[i] + c * en) + lam2 * rt * dvt[i])
        diss[4] = (lam1 * a1 * (Ht - qn * c) + lam2 * a2 * 0.5 * q2
                   + lam5 * a5 * (Ht + qn * c)
                   + lam2 * rt * sum(ut[i] * dvt[i] for i in range(3)))
        return 0.5 * (self.convective_flux(UL, m) + self.convective_flux(UR, m)) - 0.5 * diss

    # --- numerical flux along a general unit normal (curved faces) ------------------
    def normal_flux(self, U, nvec):
        """n . F_c(U) for the unit normal nvec (list of 3 arrays or numbers)."""
        return sum(nvec[m] * self.convective_flux(U, m) for m in range(3))

    def riemann_normal(self, UL, UR, nvec):
        if self.prm.riemann == "roe":
            return self.roe_normal(UL, UR, nvec)
        if self.prm.riemann == "rusanov":
            g = self.prm.gamma
            rl, vl, El, el, pl = self.primitives(UL)
            rr, vr, Er, er, pr = self.primitives(UR)
            unl = sum(vl[i] * nvec[i] for i in range(3))
            unr = sum(vr[i] * nvec[i] for i in range(3))
            smax = np.maximum(np.abs(unl) + np.sqrt(g * pl / rl), np.abs(unr) + np.sqrt(g * pr / rr))
            return 0.5 * (self.normal_flux(UL, nvec) + self.normal_flux(UR, nvec)) - 0.5 * smax * (UR - UL)
        raise ValueError(self.prm.riemann)

    def roe_normal(self, UL, UR, nvec):
        """Roe's flux with Harten's fix along the unit normal nvec: the 1D Roe solver of
        Sec. 4.4 written in the frame of the face, with normal velocity q_n = u . n and
        tangential jumps dv - (dv . n) n."""
        g = self.prm.gamma
        rl, vl, El, el, pl = self.primitives(UL)
        rr, vr, Er, er, pr = self.primitives(UR)
        Hl = (UL[4] + pl) / rl
        Hr = (UR[4] + pr) / rr
        sl = np.sqrt(rl)
        sr = np.sqrt(rr)
        wsum = sl + sr
        ut = [(sl * vl[i] + sr * vr[i]) / wsum for i in range(3)]
        Ht = (sl * Hl + sr * Hr) / wsum
        rt = sl * sr
        q2 = ut[0] ** 2 + ut[1] ** 2 + ut[2] ** 2
        c2 = (g - 1.0) * (Ht - 0.5 * q2)
        c = np.sqrt(c2)
        qn = sum(ut[i] * nvec[i] for i in range(3))
        drho = rr - rl
        dp = pr - pl
        dv = [vr[i] - vl[i] for i in range(3)]
        dvn = sum(dv[i] * nvec[i] for i in range(3))
        lam1 = np.abs(qn - c)
        lam2 = np.abs(qn)
        lam5 = np.abs(qn + c)
        if self.prm.harten > 0.0:
            lam1 = self.entropy_fix(lam1, c)
            lam5 = self.entropy_fix(lam5, c)
        a1 = (dp - rt * c * dvn) / (2.0 * c2)
        a2 = drho - dp / c2
        a5 = (dp + rt * c * dvn) / (2.0 * c2)
        dvt = [dv[i] - dvn * nvec[i] for i in range(3)]
        diss = np.empty_like(UL)
        diss[0] = lam1 * a1 + lam2 * a2 + lam5 * a5
        for i in range(3):
            diss[1 + i] = (lam1 * a1 * (ut[i] - c * nvec[i]) + lam2 * a2 * ut[i]
                           + lam5 * a5 * (ut[i] + c * nvec[i]) + lam2 * rt * dvt[i])
        diss[4] = (lam1 * a1 * (Ht - qn * c) + lam2 * a2 * 0.5 * q2
                   + lam5 * a5 * (Ht + qn * c)
                   + lam2 * rt * sum(ut[i] * dvt[i] for i in range(3)))
        return 0.5 * (self.normal_flux(UL, nvec) + self.normal_flux(UR, nvec)) - 0.5 * diss

    def interface_flux(self, uL, uR, uhat, vhat, m):
        # Sec. 4.4: Roe (or Rusanov) inviscid flux minus the centred viscous flux
        # evaluated on the average solution and the average gradient.
        return self.riemann(uL, uR, m) - self.viscous_flux(uhat, vhat, m)

    def interface_flux_b(self, uL, uR, vL, vR, m):
        # Sec. 2.1 step 4, option (b) for the viscous part: the average of the two
        # sides' viscous fluxes, each from its own trace and own interface gradient
        return self.riemann(uL, uR, m) - 0.5 * (self.viscous_flux(uL, vL, m) + self.viscous_flux(uR, vR, m))


def make_physics(kind, **kw):
    if kind == "heat":
        return Heat(kw.get("nu", 1.0))
    if kind == "pme":
        return PorousMedium(kw.get("m", 2.0))
    if kind == "ns":
        return NavierStokes(kw.get("prm"))
    raise ValueError(kind)
