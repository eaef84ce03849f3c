"""Explicit Runge-Kutta integrators for the semi-discrete system dU/dt = R(U).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* SSPRK(5,4): the five-stage, fourth-order strong-stability-preserving scheme the paper
  uses for the Taylor-Green runs (Sec. 4.4, citing Spiteri & Ruuth 2002). The paper
  does not print the coefficients; the Shu-Osher form below is the published one.
* RK4: the classical four-stage scheme (used for the 1D sin(x) diffusion case).
* LSRK(5,4): the five-stage fourth-order two-register scheme of Carpenter & Kennedy
  (NASA TM-109112, 1994): dU <- a_k dU + dt R(U); U <- U + b_k dU.

Pinned by tests/test_oracle_timestep.py: the stability polynomial of each scheme
equals exp(z) through z^4, and the observed order on a nonlinear ODE is 4.
"""
import numpy as np

SSP54 = dict(
    a10=0.391752226571890,
    a20=0.444370493651235, a21=0.555629506348765, b21=0.368410593050371,
    a30=0.620101851488403, a32=0.379898148511597, b32=0.251891774271694,
    a40=0.178079954393132, a43=0.821920045606868, b43=0.544974750228521,
    a52=0.517231671970585, a53=0.096059710526147, b53=0.063692468666290,
    a54=0.386708617503269, b54=0.226007483236906,
)

LSRK_A = (0.0,
          -567301805773.0 / 1357537059087.0,
          -2404267990393.0 / 2016746695238.0,
          -3550918686646.0 / 2091501179385.0,
          -1275806237668.0 / 842570457699.0)
LSRK_B = (1432997174477.0 / 9575080441755.0,
          5161836677717.0 / 13612068292357.0,
          1720146321549.0 / 2090206949498.0,
          3134564353537.0 / 4481467310338.0,
          2277821191437.0 / 14882151754819.0)


def rk4_step(R, U, dt):
    k1 = R(U)
    k2 = R(U + 0.5 * dt * k1)
    k3 = R(U + 0.5 * dt * k2)
    k4 = R(U + dt * k3)
    return U + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def ssprk54_step(R, U, dt):
    c = SSP54
    u0 = U
    u1 = u0 + c["a10"] * dt * R(u0)
    u2 = c["a20"] * u0 + c["a21"] * u1 + c["b21"] * dt * R(u1)
    u3 = c["a30"] * u0 + c["a32"] * u2 + c["b32"] * dt * R(u2)
    L3 = R(u3)
    u4 = c["a40"] * u0 + c["a43"] * u3 + c["b43"] * dt * L3
    L4 = R(u4)
    return c["a52"] * u2 + c["a53"] * u3 + c["b53"] * dt * L3 + c["a54"] * u4 + c["b54"] * dt * L4


def lsrk54_step(R, U, dt):
    dU = np.zeros_like(U)
    U = U.copy()
    for a, b in zip(LSRK_A, LSRK_B):
        dU = a * dU + dt * R(U)
        U = U + b * dU
    return U


STEPPERS = {"rk4": rk4_step, "ssprk54": ssprk54_step, "lsrk54": lsrk54_step}


def integrate(R, U, dt, nsteps, scheme="rk4"):
    step = STEPPERS[scheme]
    for _ in range(nsteps):
        U = step(R, U, dt)
    return U
