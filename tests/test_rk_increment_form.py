"""The increment forms of the Runge-Kutta schemes that FP32 contexts use (Sec. 4.4 time
integration; RK4 and LSRK(5,4) as well), checked in FP64 against the oracle's steps.

FP32 contexts hold, within a step, only the increments d_j = u_j - U of the stage states
over the step-start state U, and update U once per step. That is the same scheme only if
the Shu-Osher weights of every stage sum to one (then u_j = sum_k a_jk u_k + ... becomes a
recurrence on the d's). The recurrence the kernels evaluate, restated here in FP64:
  d1 = b10 K0;  d2 = a21 d1 + b21 K1;  d3 = a32 d2 + b32 K2;
  e  = a54 (a43 d3 + b43 K3) + (a52 d2 + a53 d3 + b53 K3)   (stage 3 keeps only e)
  U <- U + (e + b54 K4),  with K_j = dt R(U + d_j) and b10 = a10.
A mistake in the weights' bookkeeping (a dropped a_j0 term, a swapped register) makes the
step differ from the oracle's by O(dt), far above the 1e-14 asserted below."""
import numpy as np

from oracle.timestep import LSRK_A, LSRK_B, SSP54, lsrk54_step, rk4_step, ssprk54_step


def _increment_step(R, U, dt, c=SSP54):
    K0 = dt * R(U)
    d1 = c["a10"] * K0
    K1 = dt * R(U + d1)
    d2 = c["a21"] * d1 + c["b21"] * K1
    K2 = dt * R(U + d2)
    d3 = c["a32"] * d2 + c["b32"] * K2
    K3 = dt * R(U + d3)
    d4 = c["a43"] * d3 + c["b43"] * K3
    e = c["a54"] * d4 + (c["a52"] * d2 + c["a53"] * d3 + c["b53"] * K3)
    K4 = dt * R(U + d4)
    return U + (e + c["b54"] * K4)


def test_shu_osher_weights_sum_to_one():
    c = SSP54
    assert abs(c["a20"] + c["a21"] - 1.0) < 1e-14
    assert abs(c["a30"] + c["a32"] - 1.0) < 1e-14
    assert abs(c["a40"] + c["a43"] - 1.0) < 1e-14
    assert abs(c["a52"] + c["a53"] + c["a54"] - 1.0) < 1e-14


def test_increment_form_equals_shu_osher_step():
    rng = np.random.default_rng(3)
    n = 12
    A = rng.standard_normal((n, n)) - 4.0 * np.eye(n)
    R_lin = lambda u: A @ u                                        # noqa: E731
    R_nl = lambda u: A @ u - 0.3 * u ** 3 + np.sin(u)              # noqa: E731
    for R in (R_lin, R_nl):
        U = rng.standard_normal(n)
        for dt in (1e-3, 5e-2):
            ref = ssprk54_step(R, U, dt)
            inc = _increment_step(R, U, dt)
            assert np.abs(inc - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())


def test_a_dropped_weight_is_seen():
    # the planted mistake: stage 2 without its a20 share is a different scheme
    c = dict(SSP54)
    c["a21"] = 1.0
    rng = np.random.default_rng(4)
    A = rng.standard_normal((6, 6)) - 3.0 * np.eye(6)
    R = lambda u: A @ u                                            # noqa: E731
    U = rng.standard_normal(6)
    assert np.abs(_increment_step(R, U, 5e-2, c) - ssprk54_step(R, U, 5e-2)).max() > 1e-6


def _rk4_increment_step(R, U, dt):
    # A accumulates dt/6 K0 + dt/3 K1 + dt/3 K2; the stage inputs are U + dt/2 K0, U + dt/2 K1,
    # U + dt K2; U <- U + (A + dt/6 K3)
    K0 = R(U)
    A = dt / 6.0 * K0
    K1 = R(U + dt / 2.0 * K0)
    A = A + dt / 3.0 * K1
    K2 = R(U + dt / 2.0 * K1)
    A = A + dt / 3.0 * K2
    K3 = R(U + dt * K2)
    return U + (A + dt / 6.0 * K3)


def _lsrk_increment_step(R, U, dt):
    # W <- a W + dt K, D <- D + b W; the stage input is U + D; U <- U + D after the last stage
    W = np.zeros_like(U)
    D = np.zeros_like(U)
    for a, b in zip(LSRK_A, LSRK_B):
        W = a * W + dt * R(U + D)
        D = D + b * W
    return U + D


def test_rk4_and_lsrk_increment_forms_equal_the_oracle():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((10, 10)) - 4.0 * np.eye(10)
    R = lambda u: A @ u - 0.2 * u ** 3                             # noqa: E731
    U = rng.standard_normal(10)
    for dt in (1e-3, 5e-2):
        for inc, ref in ((_rk4_increment_step, rk4_step), (_lsrk_increment_step, lsrk54_step)):
            a, b = inc(R, U, dt), ref(R, U, dt)
            assert np.abs(a - b).max() <= 1e-14 * max(1.0, np.abs(b).max())
