"""The temporal-eigenanalysis matrices of Sec. 3, written from the paper's equations (not
from the oracle): the two computations share only the 1D operator matrices.

  H(theta)   = L + 1/2 cL cR^T L e^{-i theta} - 1/2 cL cL^T L
                 + 1/2 cR cL^T L e^{+i theta} - 1/2 cR cR^T L
  W^L        = J^-1 M [H - 1/2 cR cL^T L e^{+i theta} + 1/2 cR cR^T L]
  W^R        = J^-1 M [H - 1/2 cL cR^T L e^{-i theta} + 1/2 cL cL^T L]
  Q          = (I - cL cL^T - cR cR^T) L J^-1 M H
               + 1/2 cL cR^T L W^R e^{-i theta} + 1/2 cL cL^T L W^L
               + 1/2 cR cL^T L W^L e^{+i theta} + 1/2 cR cR^T L W^R
  Q_IP       = tau (cL cL^T - cL cR^T e^{-i theta}) L + tau (cR cL^T e^{i theta} - cR cR^T) L
  v^{F,C}    = (Q + Q_IP) u^S

For BR1 the same algebra holds with W^L = W^R = J^-1 M H (both faces extrapolate the one
v^S, Sec. 2.1). For u_t = u_xx the flux is G = -v, so du/dt = J^-1 M (Q + Q_IP) u."""
import numpy as np

from oracle.operators import operators


def bloch_Q_ip(n, theta, tau):
    """Q_IP of Sec. 3: tau (cL cL^T - cL cR^T e^{-i theta}) L + tau (cR cL^T e^{i theta} - cR cR^T) L."""
    o = operators(n)
    L, cL, cR = o.L, o.cL[:, None], o.cR[:, None]
    ep, em = np.exp(1j * theta), np.exp(-1j * theta)
    return tau * (cL @ cL.T - cL @ cR.T * em) @ L + tau * (cR @ cL.T * ep - cR @ cR.T) @ L


def bloch_Q(n, theta, scheme, Jinv=1.0):
    o = operators(n)
    L, M, cL, cR = o.L, o.M, o.cL[:, None], o.cR[:, None]
    ep, em = np.exp(1j * theta), np.exp(-1j * theta)
    H = L + 0.5 * cL @ cR.T @ L * em - 0.5 * cL @ cL.T @ L + 0.5 * cR @ cL.T @ L * ep \
        - 0.5 * cR @ cR.T @ L
    if scheme == "compact":
        WL = Jinv * M @ (H - 0.5 * cR @ cL.T @ L * ep + 0.5 * cR @ cR.T @ L)
        WR = Jinv * M @ (H - 0.5 * cL @ cR.T @ L * em + 0.5 * cL @ cL.T @ L)
    else:
        WL = WR = Jinv * M @ H
    base = L @ (Jinv * M @ H)
    Q = base - cL @ cL.T @ base - cR @ cR.T @ base \
        + 0.5 * cL @ cR.T @ L @ WR * em + 0.5 * cL @ cL.T @ L @ WL \
        + 0.5 * cR @ cL.T @ L @ WL * ep + 0.5 * cR @ cR.T @ L @ WR
    return Q


def bloch_B(n, theta, scheme, h=1.0, eta_ip=0.0):
    """du/dt = B u for the Bloch mode of u_t = u_xx on elements of size h."""
    Jinv = 2.0 / h
    Q = bloch_Q(n, theta, scheme, Jinv)
    if eta_ip:
        Q = Q + bloch_Q_ip(n, theta, eta_ip * n * n / h)
    return Jinv * operators(n).M @ Q
