"""Pin of the 1D BR1 and compact oracle residuals against the convergence-rate table the
paper prints (Sec. 4.1, Table tab:convergence; fixture tests/golden/convergence_rates.json).

The semi-discrete system is linear, so it is integrated exactly in time
(u(T) = exp(T A) u0 with A assembled column by column from the oracle residual); the
rate is the one between the two finest levels (1200 and 2400 DOF), which is what the
table's values correspond to. The paper does not state its time step; exact time
integration leaves the spatial error alone, so the values agree to a few hundredths
(three of them to the printed digit) and the even-order degradation of BR1 is
reproduced."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from oracle.diagnostics import l2_error
from oracle.grid import Grid
from oracle.physics import Heat
from oracle.residual import residual
from paper_2608_09615_b300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "convergence_rates.json")))


def operator_matrix(g, scheme):
    E, n = g.ne[0], g.n
    cols = []
    for j in range(n):
        U = np.zeros((1, E, n))
        U[0, 0, j] = 1.0
        cols.append(residual(U, g, scheme, Heat(1.0))[0])
    rows, cidx, vals = [], [], []
    for e0 in range(E):          # translation invariance of the periodic grid
        for j in range(n):
            R = np.roll(cols[j], e0, axis=0)
            for e, i in zip(*np.nonzero(R)):
                rows.append(e * n + i)
                cidx.append(e0 * n + j)
                vals.append(R[e, i])
    return sp.csr_matrix((vals, (rows, cidx)), shape=(E * n, E * n))


def gaussian_error(p, E, scheme, T=2e-5, Dti=1.0 / 2400.0):
    g = Grid(1, (E,), (0.0,), (1.0,), p)
    u0 = inputs.gaussian_1d(E, p, Dti)[0]
    (x,) = g.coordinates()
    ua = np.exp(-(x - 0.5) ** 2 / (4 * (Dti + T))) / np.sqrt(4 * np.pi * (Dti + T))
    uT = sla.expm_multiply(operator_matrix(g, scheme) * T, u0.ravel()).reshape(u0.shape)
    return l2_error(uT, ua, g)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("scheme,key", [("compact", "compact"), ("br1", "standard")])
def test_convergence_rates_match_paper(p, scheme, key):
    Es = GOLD["elements"][str(p)]
    e3 = gaussian_error(p, Es[2], scheme)
    e4 = gaussian_error(p, Es[3], scheme)
    rate = np.log(e3 / e4) / np.log(2.0)
    assert rate == pytest.approx(GOLD["rates"][key][str(p)], abs=0.08)
    nominal = GOLD["rates"]["nominal"][str(p)]
    if scheme == "br1" and p % 2 == 1:
        assert rate < nominal - 0.9          # BR1 loses one order at odd p (even order)
    else:
        assert rate > nominal - 0.1
