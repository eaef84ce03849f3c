"""What the learned closure gains over the plain method (the plain SD solver is both its
fallback and the reference its error is measured against).

A small version of the closure experiment runs end to end on the GPU:
* training data: filtered fine runs (24^3 p=4 -> 6^3 p=3, 4^3 fine elements per coarse
  element) at Re 1600 and 5000, t in [0, 10], sampled every 0.25;
* training: 2000 full-batch Adam steps of the 64-128-128-15 BF16 network;
* evaluation: the coarse 6^3 p=3 run with and without the closure at Re 3000 (not trained
  on) and at Re 1600.

The error is the relative L2 distance, over time, between the coarse run's kinetic-energy
dissipation rate and that of the filtered fine run at the same Re. The test asserts that
training converges, that the closure run stays finite, and that the closure lowers the
error at the held-out Re by at least 1.5% (measured on B300: Re 3000 0.354 -> 0.342, a 3.4%
gain; Re 1600 0.325 -> 0.315). The full-size experiment (64^3 p4 -> 16^3 p3) is
`python -m paper_2608_09615_b300.closure --holdout 3000`."""
import math

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2608_09615_b300 import closure as C  # noqa: E402

FINE, COARSE, T_END, EVERY = 24, 6, 10.0, 0.25


@pytest.fixture(scope="module")
def trained():
    X, T, curves = C.training_data(FINE, COARSE, [1600.0, 5000.0], T_END, EVERY)
    net, stats, losses = C.train(X, T, steps=2000, log_every=500)
    return net, stats, losses, curves, int(X.shape[0])


def test_training_converges(trained):
    _, _, losses, _, n = trained
    assert n == 2 * (round(T_END / EVERY) + 1) * COARSE ** 3
    first, last = losses[0][1], losses[-1][1]
    print("closure training: %d samples, MSE (standardised) %.3f -> %.3f" % (n, first, last))
    assert math.isfinite(last) and last < 0.25 * first


def test_closure_lowers_dissipation_error_at_held_out_re(trained):
    net, stats, _, curves, _ = trained
    _, _, c3000 = C.training_data(FINE, COARSE, [3000.0], T_END, EVERY)
    res = {3000.0: C.evaluate(net, stats, COARSE, 3000.0, T_END, EVERY, c3000[3000.0]),
           1600.0: C.evaluate(net, stats, COARSE, 1600.0, T_END, EVERY, curves[1600.0])}
    for re, r in res.items():
        print("Re %g: dissipation-rate error plain %.4f, closure %.4f (gain %.2f%%)"
              % (re, r["plain"], r["closure"], 100.0 * (1.0 - r["closure"] / r["plain"])))
        assert math.isfinite(r["plain"]) and math.isfinite(r["closure"])
    assert res[3000.0]["closure"] < (1.0 - 0.015) * res[3000.0]["plain"]
