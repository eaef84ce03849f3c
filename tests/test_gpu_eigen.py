"""Temporal eigenanalysis (Sec. 3) and the Dirac-delta spectra (Sec. 4.2) from the GPU
residual.

* The Bloch operator B(theta) probed from the FP64 GPU residual equals the one built from
  the paper's Sec. 3 matrices (tests/bloch_sec3.py), with and without interior penalty.
* Its eigenvalues are real (centred schemes) and the physical one is -theta^2 for small
  theta.
* Zero-dissipation structure:
  - compact: only the constant mode is undamped;
  - BR1: one more zero eigenvalue at theta = 0 for odd p (the even orders) and one at
    theta = pi for even p;
  - interior penalty damps these spurious modes.
* Dirac spectra: BR1's spurious undamped modes show up as peaks at the wavenumbers the
  eigenanalysis predicts, where the compact scheme's spectrum is far lower. Sec. 4.2 notes
  that the number and location of the peaks coincide with the eigenanalysis."""
import math

import numpy as np
import pytest

from bloch_sec3 import bloch_B

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2608_09615_b300 import eigen  # noqa: E402


@pytest.mark.parametrize("eta", [0.0, 0.02])
@pytest.mark.parametrize("scheme", ["compact", "br1"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_probed_bloch_operator_matches_sec3(p, scheme, eta):
    K = eigen.bloch_kernels(p, scheme, eta)
    reach = 1 if scheme == "compact" else 2
    for m, Km in K.items():
        if abs(m) > reach:
            assert np.abs(Km).max() == 0.0
    thetas = (0.0, 0.3, 1.1, 2.5, math.pi)
    Bp = {t: bloch_B(p + 1, t, scheme, h=1.0, eta_ip=eta) for t in thetas}
    scale = max(np.abs(B).max() for B in Bp.values())     # B(0) vanishes for BR1 at p = 1
    for t in thetas:
        assert np.abs(eigen.bloch_matrix(K, t) - Bp[t]).max() <= 1e-11 * scale


@pytest.mark.parametrize("scheme", ["compact", "br1"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_dissipation_curves_real_and_physical_mode(p, scheme):
    th, lam, imag = eigen.dissipation_curves(p, scheme, nth=61)
    assert imag <= 1e-10 * np.abs(lam).max()
    assert lam.max() <= 1e-10 * np.abs(lam).max()          # no growth
    # the physical eigenvalue is -theta^2 up to a relative error of at least second order in
    # theta (the largest, p = 1 compact, is 0.04 theta^2)
    small = (th > 0) & (th <= 0.2)
    rel = np.abs(lam[small, 0] + th[small] ** 2) / th[small] ** 2
    assert (rel <= 0.1 * th[small] ** 2).all()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_zero_dissipation_modes(p):
    assert eigen.zero_modes(p, "compact") == {"0": 1, "pi": 0}
    zb = eigen.zero_modes(p, "br1")
    assert zb == ({"0": 2, "pi": 0} if p % 2 == 1 else {"0": 1, "pi": 1})
    # interior penalty (eta = 0.02) damps BR1's spurious modes
    assert eigen.zero_modes(p, "br1", eta_ip=0.02) == {"0": 1, "pi": 0}


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dirac_spectrum_peaks_where_eigenanalysis_predicts(p):
    ne = 200
    kb, ab, _ = eigen.dirac_spectrum(p, "br1", ne)
    kc, ac, _ = eigen.dirac_spectrum(p, "compact", ne)
    theta_star = 0.0 if p % 2 == 1 else math.pi
    peaks = [k for k in eigen.predicted_peaks(p, ne, theta_star) if k <= kb[-1]]
    assert peaks
    ratios = []
    for k in peaks:
        half = 0.1 * ne
        ratios.append(eigen.window_max(kb, ab, k, half) / eigen.window_max(kc, ac, k, half))
    print("p=%d BR1 peaks at k=%s, BR1/compact window maxima %s" % (p, peaks, ["%.1f" % r for r in ratios]))
    # measured on B300: p=1 [10.1], p=2 [1.6, 5.5], p=3 [95, 159]; the p = 2 peak at k = 100
    # sits where the physical modes are still large
    assert max(ratios) >= 5.0
    assert min(ratios) >= 1.2


@pytest.mark.parametrize("eta", [0.0, 0.05])
@pytest.mark.parametrize("scheme", ["compact", "br1"])
@pytest.mark.parametrize("p", [1, 3, 4])
def test_combined_mode_of_probed_operator_matches_sec3(p, scheme, eta):
    # Appendix A's combined-mode curves from the Bloch operator probed out of the GPU
    # residual equal those of the operator built from the Sec. 3 matrices
    from oracle.operators import operators
    th, G, om = eigen.combined_curves(p, scheme, eta, t=0.1, nth=37)
    xi = operators(p + 1).xs
    G3, om3 = eigen.combined_mode(lambda a: bloch_B(p + 1, a, scheme, h=1.0, eta_ip=eta), xi, th, 0.1)
    assert np.allclose(G, G3, rtol=1e-9, atol=1e-12)
    assert np.allclose(om.imag, om3.imag, rtol=1e-7, atol=1e-9)
