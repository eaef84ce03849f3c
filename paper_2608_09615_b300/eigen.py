"""Temporal eigenanalysis of the SD discretisation of u_t = u_xx (Sec. 3), taken from the
GPU residual, and the Fourier spectrum of a diffused Dirac delta (Sec. 4.2).

Bloch operator by probing. The residual of the 1D periodic heat problem is linear and
translation invariant, so R_e = sum_m K_m u_{e-m} with n x n blocks K_m (m = -2..2 for BR1,
-1..1 for the compact scheme). One FP64 residual call on a grid of 8n elements with a unit
impulse at point j of element 8j + 4 (far enough apart not to overlap) gives every column
j of every K_m. For the Bloch mode u_e = uhat exp(i theta e), R_e = exp(i theta e) B(theta)
uhat with B(theta) = sum_m K_m exp(-i theta m). With h = 1 the inverse Jacobian is 2: the
physical eigenvalue is -theta^2 for small theta. The paper's B(theta), built from its Sec. 3
matrices, is the same operator (checked by the tests).

Dissipation curves: the eigenvalues lambda(theta) = -i omega(theta) of B for theta in
[0, pi]; for the centred schemes they are real, so Im(omega) = Re(lambda).

Dirac spectrum: one solution point (closest to x = 1/2) set to 1 / (w Dx), w its Gauss
weight on the unit interval, diffused (D = 1) to T = 2e-5 by RK4 on the GPU; the solution
is sampled at N = ne (p + 1) equally spaced points and transformed with Eq. fft. A
zero-dissipation eigenvalue at folded angle theta* leaves the wavenumbers
k = ne (theta* + 2 pi m) / (2 pi) (and their mirror images) undamped; these are the peaks.

Combined-mode analysis (Appendix A). The exact Fourier mode exp(i k x) restricted to one
element of size h = 1 is u0_j = exp(i theta (xi_j + 1) / 2), theta = k h, for the unfolded
theta in [0, (p + 1) pi]. Expanded in the eigenvectors mu_j of B(theta) (u0 = N gamma) it
evolves as u(t) = sum_j gamma_j mu_j exp(lambda_j t), lambda_j = -i omega_j; the amplification
factor of the whole mode is G(theta, t) = u0* u(t) / u0* u0 and its combined frequency
omega(theta, t) = (i / t) log G. (The appendix prints -(i / t) log G; with its own convention
u ~ exp(-i omega t) the sign that returns omega_j when u0 is the eigenvector mu_j is +i / t,
and that is the reading taken.) The dissipation is Im(omega) = log|G| / t (= -theta^2 for the
exact solution of u_t = u_xx). The appendix leaves t open; t = 0.1 (units h = nu = 1) is
the default reported.

    python -m paper_2608_09615_b300.eigen --p 1 2 3 4 --eta 0 0.01 0.02 1.0
    python -m paper_2608_09615_b300.eigen --combined --p 1 2 3 4 --eta 0 0.01 0.02 0.05
"""
import argparse
import json
import math

import numpy as np

from . import SD, Physics

# RK4's stability interval on the negative real axis is about [-2.785, 0]
RK4_REAL_LIMIT = 2.78


def bloch_kernels(p, scheme, eta_ip=0.0, stream=None):
    """Blocks K_m (m = -3..3, each n x n, K[m][i, j] = d R_{e+m, i} / d u_{e, j}) of the
    1D heat residual (nu = 1, h = 1), from one FP64 GPU residual call."""
    import torch
    n = p + 1
    E = 8 * n
    ctx = SD(1, (E,), (0.0,), (float(E),), p, scheme, Physics(kind="heat", nu=1.0, eta_ip=eta_ip), "f64",
             stream=stream)
    U = torch.zeros((1, E, n), dtype=torch.float64, device="cuda")
    for j in range(n):
        U[0, 8 * j + 4, j] = 1.0
    R = ctx.residual(U).cpu().numpy()
    ctx.close()
    return {m: np.stack([R[0, 8 * j + 4 + m, :] for j in range(n)], axis=1) for m in range(-3, 4)}


def bloch_matrix(K, theta):
    return sum(Km * np.exp(-1j * theta * m) for m, Km in K.items())


def dissipation_curves(p, scheme, eta_ip=0.0, nth=181):
    """theta in [0, pi] and the eigenvalues of B(theta), sorted in decreasing real part;
    also the largest imaginary part met (zero for the centred schemes, up to round-off)."""
    K = bloch_kernels(p, scheme, eta_ip)
    th = np.linspace(0.0, math.pi, nth)
    lam = np.array([np.linalg.eigvals(bloch_matrix(K, t)) for t in th])
    imag = float(np.abs(lam.imag).max())
    return th, -np.sort(-lam.real, axis=1), imag


def zero_modes(p, scheme, eta_ip=0.0, tol=1e-9):
    """Number of (numerically) zero eigenvalues of B at theta = 0 and theta = pi: 1 and 0
    when only the constant mode is undamped."""
    K = bloch_kernels(p, scheme, eta_ip)
    lam = {name: np.linalg.eigvals(bloch_matrix(K, t)) for name, t in (("0", 0.0), ("pi", math.pi))}
    scale = max(np.abs(v).max() for v in lam.values())
    return {name: int(np.sum(np.abs(v) < tol * scale)) for name, v in lam.items()}


def spectral_radius(p, scheme, eta_ip=0.0, nth=181):
    _, lam, _ = dissipation_curves(p, scheme, eta_ip, nth)
    return float(np.abs(lam).max())


def combined_mode(B_of_theta, xi, thetas, t, initial=None):
    """Appendix A: G(theta, t) and the combined frequency omega(theta, t) = (i / t) log G of
    the exact Fourier mode, for the Bloch operator B_of_theta(theta) (n x n) of a scheme whose
    solution points are xi (n values in [-1, 1]); thetas unfolded (up to (p + 1) pi).
    initial(theta), if given, replaces the Fourier mode as the initial data."""
    xi = np.asarray(xi, dtype=np.float64)
    G = np.empty(len(thetas), dtype=np.complex128)
    for k, th in enumerate(thetas):
        u0 = np.exp(1j * th * (xi + 1.0) / 2.0) if initial is None else np.asarray(initial(th))
        lam, N = np.linalg.eig(B_of_theta(th))
        gamma = np.linalg.solve(N, u0)
        ut = N @ (gamma * np.exp(lam * t))
        G[k] = np.vdot(u0, ut) / np.vdot(u0, u0)
    omega = 1j * np.log(G) / t
    return G, omega


def combined_curves(p, scheme, eta_ip=0.0, t=0.1, nth=181):
    """Combined-mode curves of the GPU residual's Bloch operator: theta in [0, (p + 1) pi],
    G(theta, t) and omega(theta, t)."""
    K = bloch_kernels(p, scheme, eta_ip)
    xi, _ = _gauss_points(p + 1)
    th = np.linspace(0.0, (p + 1) * math.pi, nth)
    G, om = combined_mode(lambda a: bloch_matrix(K, a), xi, th, t)
    return th, G, om


def _gauss_points(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def _lagrange_matrix(nodes, x):
    """Values of the Lagrange basis on `nodes` at the points x: (len(x), len(nodes))."""
    nodes = np.asarray(nodes, dtype=np.float64)
    A = np.ones((len(x), len(nodes)))
    for j in range(len(nodes)):
        for k in range(len(nodes)):
            if k != j:
                A[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return A


def dirac_spectrum(p, scheme, ne=200, T=2e-5, eta_ip=0.0):
    """|u_hat(k)| (Eq. fft) for k = 0 .. N/2 of the diffused Dirac delta (ne elements on
    [0, 1], D = 1, RK4 on the GPU in FP64)."""
    import torch
    n = p + 1
    h = 1.0 / ne
    rho = spectral_radius(p, scheme, eta_ip) / h ** 2          # B scales as 1/h^2
    steps = max(1, math.ceil(T * rho / (0.9 * RK4_REAL_LIMIT)))
    dt = T / steps
    ctx = SD(1, (ne,), (0.0,), (1.0,), p, scheme, Physics(kind="heat", nu=1.0, eta_ip=eta_ip), "f64")
    xi, w = ctx.points()
    U = torch.zeros((1, ne, n), dtype=torch.float64, device="cuda")
    e, i = ne // 2, 0                                          # first point right of x = 1/2
    U[0, e, i] = 1.0 / (0.5 * w[i] * h)
    for s in range(steps):
        ctx.rk_step(U, s * dt, dt, "rk4")
    u_el = U.cpu().numpy()[0]
    ctx.close()
    N = ne * n
    x = (np.arange(N) + 0.5) / N
    el = np.minimum((x / h).astype(int), ne - 1)
    loc = 2.0 * (x - el * h) / h - 1.0
    u = np.einsum("ji,ji->j", _lagrange_matrix(xi, loc), u_el[el])
    k = np.arange(N // 2 + 1)
    uh = np.array([np.sum(u * np.cos(2 * math.pi * kk * x)) for kk in k]) / (2 * math.pi)
    return k, np.abs(uh), steps


def predicted_peaks(p, ne, theta_star):
    """Unfolded wavenumbers k = ne theta_u / (2 pi), theta_u in (0, (p+1) pi], of the modes
    with folded angle theta_star (0 or pi)."""
    out = []
    m = 0
    while True:
        for tu in ((theta_star + 2 * math.pi * m), (2 * math.pi * (m + 1) - theta_star)):
            if 0 < tu <= (p + 1) * math.pi + 1e-12:
                out.append(ne * tu / (2 * math.pi))
        m += 1
        if 2 * math.pi * m > (p + 1) * math.pi:
            break
    return sorted(set(round(k, 6) for k in out))


def window_max(k, a, centre, half):
    sel = (k >= centre - half) & (k <= centre + half)
    return float(a[sel].max()) if sel.any() else 0.0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--p", type=int, nargs="+", default=[1, 2, 3, 4])
    ap.add_argument("--eta", type=float, nargs="+", default=[0.0])
    ap.add_argument("--nth", type=int, default=91)
    ap.add_argument("--combined", action="store_true", help="Appendix A combined-mode curves")
    ap.add_argument("--t", type=float, default=0.1, help="time of the combined-mode amplification factor")
    a = ap.parse_args()
    out = []
    if a.combined:
        for p in a.p:
            for eta in a.eta:
                for scheme in ("compact", "br1"):
                    th, G, om = combined_curves(p, scheme, eta, a.t, a.nth)
                    out.append({"p": p, "eta_ip": eta, "scheme": scheme, "t": a.t, "theta": th.tolist(),
                                "dissipation": om.imag.tolist(), "dispersion": om.real.tolist()})
        print(json.dumps(out))
        return
    for p in a.p:
        for eta in a.eta:
            for scheme in ("compact", "br1"):
                th, lam, imag = dissipation_curves(p, scheme, eta, a.nth)
                out.append({"p": p, "eta_ip": eta, "scheme": scheme, "theta": th.tolist(),
                            "eigenvalues": lam.tolist(), "max_imag": imag,
                            "zero_modes": zero_modes(p, scheme, eta)})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
