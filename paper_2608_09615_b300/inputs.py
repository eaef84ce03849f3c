"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no step of the SD method: it only places samples of analytic fields
at the Gauss-Legendre solution points of each element (numpy's Gauss-Legendre rule is
used for placement) and draws random numbers with numpy's PCG64 generator. Both the
CUDA path and the CPU oracle receive the arrays it returns, so the two sides always see
bit-identical inputs.

Layout of every array: U[var][E_{dim-1}]...[E_0][n]...[n] (variable-major, then the
element grid with x fastest, then the points of each element with x fastest), float64.

Workloads (the paper's Sec. 4 test cases; every one is analytic, no dataset is needed):
  sin_1d        u0 = sin(x) on [0, 2 pi] (1D linear diffusion)
  heat_modes_3d u0 = sum_k a_k sin(k . x), 8 wavevectors k in Z^3, 0 < |k| <= 4, drawn
                without replacement from the half-space whose first nonzero component
                is positive, a_k ~ U(-1, 1)
  gaussian_1d   the Gaussian profile of Sec. 4.1
  dirac_1d      one element holding 1/h at all its points (an under-resolved delta)
  barenblatt_1d the ZKB solution of the porous medium equation at time t0 (Sec. 4.3)
  tgv_3d        the Taylor-Green initial field of Sec. 4.4, optionally plus a seeded
                smooth perturbation (random Fourier modes |k| <= 6, relative size 1e-2)
  random_state  uniform random point values around a reference state (parity only)
"""
import math

import numpy as np


def gl_points(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def element_shape(dim, ne, n):
    return tuple(reversed(tuple(ne))) + (n,) * dim


def coordinates(dim, ne, lo, hi, p):
    """Physical coordinates of the solution points: list over direction d (0 = x)
    of arrays of shape element_shape(dim, ne, p + 1)."""
    n = p + 1
    xs, _ = gl_points(n)
    shp = element_shape(dim, ne, n)
    out = []
    for d in range(dim):
        h = (hi[d] - lo[d]) / ne[d]
        s_e = [1] * (2 * dim)
        s_e[dim - 1 - d] = ne[d]
        s_p = [1] * (2 * dim)
        s_p[dim + dim - 1 - d] = n
        x = (lo[d] + h * np.arange(ne[d])).reshape(s_e) + (h / 2.0) * (xs + 1.0).reshape(s_p)
        out.append(np.broadcast_to(x, shp).copy())
    return out


def sin_1d(ne, p, lo=0.0, hi=2.0 * math.pi):
    (x,) = coordinates(1, (ne,), (lo,), (hi,), p)
    return np.sin(x)[None]


def gaussian_1d(ne, p, Dti=1.0 / 2400.0):
    (x,) = coordinates(1, (ne,), (0.0,), (1.0,), p)
    return (np.exp(-(x - 0.5) ** 2 / (4.0 * Dti)) / math.sqrt(4.0 * math.pi * Dti))[None]


def heat_wavevectors(seed, count=8, kmax=4):
    cand = []
    r = range(-kmax, kmax + 1)
    for kx in r:
        for ky in r:
            for kz in r:
                k = (kx, ky, kz)
                if k == (0, 0, 0) or kx * kx + ky * ky + kz * kz > kmax * kmax:
                    continue
                first = next(c for c in k if c != 0)
                if first > 0:
                    cand.append(k)
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(cand), size=count, replace=False)
    ks = [cand[i] for i in idx]
    amps = rng.uniform(-1.0, 1.0, size=count)
    return ks, amps


def heat_modes_3d(ne, p, seed, lo=(0.0, 0.0, 0.0), hi=(2 * math.pi,) * 3):
    ks, amps = heat_wavevectors(seed)
    X = coordinates(3, ne, lo, hi, p)
    u = np.zeros_like(X[0])
    for k, a in zip(ks, amps):
        u += a * np.sin(k[0] * X[0] + k[1] * X[1] + k[2] * X[2])
    return u[None], ks, amps


def dirac_1d(ne, p, elem, lo=0.0, hi=1.0):
    h = (hi - lo) / ne
    u = np.zeros((1, ne, p + 1))
    u[0, elem, :] = 1.0 / h
    return u


def barenblatt(x, t, m, C, d=1):
    """ZKB profile of the porous medium equation (Sec. 4.3, Eq. zkb), used to make
    initial data; [.]_+ = max(., 0)."""
    alpha = d / (d * (m - 1.0) + 2.0)
    beta = alpha / d
    core = C - alpha * (m - 1.0) / (2.0 * m * d) * x * x * t ** (-2.0 * beta)
    return t ** (-alpha) * np.maximum(core, 0.0) ** (1.0 / (m - 1.0))


def barenblatt_1d(ne, p, m=2.0, C=0.1, t0=1.0, lo=-10.0, hi=10.0):
    (x,) = coordinates(1, (ne,), (lo,), (hi,), p)
    return barenblatt(x, t0, m, C)[None]


def _smooth_field(rng, X, kmax, nmodes=12):
    """Sum of random Fourier modes with integer wavevectors, |k| <= kmax, normalised to
    max |f| <= 1 by construction (sum of |amplitudes| = 1)."""
    amps = rng.uniform(-1.0, 1.0, size=nmodes)
    amps /= np.sum(np.abs(amps))
    f = np.zeros_like(X[0])
    for a in amps:
        while True:
            k = rng.integers(-kmax, kmax + 1, size=3)
            if 0 < k @ k <= kmax * kmax:
                break
        ph = rng.uniform(0.0, 2.0 * math.pi)
        f += a * np.sin(k[0] * X[0] + k[1] * X[1] + k[2] * X[2] + ph)
    return f


def tgv_3d(ne, p, gamma=1.4, Ma=0.1, rho0=1.0, u0=1.0, L=1.0, perturb_seed=None,
           amp=1e-2, X=None):
    """Conservative Taylor-Green initial state (Sec. 4.4): domain [0, 2 pi L]^3,
    x* = (x - x_c)/L, rho = rho0, u = u0 (sin x* cos y* cos z*, -cos x* sin y* cos z*, 0),
    p = p0 + rho0 u0^2/16 (cos 2x* + cos 2y*)(cos 2z* + 2), p0 = rho0 (u0/Ma)^2/gamma.
    With perturb_seed, smooth random perturbations of relative size `amp` are added to
    rho, u and p so that no symmetry of the field can hide an indexing error.
    X: optional solution-point coordinates (e.g. curvilinear_coordinates of a deformed
    grid); by default those of the uniform grid with ne elements."""
    hi = (2.0 * math.pi * L,) * 3
    if X is None:
        X = coordinates(3, ne, (0.0,) * 3, hi, p)
    xs = [(X[d] - math.pi * L) / L for d in range(3)]
    rho = rho0 * np.ones_like(xs[0])
    u = u0 * np.sin(xs[0]) * np.cos(xs[1]) * np.cos(xs[2])
    v = -u0 * np.cos(xs[0]) * np.sin(xs[1]) * np.cos(xs[2])
    w = np.zeros_like(u)
    p0 = rho0 * (u0 / Ma) ** 2 / gamma
    pr = p0 + rho0 * u0 ** 2 / 16.0 * (np.cos(2 * xs[0]) + np.cos(2 * xs[1])) * (np.cos(2 * xs[2]) + 2.0)
    if perturb_seed is not None:
        rng = np.random.default_rng(perturb_seed)
        Xn = [X[d] / L for d in range(3)]
        rho = rho * (1.0 + amp * _smooth_field(rng, Xn, 6))
        u = u + amp * u0 * _smooth_field(rng, Xn, 6)
        v = v + amp * u0 * _smooth_field(rng, Xn, 6)
        w = w + amp * u0 * _smooth_field(rng, Xn, 6)
        pr = pr + amp * rho0 * u0 ** 2 * _smooth_field(rng, Xn, 6)
    return primitive_to_conservative(rho, (u, v, w), pr, gamma)


def primitive_to_conservative(rho, vel, pr, gamma):
    U = np.empty((5,) + rho.shape)
    U[0] = rho
    for i in range(3):
        U[1 + i] = rho * vel[i]
    U[4] = pr / (gamma - 1.0) + 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    return U


def random_state(ne, p, seed, gamma=1.4, Ma=0.1, rho0=1.0, u0=1.0, rel=0.1):
    """Uniform random point values: rho in rho0 (1 +- rel), velocity components in
    u0 [-1, 1], pressure in p0 (1 +- rel). Not smooth: used only for parity tests."""
    rng = np.random.default_rng(seed)
    shp = element_shape(3, ne, p + 1)
    p0 = rho0 * (u0 / Ma) ** 2 / gamma
    rho = rho0 * (1.0 + rel * rng.uniform(-1, 1, shp))
    vel = [u0 * rng.uniform(-1, 1, shp) for _ in range(3)]
    pr = p0 * (1.0 + rel * rng.uniform(-1, 1, shp))
    return primitive_to_conservative(rho, vel, pr, gamma)


def random_scalar(dim, ne, p, seed, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (1,) + element_shape(dim, ne, p + 1))


# ------------------------------------------------------------------ curvilinear grids
# A periodic structured grid of trilinear hexahedra is given by its corner nodes,
# nodes[c][k][j][i] (c = physical component, i along x), shape (3, nz + 1, ny + 1, nx + 1):
# element (ex, ey, ez) has the corners (ex + a, ey + b, ez + c), a, b, c in {0, 1}, and the
# last node along each axis is the periodic image of the first (node[..., nx] = node[..., 0]
# + the period vector along x, the same vector for every j, k).

def periodic_lattice(ne, lo=(0.0,) * 3, hi=(2 * math.pi,) * 3):
    """Corner nodes of the uniform grid of the box [lo, hi] with ne elements per axis."""
    ax = [np.linspace(lo[d], hi[d], ne[d] + 1) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([X, Y, Z])


def _periodic_displacement(ne, field):
    """Extend a displacement given on the nz x ny x nx lattice to the image nodes."""
    D = np.empty((3, ne[2] + 1, ne[1] + 1, ne[0] + 1))
    D[:, :-1, :-1, :-1] = field
    D[:, -1, :, :] = D[:, 0, :, :]
    D[:, :, -1, :] = D[:, :, 0, :]
    D[:, :, :, -1] = D[:, :, :, 0]
    return D


def jittered_lattice(ne, lo=(0.0,) * 3, hi=(2 * math.pi,) * 3, seed=0, amp=0.1):
    """Uniform lattice with each node moved by a seeded random vector whose components
    are uniform in [-amp h_d, amp h_d] (periodic: image nodes move with their originals).
    Every element stays a valid (positive-Jacobian) trilinear hexahedron for amp <= 0.15."""
    rng = np.random.default_rng(seed)
    h = [(hi[d] - lo[d]) / ne[d] for d in range(3)]
    f = rng.uniform(-1.0, 1.0, (3, ne[2], ne[1], ne[0]))
    for d in range(3):
        f[d] *= amp * h[d]
    return periodic_lattice(ne, lo, hi) + _periodic_displacement(ne, f)


def wavy_lattice(ne, lo=(0.0,) * 3, hi=(2 * math.pi,) * 3, amp=0.1):
    """Smooth periodic deformation of the uniform lattice: component d of each node moves
    by amp h_d sin(2 pi s_{d+1}) sin(2 pi s_{d+2}), s_t the node's position along axis t as
    a fraction of the box."""
    h = [(hi[d] - lo[d]) / ne[d] for d in range(3)]
    k, j, i = np.meshgrid(np.arange(ne[2]), np.arange(ne[1]), np.arange(ne[0]), indexing="ij")
    s = [i / ne[0], j / ne[1], k / ne[2]]
    f = np.stack([amp * h[d] * np.sin(2 * math.pi * s[(d + 1) % 3]) * np.sin(2 * math.pi * s[(d + 2) % 3])
                  for d in range(3)])
    return periodic_lattice(ne, lo, hi) + _periodic_displacement(ne, f)


def rotation_matrix(axis, angle):
    """Rotation by `angle` about the unit vector along `axis` (Rodrigues' formula)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def curvilinear_coordinates(nodes, p):
    """Physical coordinates of the solution points of every trilinear element (sample
    placement only): list over d of arrays shaped like one variable of U."""
    n = p + 1
    xs, _ = gl_points(n)
    nz, ny, nx = nodes.shape[1] - 1, nodes.shape[2] - 1, nodes.shape[3] - 1
    w = [np.stack([(1 - xs) / 2, (1 + xs) / 2]) for _ in range(3)]     # w[t][a][i]
    out = []
    for d in range(3):
        X = np.zeros((nz, ny, nx, n, n, n))
        for a in range(2):
            for b in range(2):
                for c in range(2):
                    corner = nodes[d, c:c + nz, b:b + ny, a:a + nx]
                    wt = np.einsum("k,j,i->kji", w[2][c], w[1][b], w[0][a])
                    X += corner[:, :, :, None, None, None] * wt
        out.append(X)
    return out
