"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds input generation only, none of the particle method's
arithmetic: turbulent fields built from random Fourier modes, a lognormal
density, E = -v x B, and numpy-drawn particle sets.  The paper's workloads are
its own synthetic tests (Sec. 4.1, Sec. 4.2); these fields stand in for the
fluid snapshots a (R)MHD run would supply.

Field recipe (periodic on [-1, 1]^dim, cell-centred, layout [comp][z][y][x]):
  delta(x) = sum_{m=1}^{64} A_m xi_m cos(k_m . x + phi_m)
  k_m = (2 pi / L) * integer vector, |k_m| log-spaced in [1, n/4] grid modes,
  random direction; xi_m a unit vector orthogonal to k_m (solenoidal);
  A_m^2 ~ k^{-5/3} k dln k (Kolmogorov on log spacing); phi_m uniform; the sum
  is scaled so that the grid rms of |delta| equals the requested rms.
"""
from __future__ import annotations

import numpy as np

try:  # multi-threaded FFT when scipy is present
    import scipy.fft as _fft

    def _ifftn(a):
        return _fft.ifftn(a, workers=-1)
except Exception:  # pragma: no cover
    def _ifftn(a):
        return np.fft.ifftn(a)


def grid_shape(dim: int, n: int):
    """(nz, ny, nx) of a cubic/square grid with n cells per axis."""
    return (n, n, n) if dim == 3 else (1, n, n)


def _modes(rng, dim: int, n: int, nmodes: int, vector: bool):
    kmax = max(1.0, n / 4.0)
    kmag = np.exp(np.linspace(0.0, np.log(kmax), nmodes))
    out = []
    for km in kmag:
        d = rng.standard_normal(3)
        if dim == 2:
            d[2] = 0.0
        d /= np.linalg.norm(d)
        m = np.rint(km * d).astype(np.int64)
        if not m.any():
            a = int(np.argmax(np.abs(d)))
            m[a] = 1 if d[a] >= 0 else -1
        mh = m / np.linalg.norm(m)
        if vector:
            r = rng.standard_normal(3)
            xi = r - np.dot(r, mh) * mh
            xi /= np.linalg.norm(xi)
        else:
            xi = np.ones(1)
        amp = np.linalg.norm(m) ** (-1.0 / 3.0)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        out.append((m, xi, amp, phi))
    return out


def _evaluate(modes, dim: int, n: int, ncomp: int, xmin=-1.0, L=2.0):
    nz, ny, nx = grid_shape(dim, n)
    nn = (nx, ny, nz)
    out = np.zeros((ncomp, nz, ny, nx))
    for c in range(ncomp):
        X = np.zeros((nz, ny, nx), dtype=np.complex128)
        for m, xi, amp, phi in modes:
            # phase of k.x at the cell centre x_j = xmin + (j + 1/2) L/n
            th = phi + sum(2.0 * np.pi * m[a] * (xmin / L + 0.5 / nn[a])
                           for a in range(3) if nn[a] > 1)
            idx = (int(m[2]) % nz, int(m[1]) % ny, int(m[0]) % nx)
            X[idx] += amp * xi[c if xi.shape[0] > 1 else 0] * np.exp(1j * th)
        out[c] = np.real(_ifftn(X)) * X.size
    return out


def turbulent_vector(dim: int, n: int, seed: int, rms: float, nmodes: int = 64):
    """Solenoidal random-phase Kolmogorov field [3][z][y][x] with grid rms |.|."""
    rng = np.random.default_rng(seed)
    f = _evaluate(_modes(rng, dim, n, nmodes, True), dim, n, 3)
    cur = np.sqrt(np.mean(np.sum(f * f, axis=0)))
    return f * (rms / cur)


def gaussian_scalar(dim: int, n: int, seed: int, nmodes: int = 64):
    """Zero-mean, unit-variance random-phase scalar field [z][y][x]."""
    rng = np.random.default_rng(seed)
    g = _evaluate(_modes(rng, dim, n, nmodes, False), dim, n, 1)[0]
    g = g - g.mean()
    return g / g.std()


def cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


def em_fields(dim: int, n: int, seed: int, b0: float = 1.0, db_rms: float = 1.0,
              v_rms: float = 0.01, nmodes: int = 64):
    """E and B [6][z][y][x]: B = b0 z + turbulent dB (rms db_rms), E = -v x B,
    v a solenoidal turbulent velocity with rms |v| = v_rms (c = 1)."""
    B = turbulent_vector(dim, n, seed, db_rms, nmodes)
    B[2] += b0
    v = turbulent_vector(dim, n, seed + 100003, v_rms, nmodes)
    E = -cross(v, B)
    return np.concatenate([E, B], axis=0)


def uniform_em_fields(dim: int, n: int, B=(0.0, 0.0, 1.0), E=(0.0, 0.0, 0.0)):
    nz, ny, nx = grid_shape(dim, n)
    f = np.zeros((6, nz, ny, nx))
    for c in range(3):
        f[c] = E[c]
        f[3 + c] = B[c]
    return f


def fluid_snapshot(dim: int, n: int, seed: int, v_rms: float = 0.01, sigma: float = 0.5,
                   b0: float = 1.0, db_rms: float = 1.0, nmodes: int = 64):
    """(vel [3], rho [1], B [3]) for the Lagrangian-particle workload:
    solenoidal v (rms v_rms), lognormal rho = exp(sigma g - sigma^2/2),
    B = b0 z + turbulent dB."""
    vel = turbulent_vector(dim, n, seed + 100003, v_rms, nmodes)
    g = gaussian_scalar(dim, n, seed + 200003, nmodes)
    rho = np.exp(sigma * g - 0.5 * sigma * sigma)[None]
    B = turbulent_vector(dim, n, seed, db_rms, nmodes)
    B[2] += b0
    return vel, rho, B


def particles(dim: int, n_cells, npart: int, seed: int, u_th: float = 0.1,
              xmin=(-1.0, -1.0, -1.0), L=(2.0, 2.0, 2.0)):
    """Uniform random positions over the domain and Maxwellian u ~ N(0, u_th^2)
    per component; w = 1; id = index.  Positions [3][n], z pinned to the
    mid-plane when dim == 2."""
    rng = np.random.default_rng(seed)
    x = np.empty((3, npart))
    for a in range(3):
        if a < dim:
            x[a] = xmin[a] + L[a] * rng.random(npart)
            # keep strictly inside [xmin, xmin + L)
            x[a] = np.where(x[a] >= xmin[a] + L[a], xmin[a], x[a])
        else:
            x[a] = xmin[a] + 0.5 * L[a]
    u = rng.standard_normal((3, npart)) * u_th
    w = np.ones(npart)
    ids = np.arange(npart, dtype=np.uint64)
    return x, u, w, ids
