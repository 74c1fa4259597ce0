"""Seeded Eulerian velocity field and Lagrangian marker forces.

Velocity: u(x) = sum_{m=1..8} a_m sin(pi k_m . x + theta_m), k_m integer with
1 <= |k_m|_inf <= kmax, a_m a random unit 3-vector, theta_m ~ U[0, 2pi).  On
[-1,1]^3 every mode is periodic.  The field is sampled at cell centres
(midpoints of adjacent faces) and stored structure-of-arrays, u[3][nz][ny][nx]
with x fastest.
"""

from dataclasses import dataclass

import math

import numpy as np


@dataclass
class FourierModes:
    k: np.ndarray        # (n_modes, 3) int
    a: np.ndarray        # (n_modes, 3) float64, unit vectors (one amplitude per component)
    theta: np.ndarray    # (n_modes,) float64


def fourier_modes(rng, n_modes=8, kmax=4):
    k = np.zeros((n_modes, 3), dtype=np.int64)
    for m in range(n_modes):
        while True:
            kk = rng.integers(-kmax, kmax + 1, size=3)
            if np.max(np.abs(kk)) >= 1:
                k[m] = kk
                break
    a = rng.normal(size=(n_modes, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    theta = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    return FourierModes(k=k, a=a, theta=theta)


def _centres(faces):
    return 0.5 * (faces[:-1] + faces[1:])


def field_at_cells_np(modes, faces, i, j, k):
    """Velocity (3, n) float64 at the centres of cells (i, j, k) (integer arrays)."""
    xc, yc, zc = (_centres(f) for f in faces)
    x, y, z = xc[i], yc[j], zc[k]
    u = np.zeros((3, np.size(i)))
    for m in range(len(modes.theta)):
        kx, ky, kz = modes.k[m]
        s = np.sin(np.pi * (kx * x + ky * y + kz * z) + modes.theta[m])
        u += modes.a[m][:, None] * s[None, :]
    return u


def field_full_np(modes, faces, dtype=np.float64):
    """Whole field u[3][nz][ny][nx] (small grids; uses the separable phase product)."""
    xc, yc, zc = (_centres(f) for f in faces)
    u = np.zeros((3, len(zc), len(yc), len(xc)))
    for m in range(len(modes.theta)):
        kx, ky, kz = modes.k[m]
        ex = np.exp(1j * np.pi * kx * xc)
        ey = np.exp(1j * np.pi * ky * yc)
        ez = np.exp(1j * (np.pi * kz * zc + modes.theta[m]))
        s = np.imag(ez[:, None, None] * ey[None, :, None] * ex[None, None, :])
        u += modes.a[m][:, None, None, None] * s[None]
    return u.astype(dtype)


def field_full_torch(modes, faces, dtype, device):
    """Same field as :func:`field_full_np`, evaluated with torch (float64) on ``device``."""
    import torch
    xc, yc, zc = (torch.as_tensor(_centres(f), dtype=torch.float64, device=device) for f in faces)
    out = torch.zeros((3, len(zc), len(yc), len(xc)), dtype=dtype, device=device)
    for c in range(3):
        acc = torch.zeros((len(zc), len(yc), len(xc)), dtype=torch.float64, device=device)
        for m in range(len(modes.theta)):
            kx, ky, kz = (int(v) for v in modes.k[m])
            ex = torch.exp(1j * math.pi * kx * xc.to(torch.complex128))
            ey = torch.exp(1j * math.pi * ky * yc.to(torch.complex128))
            ez = torch.exp(1j * (math.pi * kz * zc.to(torch.complex128) + float(modes.theta[m])))
            s = (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).imag
            acc += float(modes.a[m][c]) * s
        out[c] = acc.to(dtype)
    return out


def forces_np(rng, m):
    """Marker forces F[3][m], N(0,1), float64."""
    return rng.normal(size=(3, m))
