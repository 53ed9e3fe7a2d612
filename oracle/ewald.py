"""Oracle: a 2D detector image cut from the 3D intensity along the Ewald sphere (paper Sec. 2.5).

TEST INFRASTRUCTURE ONLY.

Sec. 2.5 (first paragraph): for anisotropic samples, 2D data that a practical
experiment would record can be extracted by modelling the Ewald sphere as a
shell whose thickness is set by the wavelength distribution, and reading the
intensity on that surface.

Readings (the paper gives no detector model):
* Flat detector perpendicular to the beam (+z) at distance L; pixel (ix, iy)
  sits at ((ix - bx) p, (iy - by) p, L) for pixel pitch p and direct-beam
  position (bx, by) in pixel units; s is the unit vector towards it.
* Wavelength distribution: uniform over lambda0 (1 + b ((l + 1/2)/nl - 1/2)),
  l < nl (relative full width b; nl = 1, b = 0: monochromatic).  For each
  wavelength q_lab = (2 pi / lambda)(s - z_hat) (nm^-1), and the sample frame is
  q = R^T q_lab for the sample orientation R.
* The grid holds I at q = dq k, dq = 2 pi / (N dx), k the signed integer
  frequency; a q between grid points takes the trilinear interpolation of I
  over its 8 neighbours.  A sample is valid when all neighbours lie inside
  [-N/2, N/2 - 1] on every axis; a pixel is the mean over its valid samples,
  NaN when it has none.
* I is in the Eq. 1 normalisation of oracle.scatter (multiply by N^6 for
  electrons^2).
"""
from __future__ import annotations

import math

import numpy as np

from . import scatter


def pixel_directions(det: dict) -> np.ndarray:
    """Unit vectors s towards every pixel, [ny][nx][3] (x, y, z)."""
    iy, ix = np.mgrid[0:det["ny"], 0:det["nx"]].astype(np.float64)
    x = (ix - det["beam"][0]) * det["pixel_m"]
    y = (iy - det["beam"][1]) * det["pixel_m"]
    z = np.full_like(x, det["distance_m"])
    r = np.sqrt(x * x + y * y + z * z)
    return np.stack([x / r, y / r, z / r], axis=-1)


def wavelengths(det: dict) -> np.ndarray:
    nl = int(det.get("nlambda", 1))
    b = float(det.get("bandwidth", 0.0))
    lam0 = float(det["wavelength_nm"])
    return np.array([lam0 * (1.0 + b * ((l + 0.5) / nl - 0.5)) for l in range(nl)])


def q_samples(det: dict) -> np.ndarray:
    """Sample-frame q (nm^-1) of every pixel and wavelength, [nl][ny][nx][3]."""
    s = pixel_directions(det)
    zhat = np.array([0.0, 0.0, 1.0])
    rot = np.asarray(det.get("rot", np.eye(3)), dtype=np.float64).reshape(3, 3)
    out = []
    for lam in wavelengths(det):
        q_lab = (2.0 * math.pi / lam) * (s - zhat)
        out.append(q_lab @ rot)          # (R^T q)_a = sum_b R[b][a] q_b
    return np.stack(out)


def trilinear(I_full: np.ndarray, kf: np.ndarray):
    """Trilinear interpolation of I_full[kz][ky][kx] (signed frequencies wrap mod N) at the
    fractional frequencies kf[..., (kx, ky, kz)]; returns (values, valid)."""
    n = I_full.shape[0]
    i0 = np.floor(kf).astype(np.int64)
    f = kf - i0
    valid = np.all((i0 >= -(n // 2)) & (i0 + 1 <= n // 2 - 1), axis=-1)
    val = np.zeros(kf.shape[:-1])
    for dz in (0, 1):
        for dy in (0, 1):
            for dxx in (0, 1):
                w = ((f[..., 0] if dxx else 1 - f[..., 0]) * (f[..., 1] if dy else 1 - f[..., 1])
                     * (f[..., 2] if dz else 1 - f[..., 2]))
                val += w * I_full[(i0[..., 2] + dz) % n, (i0[..., 1] + dy) % n, (i0[..., 0] + dxx) % n]
    return val, valid


def ewald_image(F: np.ndarray, dx: float, det: dict) -> np.ndarray:
    """Detector image [ny][nx] of the intensity of the full-grid transform F (Eq. 1)."""
    n = F.shape[0]
    I_full = scatter.intensity(F)
    kf = q_samples(det) / scatter.dq_of(n, dx)
    val, valid = trilinear(I_full, kf)
    num = np.where(valid, val, 0.0).sum(axis=0)
    cnt = valid.sum(axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(cnt > 0, num / np.maximum(cnt, 1), np.nan)
