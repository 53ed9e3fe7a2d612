"""Oracle: Fourier transform, intensity and isotropic Q binning (paper Sec. 2.4-2.5).

TEST INFRASTRUCTURE ONLY.

Sec. 2.4 Eq. 1 defines the 3D transform with the 1/(MNL) normalisation:
    F(k) = (1/N^3) sum_x rho(x) exp(-2 pi i k.x / N).
The oracle evaluates it as one full complex FP64 FFT of the whole box (numpy's
pocketfft as a library step), not by the plane/column separation of Eq. 2, so
the separation is checked rather than assumed.  I = |F|^2 (Sec. 2.4, last
paragraph).

Sec. 2.5: every voxel gets |Q| from the box edge, the voxel count and its
distance from the centre of reciprocal space; intensities are averaged within
Q bins, with the standard error of the mean.

Readings:
* Axis index i in [0, N) has the signed frequency k = i for i < N/2, else i - N.
  |Q| = dq * sqrt(k^2), dq = 2 pi / (N dx), both in IEEE float64 (one multiply,
  one correctly rounded square root), so a voxel's bin is decided in float64
  from the integer k^2.
* Bins are half-open [e_j, e_j+1); the last bin also holds |Q| == e_B.
* Averages are over every voxel of the full N^3 grid in the bin: n_j voxels,
  mean = sum I / n_j, SEM = sqrt(sum (I - mean)^2 / (n_j (n_j - 1))).
  Empty bins have mean = NaN; bins with one voxel have SEM = NaN.
  The paper averages per slice and then combines slices with propagated
  uncertainties; the global average over all voxels is what that combination
  estimates and is the plain definition used here.
"""
from __future__ import annotations

import math

import numpy as np


def signed_freq(n: int) -> np.ndarray:
    k = np.arange(n, dtype=np.int64)
    k[k >= (n + 1) // 2] -= n
    return k


def dft3(rho: np.ndarray) -> np.ndarray:
    """Eq. 1: full complex FP64 3D DFT of rho[z][y][x], normalised by 1/N^3; F[kz][ky][kx]."""
    r = np.asarray(rho, dtype=np.float64)
    return np.fft.fftn(r) / float(r.size)


def dft_at(rho: np.ndarray, ks: np.ndarray, z_begin: int = 0) -> np.ndarray:
    """Eq. 1 evaluated directly at given signed frequencies ks[:, (kx, ky, kz)].

    rho holds planes [z_begin, z_begin + rho.shape[0]) of an N^3 box (all other
    planes zero).  The exponential factorises per axis, so each F(k) is three
    contractions over the stored voxels, in float64.
    """
    r = np.asarray(rho, dtype=np.float64)
    nzp, n, _ = r.shape
    xs = np.arange(n, dtype=np.float64)
    zs = np.arange(z_begin, z_begin + nzp, dtype=np.float64)
    out = np.empty(len(ks), dtype=np.complex128)
    for t, (kx, ky, kz) in enumerate(np.asarray(ks, dtype=np.int64)):
        ex = np.exp(-2j * np.pi * kx * xs / n)
        ey = np.exp(-2j * np.pi * ky * xs / n)
        ez = np.exp(-2j * np.pi * kz * zs / n)
        acc = r @ ex            # [z][y]
        acc = acc @ ey          # [z]
        out[t] = (acc * ez).sum()
    return out / float(n) ** 3


def intensity(F: np.ndarray) -> np.ndarray:
    return F.real * F.real + F.imag * F.imag


def dq_of(n: int, dx: float) -> float:
    return 2.0 * math.pi / (n * dx)


def q_of_k2(k2: np.ndarray, n: int, dx: float) -> np.ndarray:
    return dq_of(n, dx) * np.sqrt(np.asarray(k2, dtype=np.float64))


def bin_of_q(q: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """Bin index of each |Q| for half-open bins (last bin closed); -1 outside."""
    e = np.asarray(edges, dtype=np.float64)
    nb = len(e) - 1
    j = np.searchsorted(e, q, side="right") - 1
    j = np.where(q == e[-1], nb - 1, j)
    return np.where((j >= 0) & (j < nb), j, -1)


def _plane_k2(n: int, kz: int) -> np.ndarray:
    k = signed_freq(n)
    return kz * kz + (k * k)[:, None] + (k * k)[None, :]


def voxel_sinc(n: int) -> np.ndarray:
    """Intensity factor of one cubic voxel, prod_a sinc^2(q_a dx / 2), on the full grid [kz][ky][kx].

    Sec. 2.5 (last paragraph) mentions multiplying the pattern by a voxel-sized sinc for better
    high-Q behaviour.  Reading: the voxelised density is a sum of uniform cubes of edge dx
    centred on the samples, so its scattering amplitude is the DFT times the cube's form factor
    prod_a sin(q_a dx/2)/(q_a dx/2).  With q_a = 2 pi k_a/(N dx) the argument is pi k_a/N, so
    the factor depends on the integer frequency only.
    """
    k = signed_freq(n).astype(np.float64)
    a = np.pi * k / n
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.where(k == 0, 1.0, np.sin(a) / np.where(k == 0, 1.0, a))
    s2 = s * s
    return s2[:, None, None] * s2[None, :, None] * s2[None, None, :]


def bin_intensity(I: np.ndarray, n: int, dx: float, edges: np.ndarray) -> dict:
    """Sec. 2.5 isotropic averaging of a full-grid intensity I[kz][ky][kx] into Q bins."""
    nb = len(edges) - 1
    kz_all = signed_freq(n)
    count = np.zeros(nb, dtype=np.int64)
    s = np.zeros(nb, dtype=np.float64)
    sq = np.zeros(nb, dtype=np.float64)
    planes = []
    for iz in range(n):
        k2 = _plane_k2(n, int(kz_all[iz]))
        q = q_of_k2(k2, n, dx)
        j = bin_of_q(q, edges).ravel()
        ok = j >= 0
        jj = j[ok]
        planes.append(j)
        count += np.bincount(jj, minlength=nb)
        s += np.bincount(jj, weights=I[iz].ravel()[ok], minlength=nb)
        sq += np.bincount(jj, weights=q.ravel()[ok], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.where(count > 0, s / np.maximum(count, 1), np.nan)
    m2 = np.zeros(nb, dtype=np.float64)
    for iz in range(n):
        j = planes[iz]
        ok = j >= 0
        jj = j[ok]
        d = I[iz].ravel()[ok] - mean[jj]
        m2 += np.bincount(jj, weights=d * d, minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        sem = np.where(count > 1, np.sqrt(m2 / (count * np.maximum(count - 1, 1))), np.nan)
        mean_q = np.where(count > 0, sq / np.maximum(count, 1), np.nan)
    return {"count": count, "sum_i": s, "mean": mean, "sem": sem, "mean_q": mean_q, "m2": m2}


def forward(rho: np.ndarray, dx: float, edges: np.ndarray, voxel_sinc_correction: bool = False) -> dict:
    """ED -> F (Eq. 1) -> I = |F|^2 -> binned I(Q); returns the bins plus F and I.

    voxel_sinc_correction: bin I times voxel_sinc(N) (the intensity of the voxelised density
    rather than of point samples); the returned I is then the corrected one."""
    n = rho.shape[0]
    F = dft3(rho)
    I = intensity(F)
    if voxel_sinc_correction:
        I = I * voxel_sinc(n)
    out = bin_intensity(I, n, dx, edges)
    out["F"] = F
    out["I"] = I
    return out
