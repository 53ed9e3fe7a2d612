"""Oracle: gradient of a loss on the binned intensity.  TEST INFRASTRUCTURE ONLY.

The paper has no adjoint; this is the plain chain rule through the forward
map of Sec. 2.3-2.5 (oracle.density, oracle.scatter):

    mean_j = (1/n_j) sum_{k in bin j} |F_k|^2,  F = Eq. 1 of rho,  rho = u(x mod U) m(x).

For g_j = dL/dmean_j and G_k = g_j / n_j on the voxels of bin j (0 elsewhere):

    dL/drho(x) = (2/N^3) Re sum_k G_k F_k exp(+2 pi i k.x/N)  = 2 Re(ifftn(G F))(x)
    dL/dm(x)   = dL/drho(x) * u(x mod U)
    dL/du(c)   = sum over x with (x + o) mod U = c of dL/drho(x) * m(x)

The float32 and FP16 roundings of the forward are not differentiated (the
gradient is that of the exact map).
"""
from __future__ import annotations

import numpy as np

from . import density, scatter


def bin_weights_per_voxel(n: int, dx: float, edges: np.ndarray, g: np.ndarray, count: np.ndarray) -> np.ndarray:
    """G_k = g_j / n_j on the full grid [kz][ky][kx]; zero outside the bins and for empty bins."""
    nb = len(edges) - 1
    gk = np.zeros(nb, dtype=np.float64)
    ok = count > 0
    gk[ok] = np.asarray(g, dtype=np.float64)[ok] / count[ok]
    kz_all = scatter.signed_freq(n)
    out = np.zeros((n, n, n), dtype=np.float64)
    k = scatter.signed_freq(n)
    for iz in range(n):
        k2 = int(kz_all[iz]) ** 2 + (k * k)[:, None] + (k * k)[None, :]
        j = scatter.bin_of_q(scatter.q_of_k2(k2, n, dx), edges)
        out[iz] = np.where(j >= 0, gk[np.maximum(j, 0)], 0.0)
    return out


def grad_rho(rho: np.ndarray, dx: float, edges: np.ndarray, g: np.ndarray, count=None, F=None) -> np.ndarray:
    """dL/drho for L depending on the bin means, FP64 [z][y][x]."""
    n = rho.shape[0]
    if F is None:
        F = scatter.dft3(rho)
    if count is None:
        count = scatter.bin_intensity(scatter.intensity(F), n, dx, edges)["count"]
    G = bin_weights_per_voxel(n, dx, edges, g, count)
    return 2.0 * np.fft.ifftn(G * F).real


def grad_cell_and_mask(grho: np.ndarray, cell: np.ndarray, mask: np.ndarray, origin=(0, 0, 0)):
    """(dL/du [U][U][U], dL/dm [z][y][x]) from dL/drho, the cell and the mask values."""
    n = grho.shape[0]
    u = cell.shape[0]
    ut = density.tiled_cell(n, cell, origin).astype(np.float64)
    gm = grho * ut
    ox, oy, oz = origin
    cz = (np.arange(n) + oz) % u
    cy = (np.arange(n) + oy) % u
    cx = (np.arange(n) + ox) % u
    flat = (cz[:, None, None] * u + cy[None, :, None]) * u + cx[None, None, :]
    gu = np.bincount(flat.ravel(), weights=(grho * mask.astype(np.float64)).ravel(), minlength=u ** 3)
    return gu.reshape(u, u, u), gm


def loss_log_mse(mean: np.ndarray, target: np.ndarray):
    """L = mean over bins with finite positive mean of (ln mean - ln target)^2, and dL/dmean."""
    ok = np.isfinite(mean) & (mean > 0)
    nv = max(int(ok.sum()), 1)
    d = np.zeros_like(mean, dtype=np.float64)
    d[ok] = np.log(mean[ok]) - np.log(target[ok])
    L = float((d[ok] ** 2).sum() / nv)
    g = np.zeros_like(d)
    g[ok] = 2.0 * d[ok] / (mean[ok] * nv)
    return L, g
