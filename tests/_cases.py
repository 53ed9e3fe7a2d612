"""Shared helpers of the GPU parity tests: oracle side and comparison rules.

Tolerances (stated here once, used by every parity test):
* ED voxels, bin counts, bin thresholds: bit-exact.
* Bin means I(Q): |I_gpu - I_oracle| <= 1e-4 * I_oracle for every bin whose
  oracle mean is at least 1e-6 of the Parseval mean <I> = sum(rho^2) / N^6.
  FP32 butterflies carry an absolute error of about eps * log2(N) * rms|F|,
  so bins far below the mean intensity cannot meet a relative bound; they
  are counted and reported, not gated.
* Sum of |Q| per bin: relative 1e-12 (data independent, FP64 on both sides).
* SEM: relative 1e-3 where the within-bin spread (std / mean) is at least
  1e-3 and the mean is at least 1e-4 of <I>.  Below that spread the FP32
  transform's own error (about 1e-6 of I) is a visible part of the variance;
  shells whose voxels are equal by symmetry have an SEM of rounding size on
  both sides and are not comparable.
* Gradients: normwise relative error <= 1e-4 against the FP64 oracle.
"""
from __future__ import annotations

import json
import os

import numpy as np

from oracle import adjoint, density, scatter

MEAN_RTOL = 1e-4
FLOOR = 1e-6
GRAD_RTOL = 1e-4


def oracle_density(w, z_begin=0, z_count=None, out_dtype="f32", weights=None):
    s = w.shape
    return density.tile_mask_density(w.n, w.cell, s.kind, s.center, s.size, s.rot, origin=w.origin,
                                     weights=weights, out_dtype=out_dtype, z_begin=z_begin, z_count=z_count)


def parseval_mean(rho64: np.ndarray) -> float:
    n = rho64.shape[0]
    return float((rho64 ** 2).sum()) / float(n) ** 6


def compare_bins(gpu_bins: np.ndarray, ob: dict, rho64: np.ndarray, label: str = "") -> dict:
    """Gate GPU bins [6, B] against oracle bins; returns the error report."""
    cnt = gpu_bins[0]
    assert np.array_equal(cnt.astype(np.int64), ob["count"]), f"{label}: counts differ"
    nz = ob["count"] > 0
    sq_ref = ob["mean_q"] * ob["count"]
    assert np.allclose(gpu_bins[3][nz], sq_ref[nz], rtol=1e-12, atol=0), f"{label}: sum |Q| differs"
    mean_g = gpu_bins[4]
    mean_o = ob["mean"]
    floor = FLOOR * parseval_mean(rho64)
    gate = nz & (mean_o >= floor)
    with np.errstate(invalid="ignore", divide="ignore"):
        rel = np.abs(mean_g - mean_o) / np.abs(mean_o)
    worst = float(np.nanmax(rel[gate])) if gate.any() else 0.0
    assert worst <= MEAN_RTOL, f"{label}: max rel err {worst:.3e} over {gate.sum()} gated bins"
    assert np.all(np.isnan(mean_g[~nz])), f"{label}: empty bins must be NaN"
    # SEM where the spread is resolvable
    sem_o = ob["sem"]
    spread = sem_o * np.sqrt(np.maximum(ob["count"], 1)) / np.where(mean_o > 0, mean_o, np.inf)
    sgate = gate & (ob["count"] > 1) & (spread >= 1e-3) & (mean_o >= 1e-4 * parseval_mean(rho64))
    if sgate.any():
        srel = np.abs(gpu_bins[5][sgate] - sem_o[sgate]) / sem_o[sgate]
        assert float(srel.max()) <= 1e-3, f"{label}: SEM rel err {srel.max():.3e}"
    if os.environ.get("UR_SEM_LOG"):
        # SEM error by within-bin spread, for the record (not gated here)
        ok = gate & (ob["count"] > 1) & (sem_o > 0)
        with np.errstate(invalid="ignore", divide="ignore"):
            er = np.abs(gpu_bins[5] - sem_o) / sem_o
        rec = {"label": label, "n": int(rho64.shape[0])}
        for lo, hi in [(0.05, np.inf), (0.01, 0.05), (1e-3, 0.01), (0.0, 1e-3)]:
            sel = ok & (spread >= lo) & (spread < hi)
            rec[f"spread_{lo:g}"] = [int(sel.sum()), float(np.nanmax(er[sel])) if sel.any() else None]
        with open(os.environ["UR_SEM_LOG"], "a") as f:
            f.write(json.dumps(rec) + "\n")
    return {"gated": int(gate.sum()), "excluded": int((nz & ~gate).sum()), "max_rel_gated": worst,
            "max_rel_all": float(np.nanmax(rel[nz])) if nz.any() else 0.0}


def oracle_forward(rho, dx, edges):
    return scatter.forward(np.asarray(rho, dtype=np.float64), dx, edges)


def normwise(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_grads(rho64, cell, mask, dx, edges, g, count, origin=(0, 0, 0)):
    grho = adjoint.grad_rho(rho64, dx, edges, g, count=count)
    return adjoint.grad_cell_and_mask(grho, cell, mask, origin)


def oracle_parity_counts(n, dx, edges):
    """Per bin of the oracle's binning: voxels of the grid with kx even, and all voxels.  The
    number of k with kx^2 + ky^2 + kz^2 = s is the convolution of the three axes' histograms of
    k^2 (integer counts, convolved exactly by FFT in float64 and rounded); each s then takes the
    oracle's bin of q(s)."""
    k = scatter.signed_freq(n)
    smax = 3 * (n // 2) ** 2
    h_all = np.bincount(k * k, minlength=smax + 1).astype(np.float64)
    h_even = np.bincount((k * k)[k % 2 == 0], minlength=smax + 1).astype(np.float64)
    m = 1 << int(np.ceil(np.log2(3 * (smax + 1))))
    fa = np.fft.rfft(h_all, m)
    h3_even = np.rint(np.fft.irfft(np.fft.rfft(h_even, m) * fa * fa, m)[:smax + 1]).astype(np.int64)
    h3_all = np.rint(np.fft.irfft(fa * fa * fa, m)[:smax + 1]).astype(np.int64)
    j = scatter.bin_of_q(scatter.q_of_k2(np.arange(smax + 1), n, dx), edges)
    nb = len(edges) - 1
    ok = j >= 0
    return (np.bincount(j[ok], weights=h3_even[ok], minlength=nb).astype(np.int64),
            np.bincount(j[ok], weights=h3_all[ok], minlength=nb).astype(np.int64))
