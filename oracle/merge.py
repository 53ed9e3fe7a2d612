"""Oracle: merging the level curves ED-1/ED-2/ED-3 into one I(Q) (paper Sec. 2.5, last paragraph).

TEST INFRASTRUCTURE ONLY.

The paper combines the curves of the zoom levels with a final dataMerge step
and notes (Fig. 2 caption) that artefacts appear above Q_max/2.  The
measured curves of Sec. 2.7 are merged so that the uncertainties in the
overlapping regions are optimised.

Readings:
* Absolute units.  Each level's Eq.-1 intensity carries a 1/N^6 factor; the
  merge multiplies it back, I_abs = N^6 * mean, so every level is the squared
  modulus of the unnormalised sum over its voxels, in electrons^2.  Block sums
  keep the electron count, so I_abs(0) = N_e^2 at every level.
* Validity.  Q_max is the sampling frequency 2 pi / dx, so a level is trusted up
  to Q_max/2 = pi/dx (its Nyquist |Q| along an axis).
* mode "windows" (default).  Levels sorted by dx, coarsest first: the coarsest
  covers [0, QN_coarsest), each finer level covers [QN of the previous level,
  its own QN), and the finest level's window is closed at its QN.  An output
  bin takes the level whose window holds the bin's geometric centre
  sqrt(e_j e_j+1), and that level's statistics over the same edges.  Bins
  outside every window, or whose chosen level has no voxel in the bin, are NaN
  with count 0.
* mode "invvar" (the dataMerge-style combination of overlapping curves).  An
  output bin takes every level that is trusted at its geometric centre
  (centre <= pi/dx) and has voxels in the bin.  Levels with a finite, positive
  SEM are combined with weights 1/SEM^2: mean = sum w m / sum w,
  SEM = (sum w)^(-1/2), count = sum of the combined levels' counts, mean |Q| =
  the count-weighted mean of their mean |Q|.  When no trusted level has a
  usable SEM (one voxel, or zero spread), the bin falls back to the "windows"
  choice.  The source is the level of largest weight.
"""
from __future__ import annotations

import math

import numpy as np


def _windows_pick(qn_sorted, order, c):
    lo = 0.0
    for t, li in enumerate(order):
        last = t == len(order) - 1
        hi = qn_sorted[t]
        if lo <= c < hi or (last and c == hi):
            return li
        lo = hi
    return -1


def merge_levels(levels: list[dict], edges: np.ndarray, mode: str = "windows") -> dict:
    """levels: dicts with n (grid edge), dx (nm), count, mean, sem, mean_q over `edges`.

    Returns mean, sem (absolute units), count, mean_q and source (level index, -1 if none).
    """
    if mode not in ("windows", "invvar"):
        raise ValueError(f"unknown merge mode {mode}")
    e = np.asarray(edges, dtype=np.float64)
    nb = len(e) - 1
    order = sorted(range(len(levels)), key=lambda i: -levels[i]["dx"])
    qn = [math.pi / levels[i]["dx"] for i in order]
    mean = np.full(nb, np.nan)
    sem = np.full(nb, np.nan)
    mean_q = np.full(nb, np.nan)
    count = np.zeros(nb, dtype=np.int64)
    source = np.full(nb, -1, dtype=np.int64)
    for j in range(nb):
        c = math.sqrt(e[j] * e[j + 1])
        if mode == "invvar":
            sw = swm = cnt = sq = 0.0
            best, best_w = -1, -1.0
            for li, lv in enumerate(levels):
                if c > math.pi / lv["dx"] or lv["count"][j] <= 0:
                    continue
                s_abs = lv["sem"][j] * float(lv["n"]) ** 6
                if not (math.isfinite(s_abs) and s_abs > 0):
                    continue
                w = 1.0 / (s_abs * s_abs)
                sw += w
                swm += w * lv["mean"][j] * float(lv["n"]) ** 6
                cnt += lv["count"][j]
                sq += lv["count"][j] * lv["mean_q"][j]
                if w > best_w:
                    best, best_w = li, w
            if best >= 0:
                mean[j] = swm / sw
                sem[j] = 1.0 / math.sqrt(sw)
                count[j] = int(cnt)
                mean_q[j] = sq / cnt
                source[j] = best
                continue
        pick = _windows_pick(qn, order, c)
        if pick < 0:
            continue
        lv = levels[pick]
        if lv["count"][j] <= 0:
            continue
        scale = float(lv["n"]) ** 6
        mean[j] = lv["mean"][j] * scale
        sem[j] = lv["sem"][j] * scale
        mean_q[j] = lv["mean_q"][j]
        count[j] = lv["count"][j]
        source[j] = pick
    return {"mean": mean, "sem": sem, "count": count, "mean_q": mean_q, "source": source}


def ensemble_sum(items: list[dict], weights) -> dict:
    """Polydisperse ensemble (Sec. 3: about 200 volume-weighted single-particle simulations
    combined into one curve), over shared bin edges.

    items: dicts with n (grid edge), count, mean, sem, mean_q (Eq.-1 units of each item);
    weights: w_i per item (for volume weighting, w_i = phi_i / V_i with phi_i the volume
    fraction of the size class and V_i the particle volume).
    Readings: I_ens(Q_j) = sum_i w_i N_i^6 mean_ij (absolute units, electrons^2), valid only
    where every item of nonzero weight has voxels in bin j (else NaN, count 0);
    SEM_j = sqrt(sum_i (w_i N_i^6 SEM_ij)^2) (independent items); count and mean |Q| are the
    sums and the count-weighted mean over the items.
    """
    nb = len(items[0]["mean"])
    mean = np.full(nb, np.nan)
    sem = np.full(nb, np.nan)
    count = np.zeros(nb, dtype=np.int64)
    mean_q = np.full(nb, np.nan)
    for j in range(nb):
        ok = all(it["count"][j] > 0 for it, w in zip(items, weights) if w != 0)
        if not ok:
            continue
        s = v = cq = 0.0
        c = 0
        for it, w in zip(items, weights):
            if w == 0:
                continue
            sc = float(w) * float(it["n"]) ** 6
            s += sc * it["mean"][j]
            v += (sc * it["sem"][j]) ** 2
            c += int(it["count"][j])
            cq += it["count"][j] * it["mean_q"][j]
        mean[j] = s
        sem[j] = math.sqrt(v)
        count[j] = c
        mean_q[j] = cq / c
    return {"mean": mean, "sem": sem, "count": count, "mean_q": mean_q}
