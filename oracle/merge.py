"""Oracle: merging the level curves ED-1/ED-2/ED-3 into one I(Q) (paper Sec. 2.5, last paragraph).

TEST INFRASTRUCTURE ONLY.

The paper combines the curves of the zoom levels with a final dataMerge step
and notes (Fig. 2 caption) that artefacts appear above Q_max/2.

Readings:
* Absolute units.  Each level's Eq.-1 intensity carries a 1/N^6 factor; the
  merge multiplies it back, I_abs = N^6 * mean, so every level is the squared
  modulus of the unnormalised sum over its voxels, in electrons^2.  Block sums
  keep the electron count, so I_abs(0) = N_e^2 at every level.
* Validity.  Q_max is the sampling frequency 2 pi / dx, so a level is trusted up
  to Q_max/2 = pi/dx (its Nyquist |Q| along an axis).
* Windows.  Levels sorted by dx, coarsest first: the coarsest covers
  [0, QN_coarsest), each finer level covers [QN of the previous level, its own
  QN), and the finest level's window is closed at its QN.  An output bin takes
  the level whose window holds the bin's geometric centre sqrt(e_j e_j+1), and
  that level's statistics over the same edges.  Bins outside every window, or
  whose chosen level has no voxel in the bin, are NaN with count 0.
"""
from __future__ import annotations

import math

import numpy as np


def merge_levels(levels: list[dict], edges: np.ndarray) -> dict:
    """levels: dicts with n (grid edge), dx (nm), count, mean, sem, mean_q over `edges`.

    Returns mean, sem (absolute units), count, mean_q and source (level index, -1 if none).
    """
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
        pick = -1
        lo = 0.0
        for t, li in enumerate(order):
            last = t == len(order) - 1
            hi = qn[t]
            if lo <= c < hi or (last and c == hi):
                pick = li
                break
            lo = hi
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
