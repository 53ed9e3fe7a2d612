"""Tile autotuner for the runtime-radix (any {2,3,5,7}-smooth edge) kernels.

For every distinct grid edge of a set of plans it times the batched forward +
adjoint of one representative particle for a few tile shapes (rows per block
of the row passes, columns per block of the column passes), keeps the fastest
and applies it to every plan of that edge.  Results can be cached in a JSON
file keyed by edge and bin count.
"""
from __future__ import annotations

import json
import os

import torch

from . import api


def _candidates(n: int):
    emax = 16 * 256  # elements a 256-thread block holds
    rb_max = max(1, min(64, emax // (n // 2)))
    tx_max = max(1, min(64, emax // n))
    rbs = sorted({max(1, rb_max // d) for d in (1, 2, 4)}, reverse=True)
    txs = sorted({max(1, tx_max // d) for d in (1, 2, 4)}, reverse=True)
    return [(r, t) for r in rbs for t in txs]


def _time_batch(plan, cell, shape, reps: int) -> float:
    b = api.Batch([plan], [cell], [shape], with_backward=True)
    b.dl_dmean[0].fill_(1e-3)
    for _ in range(2):
        b.forward()
        b.backward()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        b.forward()
        b.backward()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    b.close()
    return ms


def tune(plans, cells, shapes, reps: int = 3, cache_path: str | None = None, verbose: bool = False) -> dict:
    """Choose tiles per grid edge; returns {edge: (rows, cols, ms)} and applies them."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        cache = json.load(open(cache_path))
    cells = list(cells) if isinstance(cells, (list, tuple)) else [cells] * len(plans)
    chosen = {}
    rep = {}
    for p, c, s in zip(plans, cells, shapes):
        rep.setdefault(p.n, (p, c, s))
    for n, (p, c, s) in sorted(rep.items()):
        key = f"{n}:{p.nbins}"
        if key in cache:
            chosen[n] = tuple(cache[key])
            continue
        best = None
        for rb, tx in _candidates(n):
            p.set_tiles(rb, tx)
            ms = _time_batch(p, c, s, reps)
            if verbose:
                print(f"  N={n} rows/block={rb} cols/block={tx}: {ms:.3f} ms")
            if best is None or ms < best[2]:
                best = (rb, tx, ms)
        chosen[n] = best
        cache[key] = list(best)
    for p in plans:
        rb, tx, _ = chosen[p.n]
        p.set_tiles(rb, tx)
    if cache_path:
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return chosen
