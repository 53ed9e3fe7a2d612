"""Host logic of the tile autotuner, with the GPU timing replaced by a fake.

The batched runtime-radix kernels take a tile shape per grid edge; the tuner
times a few shapes per edge, keeps the fastest, applies it to every plan of
that edge and caches the choice.  No GPU is touched here.
"""
import json

import pytest

from paper_2303_13435_gb300 import autotune


class FakePlan:
    def __init__(self, n, nbins=64):
        self.n = n
        self.nbins = nbins
        self.tiles = None

    def set_tiles(self, rows_per_block=0, cols_per_block=0):
        self.tiles = (rows_per_block, cols_per_block)


@pytest.mark.parametrize("n", [48, 96, 100, 210, 512, 1000, 2048])
def test_candidates_fit_one_block(n):
    cands = autotune._candidates(n)
    assert cands and len(set(cands)) == len(cands)
    for rb, tx in cands:
        assert 1 <= rb <= 64 and 1 <= tx <= 64
        # a 256-thread block holds at most 16 elements per thread; edges beyond that take one line
        assert rb * (n // 2) <= 16 * 256 or rb == 1
        assert tx * n <= 16 * 256 or tx == 1


def test_tune_picks_the_fastest_per_edge_applies_and_caches(tmp_path, monkeypatch):
    timed = []

    def fake_time(plan, cell, shape, reps):
        rb, tx = plan.tiles
        timed.append((plan.n, rb, tx))
        # a cost with a unique minimum inside the candidate set of each edge
        best = autotune._candidates(plan.n)[len(autotune._candidates(plan.n)) // 2]
        return 1.0 + abs(rb - best[0]) + 0.5 * abs(tx - best[1])

    monkeypatch.setattr(autotune, "_time_batch", fake_time)
    plans = [FakePlan(96), FakePlan(210), FakePlan(96), FakePlan(210)]
    cache = tmp_path / "tiles.json"
    chosen = autotune.tune(plans, [None] * 4, [None] * 4, cache_path=str(cache))
    for n in (96, 210):
        want = autotune._candidates(n)[len(autotune._candidates(n)) // 2]
        assert chosen[n][:2] == want and chosen[n][2] == 1.0
        # every candidate of the edge was timed once, on its first plan only
        assert sorted((rb, tx) for m, rb, tx in timed if m == n) == sorted(autotune._candidates(n))
    for p in plans:
        assert p.tiles == chosen[p.n][:2]
    assert json.load(open(cache)) == {f"{n}:64": list(chosen[n]) for n in (96, 210)}

    # a second tuning reads the cache and times nothing
    timed.clear()
    again = [FakePlan(210), FakePlan(96)]
    chosen2 = autotune.tune(again, [None] * 2, [None] * 2, cache_path=str(cache))
    assert timed == []
    assert {n: tuple(v) for n, v in chosen2.items()} == {n: tuple(v) for n, v in chosen.items()}
    for p in again:
        assert p.tiles == chosen[p.n][:2]


def test_cache_is_keyed_by_bin_count(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_time_batch", lambda plan, c, s, reps: float(sum(plan.tiles)))
    cache = tmp_path / "tiles.json"
    autotune.tune([FakePlan(96, nbins=64)], [None], [None], cache_path=str(cache))
    calls = []
    monkeypatch.setattr(autotune, "_time_batch", lambda plan, c, s, reps: calls.append(1) or 1.0)
    autotune.tune([FakePlan(96, nbins=128)], [None], [None], cache_path=str(cache))
    assert len(calls) == len(autotune._candidates(96))
    assert set(json.load(open(cache))) == {"96:64", "96:128"}
