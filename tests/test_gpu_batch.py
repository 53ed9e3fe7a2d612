"""Batched particles of uneven grids: one launch sequence for all of them."""
import math

import numpy as np
import pytest
import torch

from oracle import density
from paper_2303_13435_gb300 import api, autotune, build, inputs

from _cases import GRAD_RTOL, MEAN_RTOL, compare_bins, normwise, oracle_forward, oracle_grads

pytestmark = pytest.mark.gpu

DX = 2.6 / 64


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()
    torch.cuda.init()


def _setup(count=6, lo=64, hi=128, seed=7, nbins=64):
    parts = inputs.batch_particles(count=count, seed=seed, lo=lo, hi=hi)
    edges = inputs.log_edges(2 * math.pi / (hi * DX), math.pi / DX, nbins)
    cell_np = inputs.mof_like_cell(64, 2.6, 0)
    cell = torch.from_numpy(cell_np).cuda()
    plans, rhos = [], []
    for p in parts:
        rho = density.tile_mask_density(p.n, cell_np, p.shape.kind, p.shape.center, p.shape.size, p.shape.rot)
        nzp = np.flatnonzero(rho.any(axis=(1, 2)))
        plans.append(api.Plan(p.n, DX, edges, z0=int(nzp[0]), nz=int(nzp[-1] - nzp[0] + 1)))
        rhos.append(rho)
    return parts, plans, rhos, cell, cell_np, edges


def _g(bins_np):
    return np.where(bins_np[0] > 0, 1e-3 / np.maximum(np.nan_to_num(bins_np[4]), 1e-300), 0.0)


def test_batch_matches_single_instance_and_oracle():
    parts, plans, rhos, cell, cell_np, edges = _setup()
    assert len({p.n for p in parts}) > 2          # really uneven
    batch = api.Batch(plans, cell, [p.shape for p in parts])
    batch.forward()
    singles = []
    for i, (p, plan) in enumerate(zip(parts, plans)):
        ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD)
        b1 = api.fft_intensity_tiled(plan, cell, p.shape, ws=ws)
        g = torch.from_numpy(_g(b1.cpu().numpy())).cuda()
        batch.dl_dmean[i].copy_(g)
        dc1, _ = api.backward(plan, g, b1, cell, p.shape, ws, want_mask=False)
        singles.append((b1.cpu().numpy(), dc1.cpu().numpy()))
    batch.backward()
    torch.cuda.synchronize()
    for i, (b1, dc1) in enumerate(singles):
        bb = batch.bins[i].cpu().numpy()
        assert np.array_equal(bb[0], b1[0])
        ok = b1[0] > 0
        assert np.allclose(bb[4][ok], b1[4][ok], rtol=MEAN_RTOL, atol=0)
        assert normwise(batch.dl_dcell[i].cpu().numpy(), dc1) <= GRAD_RTOL
    # two particles against the FP64 oracle
    for i in (0, len(parts) - 1):
        r64 = rhos[i].astype(np.float64)
        ob = oracle_forward(r64, DX, edges)
        compare_bins(batch.bins[i].cpu().numpy(), ob, r64, f"batch item {i}")
        mask = density.mask_values(parts[i].n, parts[i].shape.kind, parts[i].shape.center, parts[i].shape.size,
                                   parts[i].shape.rot)
        g = batch.dl_dmean[i].cpu().numpy()
        gu, _ = oracle_grads(r64, cell_np.astype(np.float64), mask, DX, edges, g, ob["count"])
        assert normwise(batch.dl_dcell[i].cpu().numpy(), gu) <= GRAD_RTOL


def test_batch_at_large_smooth_edges_matches_oracle():
    """Edges 250 = 2 5^3, 270 = 2 3^3 5 and 378 = 2 3^3 7 (radix-5 and radix-7 stages, runtime
    schedules) in one batch: bins against the FP64 oracle, and dL/du of the 250 particle against
    the oracle's gradient."""
    cell_np = inputs.mof_like_cell(64, 2.6, 0)
    cell = torch.from_numpy(cell_np).cuda()
    rot = inputs.random_rotation(inputs.SplitMix64(11))
    parts = [inputs.Particle(250, inputs.Shape(inputs.SHAPE_SPHERE, (125.0, 125.0, 125.0), 60.0)),
             inputs.Particle(270, inputs.Shape(inputs.SHAPE_CUBE, (135.0, 135.0, 135.0), 40.0, rot)),
             inputs.Particle(378, inputs.Shape(inputs.SHAPE_OCTAHEDRON, (189.0, 189.0, 189.0), 90.0, rot))]
    edges = inputs.log_edges(2 * math.pi / (378 * DX), math.pi / DX, 96)
    plans, rhos = [], []
    for p in parts:
        rho = density.tile_mask_density(p.n, cell_np, p.shape.kind, p.shape.center, p.shape.size, p.shape.rot)
        nzp = np.flatnonzero(rho.any(axis=(1, 2)))
        plans.append(api.Plan(p.n, DX, edges, z0=int(nzp[0]), nz=int(nzp[-1] - nzp[0] + 1)))
        rhos.append(rho)
    batch = api.Batch(plans, cell, [p.shape for p in parts])
    batch.forward()
    torch.cuda.synchronize()
    obs = []
    for i, p in enumerate(parts):
        r64 = rhos[i].astype(np.float64)
        ob = oracle_forward(r64, DX, edges)
        print(p.n, compare_bins(batch.bins[i].cpu().numpy(), ob, r64, f"batch edge {p.n}"))
        obs.append(ob)
    for i in range(len(parts)):
        batch.dl_dmean[i].copy_(torch.from_numpy(_g(batch.bins[i].cpu().numpy())).cuda())
    batch.backward()
    torch.cuda.synchronize()
    p = parts[0]
    mask = density.mask_values(p.n, p.shape.kind, p.shape.center, p.shape.size, p.shape.rot)
    gu, _ = oracle_grads(rhos[0].astype(np.float64), cell_np.astype(np.float64), mask, DX, edges,
                         batch.dl_dmean[0].cpu().numpy(), obs[0]["count"])
    assert normwise(batch.dl_dcell[0].cpu().numpy(), gu) <= GRAD_RTOL


def test_batch_in_one_cuda_graph():
    parts, plans, _, cell, _, _ = _setup(count=4, seed=11)
    batch = api.Batch(plans, cell, [p.shape for p in parts])
    for d in batch.dl_dmean:
        d.fill_(1e-4)
    batch.forward()
    batch.backward()
    torch.cuda.synchronize()
    ref_bins = [b.clone() for b in batch.bins]
    ref_grad = [g.clone() for g in batch.dl_dcell]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        batch.forward(stream=s)   # warm-up on the capture stream
        batch.backward(stream=s)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=s):
        batch.forward(stream=s)
        batch.backward(stream=s)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for b, rb in zip(batch.bins, ref_bins):
        ok = rb[0] > 0
        assert torch.equal(b[0], rb[0])
        assert torch.allclose(b[4][ok], rb[4][ok], rtol=MEAN_RTOL, atol=0)
    for g, rg in zip(batch.dl_dcell, ref_grad):
        assert normwise(g.cpu().numpy(), rg.cpu().numpy()) <= GRAD_RTOL


def test_autotuner_sets_tiles_and_keeps_results():
    parts, plans, _, cell, _, _ = _setup(count=3, seed=5)
    before = [p.tiles() for p in plans]
    batch = api.Batch(plans, cell, [p.shape for p in parts], with_backward=False)
    b0 = [b.cpu().numpy() for b in batch.forward()]
    batch.close()
    chosen = autotune.tune(plans, cell, [p.shape for p in parts], reps=1)
    assert set(chosen) == {p.n for p in parts}
    for p in plans:
        rb, tx, _ = chosen[p.n]
        assert p.tiles() == (rb, tx)
    batch = api.Batch(plans, cell, [p.shape for p in parts], with_backward=False)
    b1 = [b.cpu().numpy() for b in batch.forward()]
    for x, y in zip(b0, b1):
        ok = x[0] > 0
        assert np.allclose(x[4][ok], y[4][ok], rtol=MEAN_RTOL, atol=0)
    assert len(before) == len(plans)


def test_polydisperse_ensemble_on_the_batch_matches_oracle_and_its_gradient_flows():
    """Sec. 3 polydispersity: the volume-weighted ensemble of the batch's particle curves
    (ur_ensemble) against the oracle's ensemble of the oracle's particle curves, and the
    ensemble adjoint (ur_ensemble_backward) feeding the batch adjoint against the oracle's
    chain rule through the weights."""
    from oracle import merge as omerge, scatter
    parts, plans, rhos, cell, cell_np, edges = _setup(count=5, lo=64, hi=96, nbins=48)
    batch = api.Batch(plans, cell, [p.shape for p in parts])
    batch.forward()
    vols = [float((r != 0).sum()) * DX ** 3 for r in rhos]
    w = np.array([0.2 / v for v in vols])
    ens = api.ensemble(batch.bins, [p.n for p in parts], w).cpu().numpy()
    items = []
    for p, r in zip(parts, rhos):
        ob = oracle_forward(r.astype(np.float64), DX, edges)
        items.append({"n": p.n, "count": ob["count"], "mean": ob["mean"], "sem": ob["sem"], "mean_q": ob["mean_q"]})
    want = omerge.ensemble_sum(items, w)
    ok = want["count"] > 0
    assert ok.sum() > 10
    assert np.array_equal(ens[2][ok].astype(np.int64), want["count"][ok])
    assert np.all(np.isnan(ens[0][~ok]))
    assert np.max(np.abs(ens[0][ok] / want["mean"][ok] - 1)) <= MEAN_RTOL
    # the kernel's arithmetic against the oracle's on identical inputs (the GPU item curves)
    gi = [{"n": p.n, "count": b[0].astype(np.int64), "mean": b[4], "sem": b[5], "mean_q": b[3] / np.maximum(b[0], 1)}
          for p, b in zip(parts, [x.cpu().numpy() for x in batch.bins])]
    same = omerge.ensemble_sum(gi, w)
    assert np.allclose(ens[0][ok], same["mean"][ok], rtol=1e-13, atol=0)
    assert np.allclose(ens[1][ok], same["sem"][ok], rtol=1e-13, atol=0)
    # gradient: dL/dmean_i = w_i N_i^6 dL/dens on valid bins
    g = torch.from_numpy(np.where(ok, 1.0 / np.where(ok, want["mean"], 1.0), 0.0)).cuda()
    api.ensemble_backward(batch.bins, [p.n for p in parts], w, g, batch.dl_dmean)
    gn = g.cpu().numpy()
    for i, p in enumerate(parts):
        d = batch.dl_dmean[i].cpu().numpy()
        assert np.allclose(d, np.where(ok, w[i] * float(p.n) ** 6 * gn, 0.0), rtol=1e-14, atol=0)
    batch.backward()
    torch.cuda.synchronize()
    for i, (p, r) in enumerate(zip(parts, rhos)):
        gu, _ = oracle_grads(r.astype(np.float64), cell_np.astype(np.float64),
                             density.mask_values(p.n, p.shape.kind, p.shape.center, p.shape.size, p.shape.rot)
                             .astype(np.float64), DX, edges, batch.dl_dmean[i].cpu().numpy(), items[i]["count"])
        assert normwise(batch.dl_dcell[i].cpu().numpy(), gu) <= GRAD_RTOL
