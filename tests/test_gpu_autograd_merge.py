"""Autograd wrapper and the three-level (ED-1/ED-2/ED-3) merge workload on the GPU."""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint, density, merge as omerge, scatter
from paper_2303_13435_gb300 import api, build, inputs
from paper_2303_13435_gb300.autograd import binned_intensity

from _cases import GRAD_RTOL, MEAN_RTOL, normwise, oracle_density, oracle_grads, parseval_mean

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()
    torch.cuda.init()


def _small_workload(n=64):
    w = inputs.mof_workload(n=n, diameter_nm=0.6 * n * 0.65 / 16, nbins=48, ucell=16, a_nm=0.65)
    return w


def _log_mse_torch(mean, target):
    ok = torch.isfinite(mean) & (mean > 0)
    d = torch.log(mean[ok]) - torch.log(target[ok])
    return (d * d).mean()


def test_autograd_gradients_match_oracle():
    w = _small_workload()
    n = w.n
    weights = np.random.default_rng(11).random((n, n, n)).astype(np.float32)
    weights[:12] = 0
    weights[52:] = 0
    rho = density.tile_mask_density(n, w.cell, density.WEIGHTS, weights=weights)
    nzp = np.flatnonzero(rho.any(axis=(1, 2)))
    plan = api.Plan(n, w.dx, w.edges, z0=int(nzp[0]), nz=int(nzp[-1] - nzp[0] + 1))
    cell = torch.from_numpy(w.cell).cuda().requires_grad_(True)
    wt = torch.from_numpy(weights).cuda().requires_grad_(True)
    mean = binned_intensity(cell, plan, inputs.Shape(inputs.SHAPE_WEIGHTS), weights=wt)
    target = torch.from_numpy(np.nan_to_num(mean.detach().cpu().numpy(), nan=1.0) * 1.3 + 1e-12).cuda()
    loss = _log_mse_torch(mean, target)
    loss.backward()
    # oracle: same dL/dmean from the same means, then the FP64 chain rule
    m = mean.detach().cpu().numpy()
    _, g = adjoint.loss_log_mse(m, target.cpu().numpy())
    count = scatter.bin_intensity(np.zeros((n, n, n)), n, w.dx, w.edges)["count"]
    gu, gm = oracle_grads(rho.astype(np.float64), w.cell.astype(np.float64), weights.astype(np.float64), w.dx, w.edges,
                          g, count)
    eu = normwise(cell.grad.cpu().numpy(), gu)
    em = normwise(wt.grad.cpu().numpy(), gm)
    assert eu <= GRAD_RTOL and em <= GRAD_RTOL, (eu, em)


def test_autograd_directional_derivative_on_the_gpu():
    """<dL/du, d> against a central difference of the GPU forward itself (FP32: 1e-2)."""
    w = _small_workload()
    plan = api.Plan(w.n, w.dx, w.edges)
    cell = torch.from_numpy(w.cell).cuda().double().float().requires_grad_(True)
    mean = binned_intensity(cell, plan, w.shape)
    target = torch.nan_to_num(mean.detach(), nan=1.0) * 0.7 + 1e-12
    loss = _log_mse_torch(mean, target)
    loss.backward()
    d = torch.from_numpy(np.random.default_rng(2).standard_normal(w.cell.shape).astype(np.float32)).cuda()
    d *= 0.01 * cell.detach().abs().mean() / d.abs().mean()
    h = 0.5
    with torch.no_grad():
        lp = _log_mse_torch(binned_intensity(cell.detach() + h * d, plan, w.shape), target).item()
        lm = _log_mse_torch(binned_intensity(cell.detach() - h * d, plan, w.shape), target).item()
    fd = (lp - lm) / (2 * h)
    an = float((cell.grad * d).sum().item())
    assert math.isclose(fd, an, rel_tol=1e-2), (fd, an)


def test_autograd_reuses_the_plan_workspace_and_survives_interleaved_forwards():
    """One workspace per plan for every forward; a backward that runs after another forward
    wrote that workspace restores its own intermediate first and gets the same gradient."""
    w = _small_workload()
    plan = api.Plan(w.n, w.dx, w.edges)
    base = torch.from_numpy(w.cell).cuda()

    def grad_of(cell_t, pl, interleave=None):
        c = cell_t.clone().requires_grad_(True)
        mean = binned_intensity(c, pl, w.shape)
        if interleave is not None:
            binned_intensity(interleave, pl, w.shape)   # claims and overwrites the workspace
        torch.nan_to_num(mean).sum().backward()
        return c.grad.clone()

    binned_intensity(base, plan, w.shape)
    ws_first = plan._ws.data_ptr()
    g_inter = grad_of(base, plan, interleave=base * 1.7)
    assert plan._ws.data_ptr() == ws_first
    g_alone = grad_of(base, api.Plan(w.n, w.dx, w.edges))
    assert normwise(g_inter.cpu().numpy(), g_alone.cpu().numpy()) <= 1e-6


def _levels_gpu(ed1_dev, n1, dx1, zooms, edges):
    """Transform every level on common edges; returns (bins tensors, N list, dx list, box totals)."""
    out_bins, ns, dxs = [], [], []
    lv = [(ed1_dev, n1, dx1)]
    for f, n_out in zooms:
        lv.append((api.zoom_density(ed1_dev, f, n_out, out_dtype="f16"), n_out, dx1 * f))
    for ed, n, dx in lv:
        occ = torch.nonzero(ed.float().abs().sum(dim=(1, 2)) > 0).flatten()
        z0, z1 = int(occ[0]), int(occ[-1])
        plan = api.Plan(n, dx, edges, z0=z0, nz=z1 - z0 + 1, ed_dtype="f16")
        out_bins.append(api.fft_intensity(plan, ed[z0:z1 + 1].contiguous()))
        ns.append(n)
        dxs.append(dx)
    return out_bins, ns, dxs, lv


def test_three_level_merge_matches_oracle_reduced():
    """Sec. 2.3 zoom-out + Sec. 2.5 merge on a reduced three-level workload:
    ED-1 = 256^3 FP16 cube filling the box, ED-2/ED-3 = 4x/16x block sums in 128^3 boxes."""
    n1 = 256
    ed1w, _ = inputs.cube_merge_levels(n1=n1, n_low=128, factors=(4, 16), edge_nm=5.0, ucell=128, a_nm=2.5,
                                       nbins=150, qlo=0.05, qhi=150.0)
    edges = ed1w.edges
    ed1 = oracle_density(ed1w, out_dtype="f16")
    bins, ns, dxs, lv = _levels_gpu(torch.from_numpy(ed1).cuda(), n1, ed1w.dx, [(4, 128), (16, 128)], edges)
    out = api.merge(bins, ns, dxs, torch.from_numpy(edges).cuda()).cpu().numpy()
    # oracle levels
    olv = []
    for (f, n_out), gb in zip([(1, n1), (4, 128), (16, 128)], bins):
        ed = ed1 if f == 1 else density.zoom_out(ed1, f, n_out, out_dtype="f16")
        r64 = ed.astype(np.float64)
        ob = scatter.forward(r64, ed1w.dx * f, edges)
        g = gb.cpu().numpy()
        assert np.array_equal(g[0].astype(np.int64), ob["count"])
        floor = 1e-6 * parseval_mean(r64)
        ok = (ob["count"] > 0) & (ob["mean"] >= floor)
        assert np.max(np.abs(g[4][ok] - ob["mean"][ok]) / ob["mean"][ok]) <= MEAN_RTOL
        olv.append({"n": n_out, "dx": ed1w.dx * f, "count": ob["count"], "mean": ob["mean"], "sem": ob["sem"],
                    "mean_q": ob["mean_q"]})
    want = omerge.merge_levels(olv, edges)
    assert np.array_equal(out[4].astype(np.int64), want["source"])
    assert np.array_equal(out[2].astype(np.int64), want["count"])
    ok = want["source"] >= 0
    assert np.nanmax(np.abs(out[0][ok] - want["mean"][ok]) / want["mean"][ok]) <= MEAN_RTOL
    assert set(np.unique(want["source"][ok])) == {0, 1, 2}
    # DC identity across levels: block sums keep the electron count
    tot = [float(e.double().sum().item()) for e, _, _ in lv]
    assert all(abs(t / tot[0] - 1) < 1e-3 for t in tot)


def test_three_level_merge_full_size():
    """The full three-level workload: ED-1 1024^3 FP16 (cube filling a 20 nm box), ED-2/ED-3
    4x/16x in 512^3 boxes, 1000 log bins 0.01-150 nm^-1, merged.  Invariants at full size:
    every window is used, means are finite and positive where the chosen level has voxels,
    counts of each level's bins are the lattice counts of its grid."""
    ed1w, zooms = inputs.cube_merge_levels()
    cell = torch.from_numpy(ed1w.cell).cuda()
    ed1 = api.build_density(ed1w.n, cell, ed1w.shape, out_dtype="f16")
    bins, ns, dxs, lv = _levels_gpu(ed1, ed1w.n, ed1w.dx, [(f, n) for f, n, _ in zooms], ed1w.edges)
    out = api.merge(bins, ns, dxs, torch.from_numpy(ed1w.edges).cuda()).cpu().numpy()
    src = out[4].astype(np.int64)
    assert set(np.unique(src[src >= 0])) == {0, 1, 2}
    used = src >= 0
    # ED-1 fills its periodic box, so it is an unbounded crystal: bins of its window without a
    # reciprocal-lattice point hold (numerically) zero intensity, and the cube's box sums vanish
    # on whole lattice planes at the coarser levels; no mean may be negative or NaN
    assert np.all(np.isfinite(out[0][used])) and np.all(out[0][used] >= 0)
    assert np.count_nonzero(out[0][used] > 0) > 0.9 * used.sum()
    # level counts: total voxels of the grid inside [e_0, e_B]
    for b, n, dx in zip(bins, ns, [ed1w.dx, ed1w.dx * 4, ed1w.dx * 16]):
        t = api.bin_thresholds(n, dx, ed1w.edges)
        k = np.arange(-(n // 2), n // 2)
        k2 = (k * k)
        # number of (kx, ky, kz) of the grid with t_0 <= k^2 < t_B: histogram kx^2 + ky^2 and kz^2
        h = np.bincount((k2[:, None] + k2[None, :]).ravel())
        hz = np.bincount(k2)
        cz = np.concatenate([[0], np.cumsum(hz)])
        s2 = np.arange(len(h))
        lo = np.clip(t[0] - s2, 0, len(hz))
        hi = np.clip(t[-1] - s2, 0, len(hz))
        tot = int((h * np.maximum(cz[hi] - cz[lo], 0)).sum())
        assert int(b[0].sum().item()) == tot
