"""Out-of-core forward: density in pinned host memory streamed to the device in slabs."""
import math
import os

import numpy as np
import pytest
import torch

from paper_2303_13435_gb300 import api, build, inputs

from _cases import compare_bins, oracle_density, oracle_forward

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()
    torch.cuda.init()


def _sphere(n, diam_vox, nbins=120):
    a = 2.6
    return inputs.mof_workload(n=n, diameter_nm=diam_vox * a / 64, nbins=nbins)


def _slab(rho):
    nzp = np.flatnonzero(rho.any(axis=(1, 2)))
    return int(nzp[0]), int(nzp[-1] - nzp[0] + 1)


@pytest.mark.parametrize("dtype,slab", [("f32", 7), ("f16", 5), ("f32", 1000)])
def test_streamed_host_ed_matches_device_path_and_oracle(dtype, slab):
    w = _sphere(256, 110)
    rho = oracle_density(w, out_dtype=dtype)
    z0, nz = _slab(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz, ed_dtype=dtype)
    plan.set_slab_planes(slab)
    host = torch.from_numpy(np.ascontiguousarray(rho[z0:z0 + nz])).pin_memory()
    got = api.fft_intensity(plan, host).cpu().numpy()
    ref = api.fft_intensity(plan, host.cuda()).cpu().numpy()
    # same kernels; the per-block FP32 bin sums are accumulated with shared-memory atomics
    # in a nondeterministic order (and the bins' shifts depend on block order), so two runs
    # agree to FP32 rounding of those sums: sum I to 2e-5, sum I^2 (its shifted squares
    # cancel more) to the SEM tolerance, sum |Q| (from the plan) exactly
    assert np.array_equal(got[0], ref[0])
    assert np.allclose(got[1], ref[1], rtol=2e-5, atol=0)
    assert np.allclose(got[2], ref[2], rtol=1e-3, atol=0)
    assert np.allclose(got[3], ref[3], rtol=1e-12, atol=0)
    r64 = rho.astype(np.float64)
    compare_bins(got, oracle_forward(r64, w.dx, w.edges), r64, f"host {dtype} slab {slab}")


def test_host_ed_must_be_pinned():
    w = _sphere(64, 30)
    rho = oracle_density(w)
    z0, nz = _slab(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    with pytest.raises(api.UrError) as e:
        api.fft_intensity(plan, torch.from_numpy(np.ascontiguousarray(rho[z0:z0 + nz])))
    assert e.value.status == 1


def test_injected_slab_failure_returns_status_and_next_call_works():
    """A host-side failure in the middle of the slab loop (UR_FAULT) is reported as
    UR_ERR_FAULT_INJECTED; nothing is faulted on the device and the next call succeeds."""
    w = _sphere(128, 60)
    rho = oracle_density(w)
    z0, nz = _slab(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    plan.set_slab_planes(8)
    host = torch.from_numpy(np.ascontiguousarray(rho[z0:z0 + nz])).pin_memory()
    os.environ["UR_FAULT"] = "host_slab:3"
    api.lib().ur_fault_reset()
    try:
        with pytest.raises(api.UrError) as e:
            api.fft_intensity(plan, host)
        assert e.value.status == 6
    finally:
        del os.environ["UR_FAULT"]
        api.lib().ur_fault_reset()
    torch.cuda.synchronize()
    got = api.fft_intensity(plan, host).cpu().numpy()
    r64 = rho.astype(np.float64)
    compare_bins(got, oracle_forward(r64, w.dx, w.edges), r64, "after fault")


def test_streamed_2048_cube_parseval_counts_and_device_path():
    """2048^3 grid, 32 nm sphere (788 planes, 13 GB of FP32 ED in pinned host memory):
    bins covering the whole grid sum to Parseval's total and count N^3 voxels, and
    the streamed result equals the device-resident one."""
    n = 2048
    w = _sphere(n, 788)
    dq = 2 * math.pi / (n * w.dx)
    edges = np.concatenate([[0.0], inputs.log_edges(0.99 * dq, math.sqrt(3) * math.pi / w.dx * 1.001, 400)])
    cell = torch.from_numpy(w.cell).cuda()
    rng = torch.tensor([2 ** 31 - 1, -1], dtype=torch.int32, device="cuda")
    # occupied slab from a density pass over the middle planes only
    z_lo = n // 2 - 400
    probe = api.build_density(n, cell, w.shape, z_begin=z_lo, z_count=800, nz_range=rng)
    del probe
    z0, z1 = rng.cpu().tolist()
    nz = z1 - z0 + 1
    host = torch.empty((nz, n, n), dtype=torch.float32, pin_memory=True)
    sumsq = 0.0
    step = 64
    for p0 in range(0, nz, step):
        cnt = min(step, nz - p0)
        d = api.build_density(n, cell, w.shape, z_begin=z0 + p0, z_count=cnt)
        sumsq += float((d.double() ** 2).sum().item())
        host[p0:p0 + cnt].copy_(d)
    del d
    plan = api.Plan(n, w.dx, edges, z0=z0, nz=nz)
    bins = api.fft_intensity(plan, host).cpu().numpy()
    assert int(bins[0].sum()) == n ** 3
    assert math.isclose(float(np.nansum(bins[1])), sumsq / float(n) ** 3, rel_tol=1e-5)
    dev = host.cuda()
    ref = api.fft_intensity(plan, dev).cpu().numpy()
    assert np.array_equal(bins[0], ref[0])
    # two runs of the same pass differ in the last bits (float32 block sums; each bin's shift is the
    # first value a block publishes, so block order decides it): over six device-resident runs up
    # to 3.1e-6 on sum I and 2.5e-5 on sum I^2.  Sum I is gated at the I(Q) tolerance, sum I^2 at
    # the SEM tolerance of the oracle comparisons; sum |Q| comes from the plan and must agree
    for f, tol in ((1, 1e-4), (2, 1e-3), (3, 1e-12)):
        bad = ~np.isclose(bins[f], ref[f], rtol=tol, atol=0)
        if bad.any():
            jb = int(np.flatnonzero(bad)[0])
            raise AssertionError(f"field {f}: {int(bad.sum())} bins differ, first {jb} (count {bins[0][jb]}): "
                                 f"{bins[f][jb]!r} vs {ref[f][jb]!r}")


def test_streamed_1024_sampled_k_against_direct_eq1():
    """The streamed path at 1024^3 (density in pinned host memory, small slabs) against
    Eq. 1 summed directly by the oracle at sampled frequencies (oracle.scatter.dft_at over
    the nonzero planes): F_out at 24 seeded k, including k = 0 and both Nyquist faces."""
    from oracle import scatter
    n = 1024
    w = _sphere(n, 500, nbins=64)
    rho = oracle_density(w)
    z0, nz = _slab(rho)
    plan = api.Plan(n, w.dx, w.edges, z0=z0, nz=nz)
    plan.set_slab_planes(37)
    host = torch.from_numpy(np.ascontiguousarray(rho[z0:z0 + nz])).pin_memory()
    H = n // 2 + 1
    F = torch.empty((n, n, H), dtype=torch.complex64, device="cuda")
    api.fft_intensity(plan, host, F_out=F)
    rng = np.random.default_rng(2048)
    ks = [(0, 0, 0), (512, 0, 0), (0, -512, 0), (0, 0, -512), (3, -7, 11)]
    ks += [(int(rng.integers(0, H)), int(rng.integers(-512, 512)), int(rng.integers(-512, 512))) for _ in range(19)]
    ks = np.array(ks, dtype=np.int64)
    want = scatter.dft_at(rho[z0:z0 + nz], ks, z_begin=z0)
    Fh = F.cpu().numpy()
    got = np.array([Fh[kz % n, ky % n, kx] for kx, ky, kz in ks])
    tol = 1e-4 * np.abs(want) + 1e-6 * abs(want[0])
    assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want) / tol)


@pytest.mark.parametrize("slab", [37, 256])
def test_slab_adjoint_equals_device_adjoint(slab):
    """Out-of-core adjoint (ur_backward_slabs, z pass recomputed per slab of output planes,
    dL/dm copied to pinned host memory) against the device-resident ur_backward on the same
    forward: same kernels, so dL/du and dL/dm agree to FP32 accumulation order; the forward
    ran from pinned host memory (streamed), so the whole out-of-core step is covered."""
    w = _sphere(256, 110, nbins=96)
    rho = oracle_density(w)
    z0, nz = _slab(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    plan.set_slab_planes(29)
    plan.set_adj_slab_planes(slab)
    cell = torch.from_numpy(w.cell).cuda()
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_HOST_SLABS | api.UR_WS_ADJ_SLABS)
    host = torch.from_numpy(np.ascontiguousarray(rho[z0:z0 + nz])).pin_memory()
    bins = api.fft_intensity(plan, host, ws=ws)
    m = bins[4]
    g = torch.where(torch.isfinite(m) & (m > 0), 1e-3 / torch.nan_to_num(m, nan=1.0).clamp(min=1e-300), 0.0)
    dm_host = torch.empty((w.n, w.n, w.n), dtype=torch.float32).pin_memory()
    dc_s, _ = api.backward_slabs(plan, g, bins, cell, w.shape, ws, dl_dmask_host=dm_host)
    api.sync_status()
    ws2 = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD)
    api.fft_intensity(plan, host.cuda(), ws=ws2)
    dc_d, dm_d = api.backward(plan, g, bins, cell, w.shape, ws2)
    torch.cuda.synchronize()
    a, b = dc_s.cpu().numpy(), dc_d.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
    a, b = dm_host.numpy(), dm_d.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


def test_slab_adjoint_2048_directional_derivative():
    """2048^3 streamed forward (density in pinned host memory) and the slab adjoint: for
    L = sum_j c_j mean_j the central difference of the streamed forward in the cell equals
    <dL/du, d> up to rounding (no N^3 inverse intermediate is ever held)."""
    n = 2048
    w = _sphere(n, 820, nbins=200)
    cell = torch.from_numpy(w.cell).cuda()
    rng = torch.tensor([2 ** 31 - 1, -1], dtype=torch.int32, device="cuda")
    z_lo = n // 2 - 420
    probe = api.build_density(n, cell, w.shape, z_begin=z_lo, z_count=840, nz_range=rng)
    del probe
    z0, z1 = rng.cpu().tolist()
    nz = z1 - z0 + 1
    plan = api.Plan(n, w.dx, w.edges, z0=z0, nz=nz)
    plan.set_adj_slab_planes(300)
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_HOST_SLABS | api.UR_WS_ADJ_SLABS)
    host = torch.empty((nz, n, n), dtype=torch.float32, pin_memory=True)

    def fill(cc):
        for p0 in range(0, nz, 64):
            cnt = min(64, nz - p0)
            host[p0:p0 + cnt].copy_(api.build_density(n, cc, w.shape, z_begin=z0 + p0, z_count=cnt))
        torch.cuda.synchronize()

    fill(cell)
    b0 = api.fft_intensity(plan, host, ws=ws)
    m0 = b0[4].double()
    c = torch.where(torch.isfinite(m0) & (m0 > 0), 1.0 / torch.nan_to_num(m0, nan=1.0).clamp(min=1e-300), 0.0)
    dcell, _ = api.backward_slabs(plan, c, b0, cell, w.shape, ws)
    api.sync_status()

    def loss(cc):
        fill(cc)
        b = api.fft_intensity(plan, host, ws=ws)
        return float((c * torch.nan_to_num(b[4].double(), nan=0.0)).sum().item())

    g = torch.Generator(device="cpu").manual_seed(2048)
    # quadratic loss: the central difference is exact, so a 10 % step keeps the forwards'
    # run-to-run rounding far below the difference
    d = (torch.randn(cell.shape, generator=g) * 0.1 * float(cell.abs().mean())).cuda()
    fd = (loss(cell + d) - loss(cell - d)) / 2.0
    an = float((dcell.double() * d.double()).sum().item())
    assert math.isclose(fd, an, rel_tol=2e-3), (fd, an)
