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
    # in a nondeterministic order, so two runs agree to FP32 rounding of those sums
    assert np.array_equal(got[0], ref[0])
    assert np.allclose(got[1:4], ref[1:4], rtol=2e-5, atol=0)
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
    assert np.allclose(bins[1:4], ref[1:4], rtol=2e-5, atol=0)
