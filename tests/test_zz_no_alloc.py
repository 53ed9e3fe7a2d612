"""ur_fft_intensity_noalloc: the forward without a caller workspace.

For callers that must not allocate device memory while they run (a fixed
memory budget set at start-up, a host program that owns all allocations):
the intermediate lives in the library's built-in scratch array.  This file
is collected last on purpose; one test repeats the check in a fresh Python
process, where the call is the first one of the library on the device.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2303_13435_gb300 import api, build, inputs

from _cases import MEAN_RTOL, oracle_density

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()
    torch.cuda.init()


def _plan_and_ed(n, diameter_nm):
    w = inputs.mof_workload(n=n, diameter_nm=diameter_nm, nbins=200)
    rho = oracle_density(w)
    nzp = np.flatnonzero(rho.any(axis=(1, 2)))
    z0, nz = int(nzp[0]), int(nzp[-1] - nzp[0] + 1)
    plan = api.Plan(n, w.dx, w.edges, z0=z0, nz=nz)
    ed = torch.from_numpy(np.ascontiguousarray(rho[z0:z0 + nz])).cuda()
    return plan, ed


def test_noalloc_matches_workspace_path_on_two_calls():
    plan, ed = _plan_and_ed(128, 4.0)
    assert plan.workspace_size(api.UR_WS_FORWARD) <= api.noalloc_scratch_bytes()
    ref = api.fft_intensity(plan, ed).cpu().numpy()
    bins = api.new_bins(plan)
    for _ in range(2):
        bins.fill_(float("nan"))  # whatever the caller's buffer held is replaced
        api.fft_intensity_noalloc(plan, ed, bins)
        got = bins.cpu().numpy()
        assert np.array_equal(got[0], ref[0])
        nz = ref[0] > 0
        assert np.allclose(got[4][nz], ref[4][nz], rtol=MEAN_RTOL, atol=0)
        assert np.allclose(got[1], ref[1], rtol=MEAN_RTOL, atol=0)


def test_noalloc_follows_a_larger_call_without_stale_data():
    # a second plan of another size reuses the same scratch array
    plan_a, ed_a = _plan_and_ed(128, 4.0)
    plan_b, ed_b = _plan_and_ed(64, 2.0)
    bins_a, bins_b = api.new_bins(plan_a), api.new_bins(plan_b)
    api.fft_intensity_noalloc(plan_a, ed_a, bins_a)
    api.fft_intensity_noalloc(plan_b, ed_b, bins_b)
    ref_b = api.fft_intensity(plan_b, ed_b).cpu().numpy()
    got_b = bins_b.cpu().numpy()
    nz = ref_b[0] > 0
    assert np.allclose(got_b[4][nz], ref_b[4][nz], rtol=MEAN_RTOL, atol=0)


def test_noalloc_rejects_plans_beyond_the_scratch_size():
    w = inputs.mof_workload(n=512, diameter_nm=10.0, nbins=64)
    plan = api.Plan(512, w.dx, w.edges, z0=133, nz=247)
    assert plan.workspace_size(api.UR_WS_FORWARD) > api.noalloc_scratch_bytes()
    ed = torch.zeros((1,), dtype=torch.float32, device="cuda")
    bins = api.new_bins(plan)
    with pytest.raises(api.UrError) as e:
        api.fft_intensity_noalloc(plan, ed, bins)
    assert e.value.status == 1 and "scratch" in str(e.value)


def test_noalloc_scratch_size_is_the_header_value():
    assert api.noalloc_scratch_bytes() == 64 << 20


def test_noalloc_injected_failure_returns_status_and_next_call_works():
    """The host-side fault site of the forward also guards this entry point."""
    plan, ed = _plan_and_ed(64, 2.0)
    bins = api.new_bins(plan)
    os.environ["UR_FAULT"] = "fft_intensity:1"
    api.lib().ur_fault_reset()
    try:
        with pytest.raises(api.UrError) as e:
            api.fft_intensity_noalloc(plan, ed, bins)
        assert e.value.status == 6
    finally:
        del os.environ["UR_FAULT"]
        api.lib().ur_fault_reset()
    ref = api.fft_intensity(plan, ed).cpu().numpy()
    got = api.fft_intensity_noalloc(plan, ed, bins).cpu().numpy()
    nz = ref[0] > 0
    assert np.allclose(got[4][nz], ref[4][nz], rtol=MEAN_RTOL, atol=0)


_FRESH = """
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np, torch
from paper_2303_13435_gb300 import api, inputs
from _cases import MEAN_RTOL, oracle_density
torch.cuda.init()
w = inputs.mof_workload(n=96, diameter_nm=3.0, nbins=120)
rho = oracle_density(w)
nzp = np.flatnonzero(rho.any(axis=(1, 2)))
z0, nz = int(nzp[0]), int(nzp[-1] - nzp[0] + 1)
plan = api.Plan(96, w.dx, w.edges, z0=z0, nz=nz)
ed = torch.from_numpy(np.ascontiguousarray(rho[z0:z0 + nz])).cuda()
bins = api.new_bins(plan)
got = [api.fft_intensity_noalloc(plan, ed, bins).cpu().numpy() for _ in range(2)]
ref = api.fft_intensity(plan, ed).cpu().numpy()
ok = ref[0] > 0
for g in got:
    assert np.array_equal(g[0], ref[0])
    assert np.allclose(g[4][ok], ref[4][ok], rtol=MEAN_RTOL, atol=0)
print("FRESH_OK")
"""


def test_noalloc_first_call_in_a_fresh_process():
    """The device address of the scratch array is looked up on the first no-allocation call
    of a process; run that first call (and a second) where no earlier one was made."""
    here = os.path.dirname(os.path.abspath(__file__))
    code = _FRESH.format(root=os.path.dirname(here), tests=here)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "FRESH_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
