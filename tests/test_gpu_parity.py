"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Sizes span several FFT tiles and ragged tails; grid edges cover radices
2, 3, 5 and 7.  Tolerances are stated in tests/_cases.py.
"""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint, density, merge as omerge, scatter
from paper_2303_13435_gb300 import api, build, inputs

from _cases import (GRAD_RTOL, compare_bins, normwise, oracle_density, oracle_forward, oracle_grads,
                    oracle_parity_counts)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()
    torch.cuda.init()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mof(n, diameter_vox, nbins=96, seed=0, ucell=64, a_nm=2.6, kind=inputs.SHAPE_SPHERE, rot_seed=None,
        origin=(0, 0, 0)):
    w = inputs.mof_workload(n=n, diameter_nm=diameter_vox * a_nm / ucell, nbins=nbins, seed=seed, ucell=ucell,
                            a_nm=a_nm)
    if kind != inputs.SHAPE_SPHERE or rot_seed is not None:
        rot = inputs.random_rotation(inputs.SplitMix64(rot_seed or 1))
        c = float(n // 2)
        size = 0.5 * diameter_vox if kind != inputs.SHAPE_CUBE else 0.5 * diameter_vox / math.sqrt(3)
        w.shape = inputs.Shape(kind, (c, c, c), float(np.float32(size)), rot)
    w.origin = origin
    return w


def z_range(rho):
    lo, hi = density.nonzero_plane_range(rho)
    return lo, hi - lo + 1


# ---------------------------------------------------------------------------
# ED generation: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["sc64", "mof96_origin", "cube_rot", "octa_rot", "all"])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_density_bit_exact(case, dtype):
    if case == "sc64":
        w = inputs.sc64_workload()
    elif case == "mof96_origin":
        w = mof(96, 60, origin=(3, 5, 7))
    elif case == "cube_rot":
        w = mof(100, 70, kind=inputs.SHAPE_CUBE, rot_seed=5)
    elif case == "octa_rot":
        w = mof(98, 80, kind=inputs.SHAPE_OCTAHEDRON, rot_seed=9)
    else:
        w = mof(64, 10)
        w.shape = inputs.Shape(inputs.SHAPE_ALL)
    want = oracle_density(w, out_dtype=dtype)
    rng = torch.tensor([2 ** 31 - 1, -1], dtype=torch.int32, device="cuda")
    got = api.build_density(w.n, dev(w.cell), w.shape, origin=w.origin, out_dtype=dtype, nz_range=rng)
    torch.cuda.synchronize()
    g = got.cpu().numpy()
    assert g.tobytes() == want.tobytes()
    lo, hi = density.nonzero_plane_range(want)
    assert rng.cpu().tolist() == [lo, hi]


@pytest.mark.parametrize("n,kind,dtype", [(96, inputs.SHAPE_SPHERE, "f32"), (128, inputs.SHAPE_CUBE, "f16"),
                                          (100, inputs.SHAPE_OCTAHEDRON, "f32")])
def test_rotated_lattice_density_bit_exact_and_fused_forward(n, kind, dtype):
    """Sec. 2.3 rotated sampling of the cell: ED bit-exact against the float32 oracle (same
    operation order), and the fused transform of that density against the oracle bins."""
    w = mof(n, 0.55 * n, kind=kind, rot_seed=3)
    c = float(n // 2)
    lat = (inputs.random_rotation(inputs.SplitMix64(11)), (c + 0.37, c - 1.21, c + 2.5))
    s = w.shape
    want = density.tile_mask_density(n, w.cell, s.kind, s.center, s.size, s.rot, lattice=lat, out_dtype=dtype)
    rng = torch.tensor([2 ** 31 - 1, -1], dtype=torch.int32, device="cuda")
    got = api.build_density(n, dev(w.cell), s, out_dtype=dtype, nz_range=rng, lattice=lat)
    torch.cuda.synchronize()
    assert got.cpu().numpy().tobytes() == want.tobytes()
    lo, hi = density.nonzero_plane_range(want)
    assert rng.cpu().tolist() == [lo, hi]
    if dtype == "f32":
        plan = api.Plan(n, w.dx, w.edges, z0=lo, nz=hi - lo + 1)
        gb = api.fft_intensity_tiled(plan, dev(w.cell), s, lattice=lat).cpu().numpy()
        r64 = want.astype(np.float64)
        compare_bins(gb, oracle_forward(r64, w.dx, w.edges), r64, f"lattice{n}")


def test_density_weights_and_plane_subrange():
    w = mof(64, 40)
    weights = np.random.default_rng(3).random((64, 64, 64)).astype(np.float32)
    w.shape = inputs.Shape(inputs.SHAPE_WEIGHTS)
    want = oracle_density(w, z_begin=9, z_count=23, weights=weights)
    got = api.build_density(64, dev(w.cell), w.shape, weights=dev(weights), z_begin=9, z_count=23)
    assert got.cpu().numpy().tobytes() == want.tobytes()


@pytest.mark.parametrize("f,n_out,src_dtype,out_dtype", [(4, 32, "f16", "f16"), (16, 16, "f16", "f16"),
                                                          (2, 48, "f16", "f32"), (4, 20, "f32", "f32")])
def test_zoom_block_sums(f, n_out, src_dtype, out_dtype):
    w = mof(64, 50)
    ed1 = oracle_density(w, out_dtype=src_dtype)
    want = density.zoom_out(ed1, f, n_out, out_dtype=out_dtype)
    got = api.zoom_density(dev(ed1), f, n_out, out_dtype=out_dtype).cpu().numpy()
    if src_dtype == "f16":
        assert got.tobytes() == want.tobytes()
    else:  # float64 sums in another order, one rounding to float32
        assert np.allclose(got, want, rtol=2 ** -23, atol=0)


# ---------------------------------------------------------------------------
# Forward: transform, |F|^2, Q bins
# ---------------------------------------------------------------------------
def gpu_forward(w, rho, F=False, dtype="f32"):
    z0, nz = z_range(rho) if np.any(rho) else (0, 1)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz, ed_dtype=dtype)
    ed = dev(rho[z0:z0 + nz])
    Fo = torch.empty((w.n, w.n, w.n // 2 + 1, 2), dtype=torch.float32, device="cuda") if F else None
    bins = api.fft_intensity(plan, ed, F_out=Fo)
    torch.cuda.synchronize()
    return plan, bins.cpu().numpy(), (Fo.cpu().numpy() if F else None)


@pytest.mark.parametrize("case", ["sc64", "mof96", "mof98", "mof100", "mof120_cube", "mof128_small", "mof160",
                                  "mof250", "mof270", "mof378"])
def test_forward_bins_match_oracle(case):
    if case == "sc64":
        w = inputs.sc64_workload()
    elif case == "mof120_cube":
        w = mof(120, 56, kind=inputs.SHAPE_CUBE, rot_seed=2)
    elif case == "mof128_small":
        w = mof(128, 11)
    else:
        n = int(case[3:])
        w = mof(n, int(n * 0.45))
    rho = oracle_density(w)
    _, gb, _ = gpu_forward(w, rho)
    ob = oracle_forward(rho, w.dx, w.edges)
    rep = compare_bins(gb, ob, rho.astype(np.float64), case)
    print(case, rep)


def test_forward_full_box_single_plane_and_zero_density():
    w = mof(64, 30)
    rho = oracle_density(w)
    # the whole box as the slab (no skipped planes)
    plan = api.Plan(64, w.dx, w.edges, z0=0, nz=64)
    gb = api.fft_intensity(plan, dev(rho)).cpu().numpy()
    compare_bins(gb, oracle_forward(rho, w.dx, w.edges), rho.astype(np.float64), "full box")
    # a single nonzero plane
    one = np.zeros_like(rho)
    one[17] = rho[32]
    plan = api.Plan(64, w.dx, w.edges, z0=17, nz=1)
    gb = api.fft_intensity(plan, dev(one[17:18])).cpu().numpy()
    compare_bins(gb, oracle_forward(one, w.dx, w.edges), one.astype(np.float64), "one plane")
    # zero density: zero means, exact counts
    zero = np.zeros((5, 64, 64), dtype=np.float32)
    plan = api.Plan(64, w.dx, w.edges, z0=30, nz=5)
    gb = api.fft_intensity(plan, dev(zero)).cpu().numpy()
    ob = oracle_forward(np.zeros((64, 64, 64)), w.dx, w.edges)
    assert np.array_equal(gb[0].astype(np.int64), ob["count"])
    nz = ob["count"] > 0
    assert np.all(gb[4][nz] == 0.0) and np.all(gb[1] == 0.0)


def test_F_out_matches_eq1():
    w = mof(96, 44)
    rho = oracle_density(w)
    _, _, F = gpu_forward(w, rho, F=True)
    Fo = scatter.dft3(rho)[:, :, : w.n // 2 + 1]
    Fg = F[..., 0] + 1j * F[..., 1]
    err = np.abs(Fg - Fo).max() / np.abs(Fo).max()
    assert err < 2e-6, err


def test_log_mse_grad_matches_oracle():
    rng = np.random.default_rng(11)
    nb = 700
    bins = np.zeros((api.BIN_FIELDS, nb))
    bins[4] = rng.uniform(1e-8, 1e-2, nb)
    bins[4][[5, 99, 300]] = np.nan
    bins[4][[7, 400]] = 0.0
    bins[4][450] = -1.0
    target = rng.uniform(1e-8, 1e-2, nb)
    L, g = adjoint.loss_log_mse(bins[4], target)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    got = api.log_mse_grad(dev(bins), dev(target), loss=loss).cpu().numpy()
    assert np.allclose(got, g, rtol=1e-12, atol=0)
    assert math.isclose(float(loss.item()), L, rel_tol=1e-12)


def test_negative_origin_is_rejected_by_every_entry_point():
    w = mof(64, 30)
    rho = oracle_density(w)
    z0, nz = z_range(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD)
    cell = dev(w.cell)
    bins = api.fft_intensity_tiled(plan, cell, w.shape, ws=ws)
    for call in (lambda: api.build_density(w.n, cell, w.shape, origin=(0, -1, 0)),
                 lambda: api.fft_intensity_tiled(plan, cell, w.shape, origin=(0, 0, -3), ws=ws),
                 lambda: api.backward(plan, torch.zeros(plan.nbins, dtype=torch.float64, device="cuda"), bins, cell,
                                      w.shape, ws, origin=(-2, 0, 0))):
        with pytest.raises(api.UrError) as e:
            call()
        assert e.value.status == 1 and "origin" in str(e.value)


def test_bounded_device_wait_reports_timeout_and_context_survives():
    """A device-side wait that nothing completes gives up after its limit (here ~2^24 SM
    cycles), records the library's error word and returns; ur_sync_status reports
    UR_ERR_TIMEOUT once, and the next work runs normally."""
    s = torch.cuda.current_stream()
    assert api.lib().ur_selftest_wait_timeout(s.cuda_stream) == 0
    with pytest.raises(api.UrError) as e:
        api.sync_status()
    assert e.value.status == 4
    api.sync_status()   # the word was cleared
    w = inputs.sc64_workload()
    rho = oracle_density(w)
    z0, nz = z_range(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    got = api.fft_intensity(plan, dev(rho[z0:z0 + nz])).cpu().numpy()
    r64 = rho.astype(np.float64)
    compare_bins(got, oracle_forward(r64, w.dx, w.edges), r64, "after timeout")


def test_sync_status_after_queued_work():
    w = mof(64, 30)
    rho = oracle_density(w)
    z0, nz = z_range(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    bins = api.fft_intensity(plan, dev(rho[z0:z0 + nz]))
    api.sync_status()  # raises on a device-side failure
    assert int(bins[0].sum().item()) > 0


def test_fp16_ed_forward():
    w = mof(128, 60)
    rho16 = oracle_density(w, out_dtype="f16")
    z0, nz = z_range(rho16)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz, ed_dtype="f16")
    gb = api.fft_intensity(plan, dev(rho16[z0:z0 + nz])).cpu().numpy()
    r64 = rho16.astype(np.float64)
    compare_bins(gb, oracle_forward(r64, w.dx, w.edges), r64, "fp16 ED")


def test_plan_thresholds_equal_host_table():
    w = inputs.sc64_workload()
    plan = api.Plan(w.n, w.dx, w.edges)
    assert np.array_equal(plan.thresholds(), api.bin_thresholds(w.n, w.dx, w.edges))


def test_bin_q_standalone():
    w = mof(64, 30, nbins=40)
    rho = oracle_density(w)
    ob = oracle_forward(rho, w.dx, w.edges)
    Ihalf = ob["I"][:, :, : w.n // 2 + 1].astype(np.float32)
    plan = api.Plan(w.n, w.dx, w.edges)
    gb = api.bin_q(plan, dev(Ihalf)).cpu().numpy()
    # the same float32 intensities binned by the oracle (mirrored voxels may differ by one ulp)
    ob32 = scatter.bin_intensity(ob["I"].astype(np.float32).astype(np.float64), w.n, w.dx, w.edges)
    assert np.array_equal(gb[0].astype(np.int64), ob32["count"])
    nz = ob32["count"] > 0
    assert np.allclose(gb[4][nz], ob32["mean"][nz], rtol=1e-6, atol=0)


def test_merge_matches_oracle():
    edges = inputs.log_edges(0.05, 20.0, 60)
    levels = []
    rng = np.random.default_rng(1)
    for n, dx in [(32, 0.4), (32, 0.8), (64, 0.1)]:
        cnt = rng.integers(0, 50, 60).astype(np.int64)
        mean = rng.random(60)
        sem = rng.random(60) * 0.1
        mq = rng.random(60) * 10
        levels.append({"n": n, "dx": dx, "count": cnt, "mean": np.where(cnt > 0, mean, np.nan), "sem": sem, "mean_q": mq})
    want = omerge.merge_levels(levels, edges)
    dev_bins = []
    for lv in levels:
        b = np.zeros((6, 60))
        b[0] = lv["count"]
        b[3] = lv["mean_q"] * lv["count"]
        b[4] = lv["mean"]
        b[5] = lv["sem"]
        dev_bins.append(dev(b))
    out = api.merge(dev_bins, [lv["n"] for lv in levels], [lv["dx"] for lv in levels], dev(edges))
    o = out.cpu().numpy()
    assert np.array_equal(o[4].astype(np.int64), want["source"])
    assert np.array_equal(o[2].astype(np.int64), want["count"])
    ok = want["source"] >= 0
    assert np.array_equal(o[0][ok], want["mean"][ok])
    assert np.array_equal(o[1][ok], want["sem"][ok])
    assert np.allclose(o[3][ok], want["mean_q"][ok], rtol=1e-15)
    assert np.all(np.isnan(o[0][~ok]))
    # uncertainty-weighted combination where levels overlap (Sec. 2.7)
    want = omerge.merge_levels(levels, edges, mode="invvar")
    o = api.merge(dev_bins, [lv["n"] for lv in levels], [lv["dx"] for lv in levels], dev(edges),
                  mode="invvar").cpu().numpy()
    assert np.array_equal(o[4].astype(np.int64), want["source"])
    assert np.array_equal(o[2].astype(np.int64), want["count"])
    ok = want["source"] >= 0
    assert np.allclose(o[0][ok], want["mean"][ok], rtol=1e-13, atol=0)
    assert np.allclose(o[1][ok], want["sem"][ok], rtol=1e-13, atol=0)
    assert np.allclose(o[3][ok], want["mean_q"][ok], rtol=1e-13)
    assert np.all(np.isnan(o[0][~ok]))


def _oracle_counts(n, dx, edges):
    """n_j of the oracle's binning (float64 |Q| of every integer k of the grid), plane by plane."""
    nb = len(edges) - 1
    cnt = np.zeros(nb, dtype=np.int64)
    for kz in scatter.signed_freq(n):
        j = scatter.bin_of_q(scatter.q_of_k2(scatter._plane_k2(n, int(kz)), n, dx), edges).ravel()
        cnt += np.bincount(j[j >= 0], minlength=nb)
    return cnt


@pytest.mark.parametrize("n,nbins,tma", [(512, 512, False), (512, 512, True), (256, 200, False), (256, 200, True),
                                         (126, 96, False), (100, 80, False)])
def test_single_voxel_bins_every_voxel_exactly(n, nbins, tma):
    """The data pass's bin index of every voxel, not the plan's geometry: a unit voxel at the
    origin transforms to F~ = 1 at every k (exactly, in FP32), so the binned sum of I is the
    number of voxels the fused z-pass walk put in each bin.  Power-of-two grids (compile-time
    kernels, and the TMA engine) make every term a power of two and the sum exact; the runtime-radix grids carry
    one FP32 rounding of 1/N^3 per term and at most 1e-6 relative error per bin, below half a
    voxel for these counts."""
    dx = 0.04
    edges = inputs.log_edges(2 * math.pi / (n * dx), math.pi / dx, nbins)
    ed = torch.zeros((1, n, n), dtype=torch.float32, device="cuda")
    ed[0, 0, 0] = 1.0
    plan = api.Plan(n, dx, edges, z0=0, nz=1)
    if tma:
        plan.set_tma_zpass(True)
        assert plan.tma_zpass()
    gb = api.fft_intensity(plan, ed).cpu().numpy()
    want = _oracle_counts(n, dx, edges)
    assert np.array_equal(gb[0].astype(np.int64), want)
    per_voxel = float(np.float32(1.0 / n ** 3)) * n ** 3   # the kernel's FP32 scale times N^3
    voxels = gb[1] * float(n) ** 6 / per_voxel
    if n & (n - 1) == 0:
        assert np.array_equal(voxels, want.astype(np.float64))
    else:
        assert np.max(np.abs(voxels - want)) < 0.25
        assert np.array_equal(np.rint(voxels).astype(np.int64), want)


@pytest.mark.parametrize("n,nbins,tma", [(512, 512, False), (512, 512, True), (256, 200, False), (256, 200, True),
                                         (2048, 1000, False), (4096, 2000, False), (126, 96, False)])
def test_two_voxel_bins_count_every_voxel(n, nbins, tma):
    """The data pass's bin of every voxel where the per-bin statistics cannot hide it: unit voxels
    at x = 0 and x = N/2 give F~ = 1 + (-1)^kx, so |F~|^2 is 4 on the voxels with kx even and 0 on
    the others.  A shifted mean (reading of the shifted sums: mean = K + sum(I - K)/n, n from the
    plan) equals the true mean only if the walk put exactly the right voxels of each bin into its
    sums; N^6 times the binned sum of I must be 4 times the oracle's count of even-kx voxels in the
    bin.  Power-of-two grids carry every term exactly; the finalize divides once by n (relative
    1e-12 here).  126 runs the runtime-radix engine (FP32 rounding of 1/N^3 per term: 1e-6)."""
    dx = 0.04
    edges = inputs.log_edges(2 * math.pi / (n * dx), math.pi / dx, nbins)
    ed = torch.zeros((1, n, n), dtype=torch.float32, device="cuda")
    ed[0, 0, 0] = 1.0
    ed[0, 0, n // 2] = 1.0
    plan = api.Plan(n, dx, edges, z0=0, nz=1)
    if tma:
        plan.set_tma_zpass(True)
        assert plan.tma_zpass()
    gb = api.fft_intensity(plan, ed).cpu().numpy()
    even, total = oracle_parity_counts(n, dx, edges)
    assert np.array_equal(gb[0].astype(np.int64), total)
    per_voxel = float(np.float32(1.0 / n ** 3)) * n ** 3
    got = gb[1] * float(n) ** 6 / per_voxel
    want = 4.0 * even
    filled = total > 0
    rel = np.abs(got[filled] - want[filled]) / np.maximum(want[filled], 1.0)
    assert float(rel.max()) <= (1e-12 if n & (n - 1) == 0 else 1e-6), float(rel.max())


# ---------------------------------------------------------------------------
# Adjoint
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["recompute", "F_given", "weights_origin"])
def test_backward_matches_oracle_gradient(mode):
    if mode == "weights_origin":
        w = mof(64, 40, ucell=16, a_nm=0.65, origin=(2, 7, 5))
        weights = np.random.default_rng(4).random((64, 64, 64)).astype(np.float32)
        weights[:10] = 0
        weights[54:] = 0
        w.shape = inputs.Shape(inputs.SHAPE_WEIGHTS)
    else:
        w = inputs.sc64_workload()
        weights = None
    rho = oracle_density(w, weights=weights)
    z0, nz = z_range(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD)
    Fo = torch.empty((w.n, w.n, w.n // 2 + 1, 2), device="cuda") if mode == "F_given" else None
    bins = api.fft_intensity(plan, dev(rho[z0:z0 + nz]), ws=ws, F_out=Fo)
    # loss: log-MSE against the closed-form sphere curve of the same electron count
    gb = bins.cpu().numpy()
    ne = float(rho.astype(np.float64).sum())
    target = inputs.sphere_target_curve(gb[3] / np.maximum(gb[0], 1), 1.0, ne) / w.n ** 6 + 1e-30
    L, g = adjoint.loss_log_mse(gb[4], target)
    dcell, dmask = api.backward(plan, dev(g), bins, dev(w.cell), w.shape, ws, origin=w.origin,
                                weights=dev(weights) if weights is not None else None, F=Fo)
    torch.cuda.synchronize()
    mask = density.mask_values(w.n, w.shape.kind, w.shape.center, w.shape.size, w.shape.rot, weights)
    ob_count = oracle_forward(rho, w.dx, w.edges)["count"]
    gu, gm = oracle_grads(rho.astype(np.float64), w.cell.astype(np.float64), mask, w.dx, w.edges, g, ob_count,
                          w.origin)
    eu = normwise(dcell.cpu().numpy(), gu)
    em = normwise(dmask.cpu().numpy(), gm)
    print(mode, "dL/du", eu, "dL/dm", em)
    assert eu <= GRAD_RTOL and em <= GRAD_RTOL


# ---------------------------------------------------------------------------
# Fused density + transform (density generated inside the plane pass)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["sc64", "mof128_cube_origin", "mof256_sphere", "mof96_generic", "mof128_weights"])
def test_tiled_forward_matches_oracle(case):
    weights = None
    if case == "sc64":
        w = inputs.sc64_workload()
    elif case == "mof128_cube_origin":
        w = mof(128, 70, kind=inputs.SHAPE_CUBE, rot_seed=4, origin=(5, 1, 9))
    elif case == "mof256_sphere":
        w = mof(256, 120)
    elif case == "mof96_generic":
        w = mof(96, 50, kind=inputs.SHAPE_OCTAHEDRON, rot_seed=8)
    else:
        w = mof(128, 60)
        weights = np.random.default_rng(6).random((128, 128, 128)).astype(np.float32)
        weights[:20] = 0
        weights[100:] = 0
        w.shape = inputs.Shape(inputs.SHAPE_WEIGHTS)
    rho = oracle_density(w, weights=weights)
    z0, nz = z_range(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    gb = api.fft_intensity_tiled(plan, dev(w.cell), w.shape, origin=w.origin,
                                 weights=dev(weights) if weights is not None else None).cpu().numpy()
    rep = compare_bins(gb, oracle_forward(rho, w.dx, w.edges), rho.astype(np.float64), case)
    # the stored-ED path gives the same bins (the same intermediate; two binning runs differ only
    # by the order of their float32 block sums and of the bins' first published shift: measured
    # up to 3e-6 of a mean at 2048^3, far less at these sizes)
    gb2 = api.fft_intensity(plan, dev(rho[z0:z0 + nz])).cpu().numpy()
    assert np.allclose(gb2[4], gb[4], rtol=1e-5, equal_nan=True)
    print(case, rep)


def test_n1024_sampled_F_parseval_and_counts():
    """Largest power-of-two size: sampled F against the direct Eq. 1 sum, Parseval over
    bins that cover the whole grid, and exact bin counts."""
    w = mof(1024, 180)
    n = w.n
    edges = inputs.log_edges(2 * math.pi / (n * w.dx) * 0.99, math.sqrt(3) * math.pi / w.dx * 1.001, 300)
    edges = np.concatenate([[0.0], edges])
    rho = oracle_density(w)
    z0, nz = z_range(rho)
    plan = api.Plan(n, w.dx, edges, z0=z0, nz=nz)
    F = torch.empty((n, n, n // 2 + 1, 2), dtype=torch.float32, device="cuda")
    gb = api.fft_intensity_tiled(plan, dev(w.cell), w.shape, F_out=F).cpu().numpy()
    rng = np.random.default_rng(0)
    ks = np.stack([rng.integers(0, n // 2 + 1, 24), rng.integers(-n // 2, n // 2, 24), rng.integers(-n // 2, n // 2, 24)], 1)
    ks[0] = (0, 0, 0)
    ks[1] = (3, -2, 1)
    want = scatter.dft_at(rho[z0:z0 + nz], ks, z_begin=z0)
    got = F[ks[:, 2] % n, ks[:, 1] % n, ks[:, 0]].cpu().numpy()
    got = got[:, 0] + 1j * got[:, 1]
    scale = abs(want[0])
    assert np.max(np.abs(got - want)) <= 1e-5 * scale
    r64 = rho[z0:z0 + nz].astype(np.float64)
    parseval = float((r64 ** 2).sum()) / float(n) ** 3  # Parseval under Eq. 1: sum_k |F_k|^2 = sum rho^2 / N^3
    tot = float(np.nansum(gb[1]))
    assert math.isclose(tot, parseval, rel_tol=1e-5)
    # the edges cover every |Q| of the grid, so the counts add up to N^3 exactly
    assert int(gb[0].sum()) == n ** 3


@pytest.mark.parametrize("case", ["mof128_weights_origin", "mof256_chunks", "mof256_chunk7", "sc64_tiled"])
def test_backward_fast_path(case):
    weights = None
    if case == "mof128_weights_origin":
        w = mof(128, 60, ucell=32, a_nm=1.3, origin=(3, 0, 7))
        weights = np.random.default_rng(7).random((128, 128, 128)).astype(np.float32)
        weights[:30] = 0
        weights[98:] = 0
        w.shape = inputs.Shape(inputs.SHAPE_WEIGHTS)
    elif case in ("mof256_chunks", "mof256_chunk7"):
        w = mof(256, 110, kind=inputs.SHAPE_CUBE, rot_seed=3)
    else:
        w = inputs.sc64_workload()
    rho = oracle_density(w, weights=weights)
    z0, nz = z_range(rho)
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    if case == "mof256_chunk7":
        # 7-plane chunks: the plane pass and the adjoint's chunk loop end on a ragged chunk
        plan.set_chunk_planes(7)
        assert plan.chunk_planes() == 7 and nz % 7 != 0 and 256 % 7 != 0
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD)
    wd = dev(weights) if weights is not None else None
    bins = api.fft_intensity_tiled(plan, dev(w.cell), w.shape, origin=w.origin, weights=wd, ws=ws)
    gb = bins.cpu().numpy()
    if case == "mof256_chunk7":
        r64 = rho.astype(np.float64)
        compare_bins(gb, oracle_forward(r64, w.dx, w.edges), r64, case)
    g = np.where(gb[0] > 0, 1.0 / np.maximum(np.nan_to_num(gb[4]), 1e-300), 0.0) * 1e-3
    dcell, dmask = api.backward(plan, dev(g), bins, dev(w.cell), w.shape, ws, origin=w.origin, weights=wd)
    mask = density.mask_values(w.n, w.shape.kind, w.shape.center, w.shape.size, w.shape.rot, weights)
    ob_count = oracle_forward(rho, w.dx, w.edges)["count"]
    gu, gm = oracle_grads(rho.astype(np.float64), w.cell.astype(np.float64), mask, w.dx, w.edges, g, ob_count,
                          w.origin)
    eu = normwise(dcell.cpu().numpy(), gu)
    em = normwise(dmask.cpu().numpy(), gm)
    print(case, "dL/du", eu, "dL/dm", em)
    assert eu <= GRAD_RTOL and em <= GRAD_RTOL


@pytest.mark.parametrize("keep_f,tma", [(True, False), (False, False), (False, True)])
def test_mof512_full_size_forward_and_adjoint(keep_f, tma):
    """The 512^3 workload of the benchmark against the FP64 oracle: fused tiled forward,
    then the adjoint from the kept half spectrum F or recomputing F along z from the
    plane-pass intermediate (the benchmark's launch configuration); the forward on both
    z-pass engines."""
    w = inputs.mof_workload(n=512, diameter_nm=10.0, nbins=512)
    rho = oracle_density(w)
    z0, nz = z_range(rho)
    assert nz == 247
    plan = api.Plan(w.n, w.dx, w.edges, z0=z0, nz=nz)
    if tma:
        plan.set_tma_zpass(True)
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD)
    Fh = torch.empty((512, 512, 257, 2), device="cuda") if keep_f else None
    bins = api.fft_intensity_tiled(plan, dev(w.cell), w.shape, ws=ws, F_out=Fh)
    gb = bins.cpu().numpy()
    r64 = rho.astype(np.float64)
    ob = oracle_forward(r64, w.dx, w.edges)
    rep = compare_bins(gb, ob, r64, "mof512")
    print("mof512 forward", rep)
    g = np.where(gb[0] > 0, 1.0 / np.maximum(np.nan_to_num(gb[4]), 1e-300), 0.0) * 1e-3
    dcell, dmask = api.backward(plan, dev(g), bins, dev(w.cell), w.shape, ws, F=Fh)
    mask = density.mask_values(w.n, w.shape.kind, w.shape.center, w.shape.size, w.shape.rot)
    gu, gm = oracle_grads(r64, w.cell.astype(np.float64), mask, w.dx, w.edges, g, ob["count"])
    eu = normwise(dcell.cpu().numpy(), gu)
    em = normwise(dmask.cpu().numpy(), gm)
    print("mof512 adjoint", eu, em)
    assert eu <= GRAD_RTOL and em <= GRAD_RTOL


@pytest.mark.parametrize("n,keep_f", [(1024, False), (2048, True)])
def test_large_grid_adjoint_directional_derivative(n, keep_f):
    """Grids beyond the oracle's reach (1024^3: 512-thread column blocks and block-barrier
    rows; 2048^3: 1024-thread column blocks): for L = sum_j c_j mean_j, a quadratic in the
    cell and in the mask weights, the central difference (L(p + d) - L(p - d)) / 2 equals
    <dL/dp, d> up to rounding.  1024^3 runs with random per-voxel weights (dL/du and dL/dm),
    2048^3 with the sphere (dL/du, F kept)."""
    w = mof(n, 0.4 * n, nbins=200)
    cell = dev(w.cell)
    half = int(0.2 * n) + 2
    z0, nz = n // 2 - half, 2 * half
    g = torch.Generator(device="cpu").manual_seed(n)
    weights = None
    shape = w.shape
    if n <= 1024:
        wt = torch.zeros((n, n, n), dtype=torch.float32)
        wt[z0:z0 + nz] = torch.rand((nz, n, n), generator=g)
        weights = wt.cuda()
        shape = inputs.Shape(inputs.SHAPE_WEIGHTS)
    plan = api.Plan(n, w.dx, w.edges, z0=z0, nz=nz)
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD)
    Fh = torch.empty((n, n, n // 2 + 1, 2), device="cuda") if keep_f else None
    b0 = api.fft_intensity_tiled(plan, cell, shape, weights=weights, ws=ws, F_out=Fh)
    m0 = b0[4].double()
    c = torch.where(torch.isfinite(m0) & (m0 > 0), 1.0 / torch.nan_to_num(m0, nan=1.0).clamp(min=1e-300), 0.0)
    dcell, dmask = api.backward(plan, c, b0, cell, shape, ws, weights=weights, F=Fh, want_mask=weights is not None)

    def loss(cc, wts):
        b = api.fft_intensity_tiled(plan, cc, shape, weights=wts, ws=ws)
        return float((c * torch.nan_to_num(b[4].double(), nan=0.0)).sum().item())

    # L is quadratic in the cell and in the weights, so the central difference has no truncation
    # error and the step can be large: a 10 % step keeps the forwards' run-to-run rounding (about
    # 3e-6 of each bin mean) far below the difference itself
    d = (torch.randn(cell.shape, generator=g) * 0.1 * float(cell.abs().mean())).cuda()
    fd = (loss(cell + d, weights) - loss(cell - d, weights)) / 2.0
    an = float((dcell.double() * d.double()).sum().item())
    print(n, "dL/du", fd, an)
    assert math.isclose(fd, an, rel_tol=2e-3), (fd, an)
    if weights is not None:
        e = torch.zeros_like(weights)
        e[z0:z0 + nz] = (torch.randn((nz, n, n), generator=g) * 0.1).cuda()
        fdm = (loss(cell, weights + e) - loss(cell, weights - e)) / 2.0
        anm = float((dmask.double() * e.double()).sum().item())
        print(n, "dL/dm", fdm, anm)
        assert math.isclose(fdm, anm, rel_tol=2e-3), (fdm, anm)


@pytest.mark.parametrize("n,rot_seed,bw,nl", [(64, None, 0.0, 1), (96, 4, 0.08, 4)])
def test_ewald_image_matches_oracle(n, rot_seed, bw, nl):
    """Sec. 2.5 Ewald-sphere extraction from the GPU's half spectrum against the oracle's
    image of its own FP64 transform.  Gate per pixel: 1e-4 of the largest intensity among
    the pixel's interpolation corners (FP32 geometry and FP32 spectrum), plus 1e-9 of I(0)."""
    from oracle import ewald
    w = mof(n, 0.45 * n, nbins=32)
    rho = oracle_density(w)
    z0, nz = z_range(rho)
    plan = api.Plan(n, w.dx, w.edges, z0=z0, nz=nz)
    H = n // 2 + 1
    F = torch.empty((n, n, H), dtype=torch.complex64, device="cuda")
    api.fft_intensity(plan, dev(rho[z0:z0 + nz]), F_out=F)
    det = {"nx": 61, "ny": 47, "pixel_m": 0.004, "distance_m": 0.3, "beam": (30.0, 20.5), "wavelength_nm": 0.154,
           "bandwidth": bw, "nlambda": nl,
           "rot": np.eye(3) if rot_seed is None else inputs.random_rotation(inputs.SplitMix64(rot_seed))}
    got = api.ewald_image(plan, F, det).cpu().numpy().astype(np.float64)
    Fo = scatter.dft3(rho.astype(np.float64))
    want = ewald.ewald_image(Fo, w.dx, det)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    # bound per pixel: the largest corner intensity over its wavelength samples
    I = scatter.intensity(Fo)
    kf = ewald.q_samples(det) / scatter.dq_of(n, w.dx)
    i0 = np.floor(kf).astype(np.int64)
    cmax = np.zeros(kf.shape[:-1])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                cmax = np.maximum(cmax, I[(i0[..., 2] + dz) % n, (i0[..., 1] + dy) % n, (i0[..., 0] + dx) % n])
    bound = 1e-4 * cmax.max(axis=0) + 1e-9 * I[0, 0, 0]
    ok = np.isfinite(want)
    assert ok.sum() > 1000
    assert np.all(np.abs(got[ok] - want[ok]) <= bound[ok])


@pytest.mark.parametrize("n,diam,tma", [(512, 240, False), (512, 240, True), (256, 110, False), (256, 110, True),
                                        (128, 60, False), (96, 44, False)])
def test_voxel_sinc_corrected_bins_match_oracle(n, diam, tma):
    """Sec. 2.5 voxel-sinc correction on every binning path (both z-pass engines at 256/512,
    the power-of-two kernel at 128, the runtime-radix engine at 96, and ur_bin_q) against the
    oracle's binning of |F|^2 times prod_a sinc^2(pi k_a / N); the adjoint refuses it."""
    w = mof(n, diam, nbins=128)
    rho = oracle_density(w)
    z0, nz = z_range(rho)
    plan = api.Plan(n, w.dx, w.edges, z0=z0, nz=nz)
    plan.set_voxel_sinc(True)
    assert plan.voxel_sinc()
    if tma:
        plan.set_tma_zpass(True)
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD)
    gb = api.fft_intensity(plan, dev(rho[z0:z0 + nz]), ws=ws).cpu().numpy()
    r64 = rho.astype(np.float64)
    ob = scatter.forward(r64, w.dx, w.edges, voxel_sinc_correction=True)
    compare_bins(gb, ob, r64, f"vsinc{n}")
    if n <= 128:
        I = torch.from_numpy(np.ascontiguousarray(scatter.intensity(scatter.dft3(r64))[:, :, :n // 2 + 1])
                             .astype(np.float32)).cuda()
        compare_bins(api.bin_q(plan, I).cpu().numpy(), ob, r64, f"vsinc bin_q {n}")
    with pytest.raises(api.UrError) as e:
        api.backward(plan, torch.zeros(plan.nbins, dtype=torch.float64, device="cuda"), dev(gb), dev(w.cell),
                     w.shape, ws)
    assert e.value.status == 5
    plan.set_voxel_sinc(False)
    assert not plan.voxel_sinc()
