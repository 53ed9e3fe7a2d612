"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test names the passage of the paper (or the piece of mathematics) it
checks.  The CUDA path is not involved.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import adjoint, density, merge, scatter
from paper_2303_13435_gb300 import inputs

RNG = np.random.default_rng(12345)


def _brute_dft_flat(rho):
    """Eq. 1 as the literal triple sum: one exponential per (voxel, frequency) pair."""
    n = rho.shape[0]
    idx = np.indices((n, n, n)).reshape(3, -1)  # (z, y, x) per flat voxel
    # (k.x) mod N is an exact integer, so the phase is exact up to cos/sin rounding.
    dot = (idx.T @ idx) % n
    e = np.exp(-2j * np.pi * dot / n)
    return (e @ rho.ravel()).reshape(n, n, n) / n ** 3


def _brute_dft_axes(rho):
    """Eq. 1 with the exponential split per axis (exact algebra), direct DFT matrices."""
    n = rho.shape[0]
    j = np.arange(n)
    w = np.exp(-2j * np.pi * ((j[:, None] * j[None, :]) % n) / n)
    return np.einsum("zyx,cz,by,ax->cba", rho, w, w, w) / n ** 3


@pytest.mark.parametrize("n", [4, 6, 8, 10])
def test_dft3_equals_eq1_triple_sum(n):
    """Sec. 2.4 Eq. 1: the oracle's FFT equals the literal definition on tiny grids."""
    rho = RNG.random((n, n, n))
    F = scatter.dft3(rho)
    Fb = _brute_dft_flat(rho)
    assert np.max(np.abs(F - Fb)) <= 1e-12 * np.max(np.abs(Fb))


@pytest.mark.parametrize("n", [12, 14, 16])
def test_dft3_equals_direct_dft_matrices(n):
    rho = RNG.random((n, n, n))
    F = scatter.dft3(rho)
    Fb = _brute_dft_axes(rho)
    assert np.max(np.abs(F - Fb)) <= 1e-12 * np.max(np.abs(Fb))


def test_eq2_separation_with_empty_planes():
    """Sec. 2.4 Eq. 2: 2D transforms of the nonzero planes, then 1D transforms along the
    remaining axis with the skipped planes as zeros, give the 3D transform."""
    n = 12
    rho = RNG.random((n, n, n))
    rho[:3] = 0
    rho[9:] = 0
    j = np.arange(n)
    w = np.exp(-2j * np.pi * ((j[:, None] * j[None, :]) % n) / n)
    planes = {}
    for z in range(3, 9):
        planes[z] = (w @ rho[z] @ w.T) / (n * n)   # 2D DFT over (y, x) of plane z
    F = np.zeros((n, n, n), dtype=complex)
    for kz in range(n):
        acc = np.zeros((n, n), dtype=complex)
        for z, p in planes.items():
            acc += w[kz, z] * p
        F[kz] = acc / n
    assert np.max(np.abs(F - scatter.dft3(rho))) <= 1e-12 * np.max(np.abs(F))


def test_dft_at_matches_definition():
    n = 10
    rho = RNG.random((n, n, n))
    rho[:2] = 0
    ks = np.array([[0, 0, 0], [1, -2, 3], [-5, 4, -1], [2, 2, -5]])
    Fb = _brute_dft_flat(rho)
    vals = scatter.dft_at(rho[2:], ks, z_begin=2)
    for (kx, ky, kz), v in zip(ks, vals):
        assert abs(v - Fb[kz % n, ky % n, kx % n]) <= 1e-12 * np.abs(Fb).max()


def test_parseval():
    """sum_k |F_k|^2 = (1/N^3) sum_x rho^2 under the 1/N^3 normalisation of Eq. 1."""
    n = 16
    rho = RNG.random((n, n, n))
    I = scatter.intensity(scatter.dft3(rho))
    assert math.isclose(I.sum(), (rho ** 2).sum() / n ** 3, rel_tol=1e-12)


def test_dc_is_electron_count():
    """F(0) = sum rho / N^3 (Eq. 1), so N^6 I(0) = N_e^2 (Sec. 2.2 electron count)."""
    n = 16
    rho = RNG.random((n, n, n))
    F = scatter.dft3(rho)
    assert math.isclose(F[0, 0, 0].real * n ** 3, rho.sum(), rel_tol=1e-13)
    assert math.isclose(scatter.intensity(F)[0, 0, 0] * n ** 6, rho.sum() ** 2, rel_tol=1e-12)


def test_tiling_identity():
    """Sec. 2.3 tiling: an unmasked T-fold tiling of a U^3 cell has F_N(T h) = F_U(h)
    under Eq. 1 normalisation and F_N(k) = 0 for k not divisible by T."""
    u, t = 4, 3
    n = u * t
    cell = RNG.random((u, u, u)).astype(np.float32)
    rho = density.tile_mask_density(n, cell, density.ALL).astype(np.float64)
    FN = scatter.dft3(rho)
    FU = _brute_dft_flat(cell.astype(np.float64))
    sub = FN[::t, ::t, ::t]
    assert np.max(np.abs(sub - FU)) <= 1e-12 * np.abs(FU).max()
    mask = np.ones_like(FN, dtype=bool)
    mask[::t, ::t, ::t] = False
    assert np.max(np.abs(FN[mask])) <= 1e-12 * np.abs(FU).max()


# r3(m): number of integer vectors h with |h|^2 = m (sums of three squares; OEIS A005875).
R3 = {1: 6, 2: 12, 3: 8, 4: 6, 5: 24, 6: 24, 7: 0, 8: 12, 9: 30}


def test_bragg_sc_positions_multiplicities_and_intensity():
    """Simple-cubic Gaussian-atom lattice (a = 1 nm, 16^3 cell tiled 4^3, no mask):
    intensity only at Q = 2 pi sqrt(m)/a with multiplicity r3(m), each reflection
    Z^2 exp(-sigma^2 G^2) / U^6 (Fourier transform of a normalised Gaussian)."""
    ucell, t, a, z, sig = 16, 4, 1.0, 20.0, 0.08
    n = ucell * t
    cell = inputs.sc_cell(ucell, a, z, sig)
    rho = density.tile_mask_density(n, cell, density.ALL).astype(np.float64)
    I = scatter.intensity(scatter.dft3(rho))
    k = scatter.signed_freq(n)
    k2 = (k * k)[:, None, None] + (k * k)[None, :, None] + (k * k)[None, None, :]
    strong = I > 1e-12 * I.max()
    for m, mult in R3.items():
        on_shell = k2 == t * t * m
        assert int(np.count_nonzero(strong & on_shell)) == mult
        if mult:
            g = 2 * math.pi * math.sqrt(m) / a
            expect = z * z * math.exp(-sig * sig * g * g) / ucell ** 6
            assert np.allclose(I[on_shell], expect, rtol=2e-6)
    # nothing off the reciprocal lattice (k divisible by T on every axis)
    lattice = (k[:, None, None] % t == 0) & (k[None, :, None] % t == 0) & (k[None, None, :] % t == 0)
    assert I[~lattice].max() <= 1e-20 * I.max()
    # Q positions through the binning: shells fall into the bins around 2 pi sqrt(m)/a
    dx = a / ucell
    for m in (1, 2, 3):
        q = 2 * math.pi * math.sqrt(m) / a
        edges = np.array([q * 0.999, q * 1.001])
        b = scatter.bin_intensity(I, n, dx, edges)
        assert b["count"][0] == R3[m]
        assert math.isclose(b["mean_q"][0], q, rel_tol=1e-12)


def test_sphere_form_factor():
    """Uniform voxelised sphere, padded (R <= N dx / 4): binned N^6 <I> follows
    N_e^2 [3 (sin qR - qR cos qR)/(qR)^3]^2 at low qR (staircase and voxel-sinc
    deviations of a few percent, Sec. 2.5)."""
    n, dx = 64, 0.1
    rvox = 10.0
    shape = inputs.centred_sphere(n, rvox)
    cell = np.ones((1, 1, 1), dtype=np.float32)
    rho = density.tile_mask_density(n, cell, density.SPHERE, shape.center, shape.size).astype(np.float64)
    ne = rho.sum()
    reff = (3 * ne / (4 * math.pi)) ** (1 / 3) * dx
    edges = inputs.linear_edges(inputs.nyquist_q(dx), 64)
    b = scatter.forward(rho, dx, edges)
    q = b["mean_q"]
    x = q * reff
    th = inputs.sphere_target_curve(q, reff, ne)
    meas = b["mean"] * n ** 6
    env = ne ** 2 * np.minimum(1.0, 9.0 / np.maximum(x, 1e-9) ** 4)
    sel = (x > 0.2) & (x < 8.0) & (b["count"] > 0)
    assert sel.sum() > 10
    assert np.all(np.abs(meas[sel] - th[sel]) <= 0.05 * env[sel])
    low = sel & (x < 2.0)
    assert np.all(np.abs(meas[low] / th[low] - 1) < 0.03)


def test_bin_counts_match_integer_lattice_enumeration():
    """Sec. 2.5 binning: with edges placed at dq*sqrt(t + 1/2) (never on a lattice shell),
    n_j is the number of integer vectors k in the grid with t_j < k^2 < t_j+1."""
    n, dx = 10, 0.2
    dq = 2 * math.pi / (n * dx)
    ts = [0, 1, 2, 4, 7, 12, 20, 33, 50, 74]
    edges = np.array([dq * math.sqrt(t + 0.5) for t in ts])
    b = scatter.bin_intensity(np.ones((n, n, n)), n, dx, edges)
    ks = range(-(n // 2), n - n // 2)
    counts = [0] * (len(ts) - 1)
    for kx in ks:
        for ky in ks:
            for kz in ks:
                s = kx * kx + ky * ky + kz * kz
                for j in range(len(ts) - 1):
                    if ts[j] < s <= ts[j + 1]:
                        counts[j] += 1
    assert list(b["count"]) == counts
    assert np.allclose(b["mean"][np.array(counts) > 0], 1.0)


def test_bin_edge_conventions():
    e = np.array([1.0, 2.0, 4.0])
    q = np.array([0.5, 1.0, 1.999, 2.0, 4.0, 4.0000001])
    assert list(scatter.bin_of_q(q, e)) == [-1, 0, 0, 1, 1, -1]


def test_sem_definition():
    """SEM = std (ddof 1) / sqrt(n) within a bin (Sec. 2.5 standard error on the mean)."""
    n, dx = 8, 0.5
    dq = 2 * math.pi / (n * dx)
    I = RNG.random((n, n, n))
    edges = np.array([dq * 0.5, dq * math.sqrt(2.5), dq * math.sqrt(6.5)])
    b = scatter.bin_intensity(I, n, dx, edges)
    k = scatter.signed_freq(n)
    k2 = (k * k)[:, None, None] + (k * k)[None, :, None] + (k * k)[None, None, :]
    for j, (lo, hi) in enumerate([(1, 2), (3, 6)]):
        vals = I[(k2 >= lo) & (k2 <= hi)]
        assert b["count"][j] == vals.size
        assert math.isclose(b["mean"][j], vals.mean(), rel_tol=1e-13)
        assert math.isclose(b["sem"][j], vals.std(ddof=1) / math.sqrt(vals.size), rel_tol=1e-10)


def _exact_half(x: Fraction) -> Fraction:
    """Round a rational to the nearest IEEE binary16 value, ties to even (subnormals included)."""
    if x == 0:
        return Fraction(0)
    sgn = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -14)
    ulp = Fraction(2) ** (e - 10)
    q = a / ulp
    fl = math.floor(q)
    rem = q - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sgn * fl * ulp


def test_fp16_storage_rounding_is_round_to_nearest_even():
    """ED stored as FP16 (the ED-1 storage of the three-level workload): float32 -> binary16 RNE."""
    vals = np.concatenate([RNG.random(200) * 10, RNG.random(50) * 1e-5,
                           np.array([1 + 2 ** -11, 1 + 3 * 2 ** -11, 2049.0, 2051.0, 6e-8, 3e-8]),
                           RNG.random(343 - 256) * 1e3]).astype(np.float32)
    cell = vals.reshape(7, 7, 7)
    ed = density.tile_mask_density(7, cell, density.ALL, out_dtype="f16")
    assert ed.dtype == np.float16
    for x, h in zip(cell.ravel(), ed.ravel()):
        assert Fraction(float(h)) == _exact_half(Fraction(float(x)))


def test_block_sums_exact_for_fp16_and_preserve_electrons():
    """Sec. 2.3 block integration: FP16 block sums are exact rationals; sum ED-2 = sum ED-1."""
    ed = (RNG.random((16, 16, 16)) * RNG.choice([1e-3, 1.0, 300.0], size=(16, 16, 16))).astype(np.float16)
    s = density.block_sums(ed, 4)
    for (i, j, k) in [(0, 0, 0), (1, 2, 3), (3, 3, 3)]:
        blk = ed[4 * i:4 * i + 4, 4 * j:4 * j + 4, 4 * k:4 * k + 4]
        exact = sum(Fraction(float(v)) for v in blk.ravel())
        assert Fraction(float(s[i, j, k])) == exact
    assert Fraction(float(s.sum())) == sum(Fraction(float(v)) for v in ed.ravel())
    z = density.zoom_out(ed, 4, 8, out_dtype="f16")
    assert z.shape == (8, 8, 8)
    assert np.all(z[:2] == 0) and np.all(z[6:] == 0)
    for (i, j, k) in [(0, 0, 0), (3, 1, 2)]:
        assert Fraction(float(z[2 + i, 2 + j, 2 + k])) == _exact_half(Fraction(float(s[i, j, k])))


def test_mask_voxel_counts():
    """Sec. 2.3 mask: integer-lattice counts of the sphere, cube and octahedron predicates."""
    n = 24
    c = (12.0, 12.0, 12.0)
    rr = 7.0
    m = density.shape_mask(n, density.SPHERE, c, rr, np.eye(3))
    cnt = sum(1 for i in range(-12, 12) for j in range(-12, 12) for k in range(-12, 12) if i * i + j * j + k * k <= 49)
    assert int(m.sum()) == cnt
    m = density.shape_mask(n, density.CUBE, c, 5.5, np.eye(3))
    assert int(m.sum()) == 11 ** 3
    s = 6
    m = density.shape_mask(n, density.OCTAHEDRON, c, float(s), np.eye(3))
    assert int(m.sum()) == (2 * s + 1) * (2 * s * s + 2 * s + 3) // 3
    # rotated solids keep their volume up to the surface voxels
    rot = inputs.random_rotation(inputs.SplitMix64(3))
    n = 64
    c = (32.0, 32.0, 32.0)
    m = density.shape_mask(n, density.CUBE, c, 12.0, rot)
    assert abs(m.sum() / 24.0 ** 3 - 1) < 0.03
    m = density.shape_mask(n, density.OCTAHEDRON, c, 20.0, rot)
    assert abs(m.sum() / (4.0 / 3.0 * 20.0 ** 3) - 1) < 0.05


def test_tile_wrap_and_origin():
    cell = np.arange(27, dtype=np.float32).reshape(3, 3, 3)
    t = density.tiled_cell(7, cell, origin=(1, 2, 0))
    for (z, y, x) in [(0, 0, 0), (6, 5, 4), (3, 1, 2)]:
        assert t[z, y, x] == cell[z % 3, (y + 2) % 3, (x + 1) % 3]


def _loss_from_um(u, m, dx, edges, coeff, origin=(0, 0, 0)):
    n = m.shape[0]
    rho = density.tiled_cell(n, u.astype(np.float32), origin).astype(np.float64)
    # float64 cell values (not the float32 copy) so the finite differences see small steps
    uu = u[np.ix_((np.arange(n) + origin[2]) % u.shape[0], (np.arange(n) + origin[1]) % u.shape[0],
                  (np.arange(n) + origin[0]) % u.shape[0])]
    rho = uu * m
    b = scatter.forward(rho, dx, edges)
    mean = np.nan_to_num(b["mean"])
    return float((coeff * mean ** 2).sum()), b, rho


def test_adjoint_matches_finite_differences():
    """Chain rule of the forward map checked by central differences in FP64."""
    n, ucell, dx = 8, 4, 0.25
    u = RNG.random((ucell, ucell, ucell))
    m = RNG.random((n, n, n))
    edges = inputs.log_edges(2 * math.pi / (n * dx) * 0.9, math.pi / dx * 1.6, 7)
    coeff = RNG.random(7) + 0.5
    L, b, rho = _loss_from_um(u, m, dx, edges, coeff, origin=(1, 0, 2))
    g = 2 * coeff * np.nan_to_num(b["mean"])
    grho = adjoint.grad_rho(rho, dx, edges, g, count=b["count"])
    gu, gm = adjoint.grad_cell_and_mask(grho, u, m, origin=(1, 0, 2))
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 3), (3, 3, 1)]:
        up, um_ = u.copy(), u.copy()
        up[idx] += h
        um_[idx] -= h
        fd = (_loss_from_um(up, m, dx, edges, coeff, (1, 0, 2))[0] - _loss_from_um(um_, m, dx, edges, coeff, (1, 0, 2))[0]) / (2 * h)
        assert math.isclose(fd, gu[idx], rel_tol=1e-6, abs_tol=1e-9 * abs(L))
    for idx in [(0, 0, 0), (4, 5, 6), (7, 1, 3)]:
        mp, mm = m.copy(), m.copy()
        mp[idx] += h
        mm[idx] -= h
        fd = (_loss_from_um(u, mp, dx, edges, coeff, (1, 0, 2))[0] - _loss_from_um(u, mm, dx, edges, coeff, (1, 0, 2))[0]) / (2 * h)
        assert math.isclose(fd, gm[idx], rel_tol=1e-6, abs_tol=1e-9 * abs(L))


def test_adjoint_directional_derivative():
    """<dL/drho, d> equals d/dt L(rho + t d) (central difference in t)."""
    n, dx = 10, 0.1
    rho = RNG.random((n, n, n))
    d = RNG.standard_normal((n, n, n))
    edges = inputs.linear_edges(inputs.nyquist_q(dx), 9)
    coeff = RNG.random(9)

    def L(r):
        mean = np.nan_to_num(scatter.forward(r, dx, edges)["mean"])
        return float((coeff * mean ** 2).sum()), mean

    L0, mean0 = L(rho)
    grho = adjoint.grad_rho(rho, dx, edges, 2 * coeff * mean0)
    t = 1e-5
    fd = (L(rho + t * d)[0] - L(rho - t * d)[0]) / (2 * t)
    assert math.isclose(fd, float((grho * d).sum()), rel_tol=1e-7)


def test_merge_windows_and_absolute_scale():
    """Sec. 2.5 merge: each output bin comes from the level whose validity window
    (up to pi/dx) holds its geometric centre, scaled by N^6 to absolute units."""
    edges = inputs.log_edges(0.05, 20.0, 30)
    nb = 30
    lv = []
    for n, dx, val in [(16, 0.4, 1.0), (16, 0.8, 2.0), (32, 0.1, 3.0)]:
        lv.append({"n": n, "dx": dx, "count": np.full(nb, 5), "mean": np.full(nb, val),
                   "sem": np.full(nb, val / 10), "mean_q": np.full(nb, dx)})
    lv[0]["count"][3] = 0
    out = merge.merge_levels(lv, edges)
    qn = {1: math.pi / 0.8, 0: math.pi / 0.4, 2: math.pi / 0.1}
    for j in range(nb):
        c = math.sqrt(edges[j] * edges[j + 1])
        want = 1 if c < qn[1] else (0 if c < qn[0] else (2 if c <= qn[2] else -1))
        if want == 0 and j == 3:
            want = -1
        assert out["source"][j] == want
        if want >= 0:
            assert out["mean"][j] == lv[want]["mean"][j] * lv[want]["n"] ** 6
            assert out["sem"][j] == lv[want]["sem"][j] * lv[want]["n"] ** 6
        else:
            assert math.isnan(out["mean"][j]) and out["count"][j] == 0


def test_merge_levels_share_forward_scattering():
    """Block integration keeps the electron count, so N^6 I(0) = N_e^2 at every level
    (Sec. 2.2 electron-count identity carried through Sec. 2.3 zoom-out)."""
    n1 = 32
    shape = inputs.centred_sphere(n1, 10.0)
    cell = inputs.sc_cell(8, 1.0)
    ed1 = density.tile_mask_density(n1, cell, density.SPHERE, shape.center, shape.size, out_dtype="f16")
    ne = float(ed1.astype(np.float64).sum())
    for f, nout in [(2, 32), (4, 32)]:
        ed = density.zoom_out(ed1, f, nout, out_dtype="f32")
        F = scatter.dft3(ed)
        assert math.isclose(scatter.intensity(F)[0, 0, 0] * nout ** 6, ne ** 2, rel_tol=1e-6)


def test_log_mse_loss_gradient_matches_central_differences():
    """The log-I(Q) MSE of the oracle against central differences of its own value;
    bins that are empty (NaN) or non-positive take no part."""
    rng = np.random.default_rng(5)
    mean = rng.uniform(0.5, 2.0, 40)
    mean[[3, 17]] = np.nan
    mean[25] = 0.0
    target = rng.uniform(0.5, 2.0, 40)
    L, g = adjoint.loss_log_mse(mean, target)
    ok = np.isfinite(mean) & (mean > 0)
    assert np.all(g[~ok] == 0.0)
    h = 1e-6
    for j in np.flatnonzero(ok)[:10]:
        mp, mm = mean.copy(), mean.copy()
        mp[j] += h
        mm[j] -= h
        fd = (adjoint.loss_log_mse(mp, target)[0] - adjoint.loss_log_mse(mm, target)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-7 * max(1.0, abs(g[j]))
    # value: a plain mean of squared log ratios over the valid bins
    assert math.isclose(L, float(np.mean(np.log(mean[ok] / target[ok]) ** 2)), rel_tol=1e-12)


def _blocky_sphere_levels(voxel_sinc_correction):
    """ED-1 (64^3, dx 0.05 nm) of a sphere built from whole 4^3 blocks, and its 2x and 4x
    block sums (Sec. 2.3 zoom-out) in boxes of the same physical size (32^3, 16^3).  Bin edges
    put the level limits pi/dx on bin edges (just below, so no lattice shell sits on one)."""
    n1, dx1 = 64, 0.05
    b = np.arange(n1 // 4) + 0.5 - n1 // 8
    blocks = ((b[:, None, None] ** 2 + b[None, :, None] ** 2 + b[None, None, :] ** 2) <= 16.0).astype(np.float64)
    ed1 = np.repeat(np.repeat(np.repeat(blocks, 4, 0), 4, 1), 4, 2)
    q3, q2, q1 = math.pi / (4 * dx1), math.pi / (2 * dx1), math.pi / dx1
    lo = 0.9 * 2 * math.pi / (n1 * dx1)
    edges = np.concatenate([inputs.log_edges(lo, q3 * (1 - 1e-9), 12)[:-1],
                            inputs.log_edges(q3 * (1 - 1e-9), q2 * (1 - 1e-9), 6)[:-1],
                            inputs.log_edges(q2 * (1 - 1e-9), q1, 6)])
    levels = []
    for f, n_out in [(1, 64), (2, 32), (4, 16)]:
        ed = ed1 if f == 1 else density.zoom_out(ed1, f, n_out, out_dtype="f32").astype(np.float64)
        ob = scatter.forward(ed, dx1 * f, edges, voxel_sinc_correction=voxel_sinc_correction)
        levels.append({"n": n_out, "dx": dx1 * f, "count": ob["count"], "mean": ob["mean"], "sem": ob["sem"],
                       "mean_q": ob["mean_q"]})
    return ed1, dx1, edges, levels


def test_merge_absolute_scale_and_seam_continuity():
    """Sec. 2.5 merge of zoom levels, pinned without the merge's own formula.

    A density made of whole 4^3 blocks is represented exactly by its 2x and 4x block sums, and
    the unnormalised transforms of the three levels then differ, frequency by frequency, by the
    ratio of their voxels' form factors (the geometric sum over a block equals
    f sinc(f q dx/2)/sinc(q dx/2) per axis).  With the voxel-sinc correction the absolute
    level curves are therefore equal in every bin below the coarser level's limit, so
    merging all three levels must reproduce ED-1 alone there (continuity at both seams),
    and the lowest bin must follow N_e^2 [3 (sin qR - qR cos qR)/(qR)^3]^2 (Sec. 2.2 electron
    count, uniform-sphere form factor).  Scaling a level by N^3 instead of N^6, or by another
    level's N, breaks both."""
    ed1, dx1, edges, levels = _blocky_sphere_levels(True)
    m_all = merge.merge_levels(levels, edges)
    m_ed1 = merge.merge_levels(levels[:1], edges)
    q2 = math.pi / (2 * dx1)
    below = (edges[1:] <= q2) & (m_ed1["count"] > 0)
    assert set(m_all["source"][below]) == {1, 2}
    assert np.array_equal(m_all["count"][below], m_ed1["count"][below])
    rel = np.abs(m_all["mean"][below] / m_ed1["mean"][below] - 1)
    assert rel.max() < 1e-9
    # within the SEM of either level at each seam (here: to rounding; a shell of symmetric
    # voxels has an SEM at rounding level itself)
    for j in np.flatnonzero(below):
        tol = min(m_all["sem"][j], m_ed1["sem"][j]) + 1e-12 * m_ed1["mean"][j]
        assert abs(m_all["mean"][j] - m_ed1["mean"][j]) <= tol
    # absolute scale: electrons^2 of the unnormalised transform
    ne = float(ed1.sum())
    reff = (3 * ne * dx1 ** 3 / (4 * math.pi)) ** (1 / 3)
    first = np.flatnonzero((m_all["count"] > 0) & (m_all["mean_q"] * reff < 2.4))
    assert len(first) >= 2
    th = inputs.sphere_target_curve(m_all["mean_q"][first], reff, ne)
    # staircase of the blocky surface: a few percent at qR ~ 2 (the first shell: 1 %)
    assert np.all(np.abs(m_all["mean"][first] / th - 1) < 0.03)
    assert m_all["source"][first[0]] == 2


def test_voxel_sinc_is_what_aligns_block_summed_levels():
    """Without the voxel-sinc factor the 4x level of the block density is damped towards its
    limit by the block's geometric sum (ratio ~0.45 at the axis Nyquist), and with it the
    levels agree: the factor is prod_a sinc^2(pi k_a / N), not a look-alike."""
    _, dx1, edges, raw = _blocky_sphere_levels(False)
    _, _, _, cor = _blocky_sphere_levels(True)
    q3 = math.pi / (4 * dx1)
    sel = (edges[1:] <= q3) & (raw[0]["count"] > 0)
    ratio_raw = raw[2]["mean"][sel] * 16.0 ** 6 / (raw[0]["mean"][sel] * 64.0 ** 6)
    ratio_cor = cor[2]["mean"][sel] * 16.0 ** 6 / (cor[0]["mean"][sel] * 64.0 ** 6)
    assert np.allclose(ratio_cor, 1.0, rtol=1e-9)
    assert ratio_raw[-1] > 1.2  # the coarse point-sample transform overshoots the voxelised one near its limit
    assert np.all(ratio_raw >= 1.0 - 1e-12)
    # the factor itself: one at k = 0, (2/pi)^2 per axis at the Nyquist index, symmetric in k
    s = scatter.voxel_sinc(8)
    assert s[0, 0, 0] == 1.0
    assert math.isclose(s[0, 0, 4], (2 / math.pi) ** 2, rel_tol=1e-15)
    assert math.isclose(s[4, 4, 4], (2 / math.pi) ** 6, rel_tol=1e-14)
    assert np.allclose(s[1], s[7])


def _invvar_levels(means, sems, ns, dxs, counts=None):
    nb = len(means[0])
    out = []
    for i, (m, s, n, dx) in enumerate(zip(means, sems, ns, dxs)):
        out.append({"n": n, "dx": dx, "count": np.full(nb, 10) if counts is None else counts[i],
                    "mean": np.asarray(m, dtype=np.float64) / float(n) ** 6,
                    "sem": np.asarray(s, dtype=np.float64) / float(n) ** 6, "mean_q": np.full(nb, 1.0)})
    return out


def test_invvar_merge_is_the_maximum_likelihood_combination():
    """Sec. 2.7 (uncertainty-optimised merge of overlapping curves): for independent Gaussian
    errors the combined value maximises the likelihood; found here by a 1-D minimisation of
    chi^2, independent of the closed form, and its spread over repeated draws is the SEM."""
    from scipy.optimize import minimize_scalar
    edges = np.array([1.0, 1.1, 1.2])
    means = [[5.0, 7.0], [5.6, 6.1], [4.2, 9.0]]
    sems = [[0.3, 1.0], [0.5, 0.2], [1.5, 3.0]]
    lv = _invvar_levels(means, sems, [8, 12, 16], [0.01, 0.02, 0.04])
    out = merge.merge_levels(lv, edges, mode="invvar")
    for j in range(2):
        chi2 = lambda mu: sum((means[l][j] - mu) ** 2 / sems[l][j] ** 2 for l in range(3))
        r = minimize_scalar(chi2, bounds=(0, 20), method="bounded", options={"xatol": 1e-12})
        assert math.isclose(out["mean"][j], r.x, rel_tol=1e-9)
        # curvature of chi^2 = 2 / SEM^2 (second difference, independent of the weights' form)
        h = 1e-3
        curv = (chi2(r.x + h) - 2 * chi2(r.x) + chi2(r.x - h)) / h ** 2
        assert math.isclose(out["sem"][j], math.sqrt(2.0 / curv), rel_tol=1e-6)
        assert out["count"][j] == 30
    # repeated draws: the combined estimate is unbiased and spreads by its SEM
    rng = np.random.default_rng(4)
    mu, sig = 3.0, np.array([0.2, 0.35, 0.9])
    draws = []
    for _ in range(4000):
        m = mu + sig * rng.standard_normal(3)
        lv = _invvar_levels([[v] for v in m], [[s] for s in sig], [8, 8, 8], [0.01, 0.02, 0.04])
        draws.append(merge.merge_levels(lv, np.array([1.0, 1.1]), mode="invvar")["mean"][0])
    draws = np.array(draws)
    sem_c = 1.0 / math.sqrt(float((1.0 / sig ** 2).sum()))
    assert abs(draws.mean() - mu) < 4 * sem_c / math.sqrt(len(draws))
    assert abs(draws.std(ddof=1) / sem_c - 1) < 0.05


def test_invvar_merge_respects_level_limits_and_falls_back():
    """Levels beyond their pi/dx limit take no part; a bin where no trusted level has a usable
    SEM takes the windows choice."""
    edges = np.array([10.0, 11.0, 100.0, 110.0])
    # level 0: dx 0.02 (limit 157); level 1: dx 0.2 (limit 15.7)
    lv = _invvar_levels([[2.0, 8.0, 1.0], [3.0, 9.0, 5.0]], [[1.0, 1.0, 0.5], [1.0, 1.0, 0.5]], [16, 8],
                        [0.02, 0.2])
    lv[0]["sem"][1] = np.nan
    out = merge.merge_levels(lv, edges, mode="invvar")
    assert math.isclose(out["mean"][0], 2.5, rel_tol=1e-12) and out["count"][0] == 20
    assert math.isclose(out["sem"][0], 1 / math.sqrt(2), rel_tol=1e-12)
    # bin 1 (centre 33 > 15.7): only level 0 is trusted and its SEM is NaN -> windows choice
    w = merge.merge_levels(lv, edges)
    assert out["source"][1] == w["source"][1] == 0 and math.isclose(out["mean"][1], 8.0, rel_tol=1e-12)
    # bin 2 (centre 105): level 1 is beyond its limit
    assert out["source"][2] == 0 and math.isclose(out["mean"][2], 1.0, rel_tol=1e-12)
    assert math.isclose(out["sem"][2], 0.5, rel_tol=1e-12)


def test_rotated_lattice_identity_and_quarter_turn_are_exact_index_maps():
    """Sec. 2.3 rotated sampling of the cell: with R = I and an integer offset the samples
    fall on cell voxels (weights 0/1) and reproduce the integer wrap exactly; a quarter turn
    about z permutes the axes exactly."""
    cell = inputs.mof_like_cell(16, 0.65, 0)
    n, c = 24, (12.0, 12.0, 12.0)
    a = density.rotated_cell(n, cell, np.eye(3), (12 + 3, 12 + 5, 12 + 7), center=c)
    assert np.array_equal(a, density.tiled_cell(n, cell, origin=(3, 5, 7)))
    quarter = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], dtype=np.float32)
    a = density.rotated_cell(n, cell, quarter, c, center=c)
    zz, yy, xx = np.indices((n, n, n))
    assert np.array_equal(a, cell[zz % 16, xx % 16, (24 - yy) % 16])


def test_rotated_lattice_matches_scipy_grid_wrap_linear_interpolation():
    """The sampling the paper names (scipy.ndimage.map_coordinates, grid-wrap), at order 1
    and in float64, agrees with the float32 oracle to float32 rounding."""
    from scipy import ndimage
    cell = inputs.mof_like_cell(16, 0.65, 0)
    n, c = 24, (12.0, 12.0, 12.0)
    rot = inputs.random_rotation(inputs.SplitMix64(5))
    q = (12.3, 11.7, 12.9)
    a = density.rotated_cell(n, cell, rot, q, center=c)
    zz, yy, xx = np.indices((n, n, n))
    d = np.stack([xx - 12.0, yy - 12.0, zz - 12.0]).reshape(3, -1)
    p = rot.astype(np.float64) @ d + np.asarray(q)[:, None]
    ref = ndimage.map_coordinates(cell.astype(np.float64), [p[2], p[1], p[0]], order=1, mode="grid-wrap")
    assert np.abs(a - ref.reshape(n, n, n)).max() <= 4e-6 * np.abs(cell).max()
    # a rotated lattice keeps the cell's mean density to interpolation accuracy
    big = density.rotated_cell(64, cell, rot, (32.0, 32.0, 32.0), center=(32.0, 32.0, 32.0))
    assert abs(big.mean() / cell.mean() - 1) < 0.02


def test_ensemble_of_voxelised_spheres_follows_the_polydisperse_closed_form():
    """Sec. 3 polydispersity as volume-weighted single-particle simulations: the ensemble of
    voxelised uniform spheres of three radii, with w_i = phi_i / V_i and equal volume
    fractions, follows sum_i w_i (rho V_i)^2 [3 (sin qR_i - qR_i cos qR_i)/(qR_i)^3]^2 at low
    q, and its forward scattering is rho^2 sum_i phi_i V_i (the volume-weighted mean volume)."""
    n, dx = 48, 0.1
    radii = [5.0, 7.0, 9.0]
    edges = inputs.linear_edges(inputs.nyquist_q(dx), 40)
    items, vols, nes = [], [], []
    cell = np.ones((1, 1, 1), dtype=np.float32)
    for r in radii:
        sh = inputs.centred_sphere(n, r)
        rho = density.tile_mask_density(n, cell, density.SPHERE, sh.center, sh.size).astype(np.float64)
        ob = scatter.forward(rho, dx, edges)
        items.append({"n": n, "count": ob["count"], "mean": ob["mean"], "sem": ob["sem"], "mean_q": ob["mean_q"]})
        nes.append(rho.sum())
        vols.append(rho.sum() * dx ** 3)   # unit density: electrons = voxels
    phi = [1 / 3] * 3
    w = [p / v for p, v in zip(phi, vols)]
    ens = merge.ensemble_sum(items, w)
    q = ens["mean_q"]
    th = np.zeros_like(q)
    for wi, ne, v in zip(w, nes, vols):
        reff = (3 * v / (4 * math.pi)) ** (1 / 3)
        th += wi * inputs.sphere_target_curve(q, reff, ne)
    sel = (ens["count"] > 0) & (q * 9 * dx < 2.0)
    assert sel.sum() >= 2
    assert np.all(np.abs(ens["mean"][sel] / th[sel] - 1) < 0.04)
    # forward scattering through the DC voxel: sum_i w_i N_e,i^2 = sum_i phi_i V_i / dx^6 (unit density)
    i0 = sum(wi * (float(scatter.dft3(
        density.tile_mask_density(n, cell, density.SPHERE, inputs.centred_sphere(n, r).center, np.float32(r)))[0, 0, 0].real
        * n ** 3)) ** 2 for wi, r in zip(w, radii))
    assert math.isclose(i0, sum(p * v for p, v in zip(phi, vols)) / dx ** 6, rel_tol=1e-12)


def test_ensemble_is_linear_and_needs_every_member():
    nb = 5
    a = {"n": 8, "count": np.array([3, 3, 0, 3, 3]), "mean": np.array([1.0, 2, 3, 4, 5]) / 8 ** 6,
         "sem": np.full(nb, 0.1) / 8 ** 6, "mean_q": np.ones(nb)}
    b = {"n": 16, "count": np.array([4, 4, 4, 4, 0]), "mean": np.array([5.0, 4, 3, 2, 1]) / 16 ** 6,
         "sem": np.full(nb, 0.2) / 16 ** 6, "mean_q": np.full(nb, 2.0)}
    e = merge.ensemble_sum([a, b], [2.0, 0.5])
    assert np.allclose(e["mean"][[0, 1, 3]], 2.0 * np.array([1, 2, 4]) + 0.5 * np.array([5, 4, 2]), rtol=1e-14)
    assert np.isnan(e["mean"][2]) and np.isnan(e["mean"][4]) and e["count"][2] == 0
    assert math.isclose(e["sem"][0], math.hypot(2.0 * 0.1, 0.5 * 0.2), rel_tol=1e-14)
    assert e["count"][0] == 7 and math.isclose(e["mean_q"][0], (3 * 1 + 4 * 2) / 7)
    # a member of zero weight does not invalidate a bin
    e = merge.ensemble_sum([a, b], [1.0, 0.0])
    assert math.isclose(e["mean"][4], 5.0, rel_tol=1e-14) and np.isnan(e["mean"][2])


def _ewald_det(**kw):
    d = {"nx": 33, "ny": 29, "pixel_m": 0.002, "distance_m": 0.5, "beam": (16.0, 14.0), "wavelength_nm": 0.154,
         "bandwidth": 0.0, "nlambda": 1, "rot": np.eye(3)}
    d.update(kw)
    return d


def test_ewald_image_of_a_gaussian_follows_its_closed_form():
    """Sec. 2.5 Ewald-sphere extraction: a well-sampled Gaussian blob has I(q) = I(0)
    exp(-sigma^2 |q|^2), so each pixel must read that at |q| = (4 pi / lambda) sin(theta),
    2 theta the pixel's scattering angle; with a wavelength band, the mean over the band."""
    from oracle import ewald
    n, dx, sv = 64, 0.05, 1.0
    zz, yy, xx = np.indices((n, n, n)).astype(np.float64)
    rho = np.exp(-((xx - 32) ** 2 + (yy - 32) ** 2 + (zz - 32) ** 2) / (2 * sv * sv))
    F = scatter.dft3(rho)
    i0 = scatter.intensity(F)[0, 0, 0]
    sig = sv * dx
    for det in (_ewald_det(pixel_m=0.006),
                _ewald_det(pixel_m=0.006, bandwidth=0.1, nlambda=5, rot=inputs.random_rotation(inputs.SplitMix64(2)))):
        img = ewald.ewald_image(F, dx, det)
        s = ewald.pixel_directions(det)
        two_theta = np.arccos(np.clip(s[..., 2], -1, 1))
        want = np.zeros_like(img)
        for lam in ewald.wavelengths(det):
            q = 4 * math.pi / lam * np.sin(two_theta / 2)
            want += i0 * np.exp(-(sig * q) ** 2)
        want /= len(ewald.wavelengths(det))
        ok = np.isfinite(img) & (want > 1e-3 * i0)
        assert ok.sum() > 100
        # trilinear interpolation of a Gaussian 10 grid steps wide: under 1 %
        assert np.max(np.abs(img[ok] / want[ok] - 1)) < 0.01


def test_ewald_beam_centre_reads_forward_scattering_and_trilinear_is_scipys():
    """The direct-beam pixel samples q = 0 (I(0) exactly, at every wavelength); the
    interpolation agrees with scipy.ndimage.map_coordinates at order 1."""
    from scipy import ndimage
    from oracle import ewald
    n, dx = 16, 0.2
    rho = RNG.random((n, n, n))
    F = scatter.dft3(rho)
    I = scatter.intensity(F)
    det = _ewald_det(nx=9, ny=9, beam=(4.0, 4.0), pixel_m=0.02, distance_m=0.3, wavelength_nm=0.5,
                     bandwidth=0.2, nlambda=3, rot=inputs.random_rotation(inputs.SplitMix64(8)))
    img = ewald.ewald_image(F, dx, det)
    assert img[4, 4] == I[0, 0, 0]
    kf = ewald.q_samples(det) / scatter.dq_of(n, dx)
    val, valid = ewald.trilinear(I, kf)
    Ish = np.fft.fftshift(I)
    ref = ndimage.map_coordinates(Ish, [kf[..., 2].ravel() + n // 2, kf[..., 1].ravel() + n // 2,
                                        kf[..., 0].ravel() + n // 2], order=1, mode="nearest").reshape(val.shape)
    assert valid.sum() > 50
    assert np.allclose(val[valid], ref[valid], rtol=1e-12, atol=1e-15)


def test_parity_count_helper_matches_brute_force():
    """The helper behind the GPU two-voxel walk test (per-bin counts of all voxels and of the
    kx-even ones, from the axes' k^2 histograms convolved by FFT) against a brute-force count
    over every k of small grids, including an odd-radix edge."""
    import math
    from _cases import oracle_parity_counts
    from paper_2303_13435_gb300 import inputs
    for n, nb in [(32, 20), (64, 40), (126, 96)]:
        dx = 0.04
        edges = inputs.log_edges(2 * math.pi / (n * dx), math.pi / dx, nb)
        even, total = oracle_parity_counts(n, dx, edges)
        k = scatter.signed_freq(n)
        kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
        j = scatter.bin_of_q(scatter.q_of_k2(kx ** 2 + ky ** 2 + kz ** 2, n, dx), edges)
        assert np.array_equal(total, np.bincount(j[j >= 0], minlength=nb))
        assert np.array_equal(even, np.bincount(j[(j >= 0) & (kx % 2 == 0)], minlength=nb))
