"""Oracle: electron-density generation (paper Sec. 2.3).  TEST INFRASTRUCTURE ONLY.

ED-1 (Sec. 2.3, first paragraph): the unit-cell density ED-Unit is repeated
outside its boundaries (periodic wrap) and multiplied, plane by plane, by a mask
that defines the particle boundary.  The paper samples the cell on rotated
planes with spline interpolation; this oracle takes the axis-aligned integer
wrap, rho(x) = u((x + o) mod U) * m(x).

ED-2 / ED-3 (Sec. 2.3, second paragraph): block integration (a sum over f^3
blocks, as skimage's block_reduce with np.sum does) followed by zero padding,
the block-summed particle centred in the new box.

Readings:
* Voxel i of an axis has the coordinate d = fl32(i - c) in voxel units, c the
  particle centre.  The mask decision is taken in float32 with every product
  and sum rounded separately in the order written below, because the CUDA
  kernel takes the same decision in float32; the voxel set then agrees exactly.
* sphere:     (dx*dx + dy*dy) + dz*dz <= s*s
  cube:       max_a |p_a| <= s,     p_a = (R[0,a] dx + R[1,a] dy) + R[2,a] dz
  octahedron: (|p_0| + |p_1|) + |p_2| <= s
* rho = fl32(u * m); an FP16 ED is that float32 value rounded to nearest even.
* Block sums are taken in float64.  For FP16 inputs (multiples of 2^-24 below
  2^16 in magnitude) and up to 4096 terms every partial sum is exact, so the
  result does not depend on the summation order; it is then rounded once to
  the output type.
"""
from __future__ import annotations

import numpy as np

SPHERE, CUBE, OCTAHEDRON, ALL, WEIGHTS = 0, 1, 2, 3, 4


def _axis_offsets(n: int, c: np.float32) -> np.ndarray:
    return np.arange(n, dtype=np.float32) - np.float32(c)


def shape_mask(n: int, kind: int, center, size, rot, z_begin: int = 0, z_count: int | None = None) -> np.ndarray:
    """0/1 float32 mask [z][y][x] for planes [z_begin, z_begin + z_count)."""
    if z_count is None:
        z_count = n - z_begin
    c = np.asarray(center, dtype=np.float32)
    s = np.float32(size)
    r = np.asarray(rot, dtype=np.float32).reshape(3, 3)
    dxv = _axis_offsets(n, c[0])
    dyv = _axis_offsets(n, c[1])
    dzv = (np.arange(z_begin, z_begin + z_count, dtype=np.float32) - np.float32(c[2]))
    if kind == ALL:
        return np.ones((z_count, n, n), dtype=np.float32)
    if kind == SPHERE:
        xy = (dxv * dxv)[None, None, :] + (dyv * dyv)[None, :, None]
        tot = xy + (dzv * dzv)[:, None, None]
        inside = tot <= s * s
    elif kind in (CUBE, OCTAHEDRON):
        p = []
        for a in range(3):
            pa = (r[0, a] * dxv)[None, None, :] + (r[1, a] * dyv)[None, :, None]
            pa = pa + (r[2, a] * dzv)[:, None, None]
            p.append(np.abs(pa))
        if kind == CUBE:
            inside = (p[0] <= s) & (p[1] <= s) & (p[2] <= s)
        else:
            inside = ((p[0] + p[1]) + p[2]) <= s
    else:
        raise ValueError(f"unknown shape kind {kind}")
    return inside.astype(np.float32)


def tiled_cell(n: int, cell: np.ndarray, origin=(0, 0, 0), z_begin: int = 0, z_count: int | None = None) -> np.ndarray:
    """u((x + o) mod U) for planes [z_begin, z_begin + z_count), float32 [z][y][x]."""
    if z_count is None:
        z_count = n - z_begin
    u = cell.shape[0]
    ox, oy, oz = origin
    iz = (np.arange(z_begin, z_begin + z_count) + oz) % u
    iy = (np.arange(n) + oy) % u
    ix = (np.arange(n) + ox) % u
    return cell[np.ix_(iz, iy, ix)].astype(np.float32)


def rotated_cell(n: int, cell: np.ndarray, lat_rot, lat_offset, z_begin: int = 0, z_count: int | None = None,
                 center=None) -> np.ndarray:
    """The unit cell sampled on a rotated lattice with periodic wrap, float32 [z][y][x].

    Sec. 2.3 (first paragraph) interpolates the reduced cell over rotated planes with
    scipy's map_coordinates in grid-wrap mode, the cell repeating outside its bounds, to
    give the crystal an orientation (the way to polycrystalline grains).  Reading: the
    sample point of voxel x, in cell-voxel units, is p = R (x - c) + q, with R the lattice
    rotation, c the rotation centre (the particle centre) and q = c + o an offset; the
    value is the trilinear interpolation (order 1) of the periodic cell at p.  Every step
    is float32 with each product, sum and difference rounded separately, in this order:
      d_b = x_b - c_b;  p_a = ((R[a][0] d_0 + R[a][1] d_1) + R[a][2] d_2) + q_a
      i = floor(p), f = p - i (exact), lerp(a, b, f) = a + f (b - a)
      along x, then y, then z over the 8 neighbours (i + {0,1}) mod U.
    (x, y, z) = (index 2, 1, 0) of the [z][y][x] arrays, as for the shape masks.
    """
    if z_count is None:
        z_count = n - z_begin
    u = cell.shape[0]
    cl = np.asarray(cell, dtype=np.float32)
    r = np.asarray(lat_rot, dtype=np.float32).reshape(3, 3)
    c = np.asarray(center if center is not None else (n // 2, n // 2, n // 2), dtype=np.float32)
    q = np.asarray(lat_offset, dtype=np.float32)
    dx = (np.arange(n, dtype=np.float32) - c[0])[None, None, :]
    dy = (np.arange(n, dtype=np.float32) - c[1])[None, :, None]
    dz = (np.arange(z_begin, z_begin + z_count, dtype=np.float32) - c[2])[:, None, None]
    p = []
    for a in range(3):
        pa = (r[a, 0] * dx + r[a, 1] * dy)
        pa = pa + r[a, 2] * dz
        p.append((pa + q[a]).astype(np.float32))
    i = [np.floor(pa) for pa in p]
    f = [(pa - ia).astype(np.float32) for pa, ia in zip(p, i)]
    ii = [np.mod(ia.astype(np.int64), u) for ia in i]
    ij = [np.mod(ia + 1, u) for ia in ii]

    def lerp(a0, a1, t):
        return (a0 + t * (a1 - a0)).astype(np.float32)

    def g(iz, iy, ix):
        return cl[iz, iy, ix]

    x0, x1 = ii[0], ij[0]
    y0, y1 = ii[1], ij[1]
    z0, z1 = ii[2], ij[2]
    c00 = lerp(g(z0, y0, x0), g(z0, y0, x1), f[0])
    c01 = lerp(g(z0, y1, x0), g(z0, y1, x1), f[0])
    c10 = lerp(g(z1, y0, x0), g(z1, y0, x1), f[0])
    c11 = lerp(g(z1, y1, x0), g(z1, y1, x1), f[0])
    c0 = lerp(c00, c01, f[1])
    c1 = lerp(c10, c11, f[1])
    return lerp(c0, c1, f[2]).astype(np.float32)


def mask_values(n: int, kind: int, center=(0, 0, 0), size=0.0, rot=np.eye(3), weights=None,
                z_begin: int = 0, z_count: int | None = None) -> np.ndarray:
    if kind == WEIGHTS:
        if z_count is None:
            z_count = n - z_begin
        return np.asarray(weights, dtype=np.float32)[z_begin:z_begin + z_count]
    return shape_mask(n, kind, center, size, rot, z_begin, z_count)


def tile_mask_density(n: int, cell: np.ndarray, kind: int, center=(0, 0, 0), size=0.0, rot=np.eye(3),
                      origin=(0, 0, 0), weights=None, out_dtype: str = "f32",
                      z_begin: int = 0, z_count: int | None = None, lattice=None) -> np.ndarray:
    """ED-1 for planes [z_begin, z_begin + z_count): rho = fl32(u(x mod U) * m(x)), optionally to FP16.

    lattice: None (axis-aligned integer wrap with `origin`) or (R, q) for rotated_cell, the
    rotation centre being the shape's centre."""
    if lattice is None:
        u = tiled_cell(n, cell, origin, z_begin, z_count)
    else:
        u = rotated_cell(n, cell, lattice[0], lattice[1], z_begin, z_count, center=center)
    m = mask_values(n, kind, center, size, rot, weights, z_begin, z_count)
    rho = u * m  # float32 * float32 -> float32, one rounding
    if out_dtype == "f16":
        return rho.astype(np.float16)
    return rho


def nonzero_plane_range(rho: np.ndarray) -> tuple[int, int]:
    """(first, last) plane index with any nonzero voxel; (n, -1) when all planes are zero."""
    nz = np.flatnonzero(np.any(rho != 0, axis=(1, 2)))
    if nz.size == 0:
        return rho.shape[0], -1
    return int(nz[0]), int(nz[-1])


def block_sums(ed: np.ndarray, f: int) -> np.ndarray:
    """Float64 sums of ED over aligned f^3 blocks (ED edge divisible by f)."""
    n1 = ed.shape[0]
    if n1 % f:
        raise ValueError("edge not divisible by the block factor")
    m = n1 // f
    e64 = ed.astype(np.float64)
    return e64.reshape(m, f, m, f, m, f).sum(axis=(1, 3, 5))


def zoom_out(ed: np.ndarray, f: int, n_out: int, out_dtype: str = "f16") -> np.ndarray:
    """ED-2/ED-3: f^3 block integration of ED, centred in a zero box of edge n_out."""
    s = block_sums(ed, f)
    m = s.shape[0]
    if m > n_out:
        raise ValueError("zoomed particle larger than the box")
    o = (n_out - m) // 2
    out = np.zeros((n_out, n_out, n_out), dtype=np.float64)
    out[o:o + m, o:o + m, o:o + m] = s
    if out_dtype == "f16":
        return out.astype(np.float16)
    return out.astype(np.float32)
