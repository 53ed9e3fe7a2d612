"""Seeded synthetic inputs shared by the CUDA path's tests and by the oracle.

This module generates inputs only: unit-cell densities, particle shapes, Q-bin
edges and workload descriptions.  It contains none of the simulation's own
arithmetic (tiling, masking, Fourier transform, binning, merging, adjoint).

The paper computes its unit-cell electron density (ED-Unit, Sec. 2.2) with
DFT, which is not available here.  The stand-in is a cell of Gaussian atoms,
point-sampled on the voxel grid and summed over neighbouring periodic images,
in electrons per voxel.  Random numbers come from SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), written
out here so that a seed gives the same inputs on every machine and numpy
version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based 64-bit generator (golden-ratio increment + two xor-shift-multiply rounds)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def randint(self, n: int) -> int:
        """Integer in [0, n)."""
        return min(int(self.uniform() * n), n - 1)

    def normal(self) -> float:
        u1 = max(self.uniform(), 1e-300)
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# Unit cells
# ----------------------------------------------------------------------------

@dataclass
class Atom:
    frac: tuple  # fractional position (x, y, z) in the cell
    z: float     # electrons
    sigma: float  # Gaussian width, nm


def gaussian_cell(ucell: int, a_nm: float, atoms: list[Atom]) -> np.ndarray:
    """Periodic cubic cell of Gaussian atoms, float32 [z][y][x], electrons per voxel.

    Voxel v sits at v * a/U.  Each atom contributes
    Z (2 pi s^2)^(-3/2) exp(-|r - r_a - a n|^2 / 2 s^2) dx^3 summed over the
    27 images n in {-1,0,1}^3; the Gaussian factorises per axis, so the image
    sum is a product of three 1-D image sums.
    """
    dx = a_nm / ucell
    coords = np.arange(ucell, dtype=np.float64) * dx
    cell = np.zeros((ucell, ucell, ucell), dtype=np.float64)
    for at in atoms:
        s2 = 2.0 * at.sigma * at.sigma
        norm = at.z * (2.0 * math.pi * at.sigma * at.sigma) ** -1.5 * dx ** 3
        axes = []
        for ax in range(3):
            ra = at.frac[ax] * a_nm
            g = np.zeros(ucell, dtype=np.float64)
            for n in (-1, 0, 1):
                d = coords - ra - n * a_nm
                g += np.exp(-(d * d) / s2)
            axes.append(g)
        gx, gy, gz = axes
        cell += norm * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return cell.astype(np.float32)


def sc_cell(ucell: int = 16, a_nm: float = 1.0, z: float = 20.0, sigma: float = 0.08) -> np.ndarray:
    """Simple-cubic cell: one Gaussian atom at the cell origin."""
    return gaussian_cell(ucell, a_nm, [Atom((0.0, 0.0, 0.0), z, sigma)])


def mof_like_atoms(seed: int, natoms: int = 60, zs=(1.0, 6.0, 8.0, 30.0),
                   sigma_range=(0.05, 0.1)) -> list[Atom]:
    """Atoms at uniform fractional positions, Z uniform over `zs`, sigma uniform in range."""
    rng = SplitMix64(seed)
    atoms = []
    for _ in range(natoms):
        frac = (rng.uniform(), rng.uniform(), rng.uniform())
        zval = zs[rng.randint(len(zs))]
        sig = rng.uniform_range(*sigma_range)
        atoms.append(Atom(frac, zval, sig))
    return atoms


def mof_like_cell(ucell: int = 64, a_nm: float = 2.6, seed: int = 0, natoms: int = 60) -> np.ndarray:
    return gaussian_cell(ucell, a_nm, mof_like_atoms(seed, natoms))


# ----------------------------------------------------------------------------
# Shapes
# ----------------------------------------------------------------------------

SHAPE_SPHERE = 0
SHAPE_CUBE = 1
SHAPE_OCTAHEDRON = 2
SHAPE_ALL = 3       # no mask: every voxel inside
SHAPE_WEIGHTS = 4   # explicit per-voxel weight array

SHAPE_NAMES = {SHAPE_SPHERE: "sphere", SHAPE_CUBE: "cube", SHAPE_OCTAHEDRON: "octahedron",
               SHAPE_ALL: "all", SHAPE_WEIGHTS: "weights"}


@dataclass
class Shape:
    """Particle shape in voxel units.

    kind   : SHAPE_* code
    center : (cx, cy, cz) float32, voxel-index coordinates of the particle centre
    size   : float32; sphere radius, cube half-edge, or octahedron vertex distance
    rot    : 3x3 float32 row-major; body coordinates are p = rot^T d
    """
    kind: int
    center: tuple = (0.0, 0.0, 0.0)
    size: float = 0.0
    rot: np.ndarray = field(default_factory=lambda: np.eye(3, dtype=np.float32))

    def f32(self):
        c = np.asarray(self.center, dtype=np.float32)
        return c, np.float32(self.size), np.asarray(self.rot, dtype=np.float32).reshape(3, 3)


def random_rotation(rng: SplitMix64) -> np.ndarray:
    """Uniform random rotation from a uniform unit quaternion (Shoemake's subgroup method)."""
    u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    qw = a * math.sin(2 * math.pi * u2)
    qx = a * math.cos(2 * math.pi * u2)
    qy = b * math.sin(2 * math.pi * u3)
    qz = b * math.cos(2 * math.pi * u3)
    r = np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
    ], dtype=np.float64)
    return r.astype(np.float32)


def centred_sphere(n: int, radius_vox: float) -> Shape:
    c = float(n // 2)
    return Shape(SHAPE_SPHERE, (c, c, c), float(np.float32(radius_vox)))


# ----------------------------------------------------------------------------
# Bin edges (inputs to both sides, FP64)
# ----------------------------------------------------------------------------

def nyquist_q(dx_nm: float) -> float:
    return math.pi / dx_nm


def linear_edges(qmax: float, nbins: int) -> np.ndarray:
    return np.array([(j * qmax) / nbins for j in range(nbins + 1)], dtype=np.float64)


def log_edges(qlo: float, qhi: float, nbins: int) -> np.ndarray:
    r = qhi / qlo
    e = [qlo * r ** (j / nbins) for j in range(nbins)] + [qhi]
    return np.array(e, dtype=np.float64)


# ----------------------------------------------------------------------------
# Workloads (paper-shaped synthetic stand-ins)
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n: int                 # grid edge
    dx: float              # voxel edge, nm
    cell: np.ndarray       # float32 [U][U][U]
    shape: Shape
    edges: np.ndarray      # FP64 [B+1]
    origin: tuple = (0, 0, 0)
    ed_dtype: str = "f32"

    @property
    def ucell(self) -> int:
        return self.cell.shape[0]

    @property
    def nbins(self) -> int:
        return len(self.edges) - 1


def sc64_workload() -> Workload:
    """64^3 grid, simple-cubic 1 nm cell at 16^3, tiled 4x4x4, sphere radius 1.8 nm, 128 linear bins."""
    n, ucell, a = 64, 16, 1.0
    dx = a / ucell
    return Workload("sc64_sphere1.8nm_lin128", n, dx, sc_cell(ucell, a),
                    centred_sphere(n, 1.8 / dx), linear_edges(nyquist_q(dx), 128))


def mof_workload(n: int = 512, diameter_nm: float = 10.0, nbins: int = 512, seed: int = 0,
                 ucell: int = 64, a_nm: float = 2.6) -> Workload:
    """MOF-like 2.6 nm cell at 64^3 (dx 0.040625 nm) tiled over n^3 and cut by a sphere; log bins."""
    dx = a_nm / ucell
    dq = 2.0 * math.pi / (n * dx)
    return Workload(f"mof{n}_sphere{diameter_nm:g}nm_log{nbins}", n, dx, mof_like_cell(ucell, a_nm, seed),
                    centred_sphere(n, 0.5 * diameter_nm / dx), log_edges(dq, nyquist_q(dx), nbins))


def cube_merge_levels(n1: int = 1024, n_low: int = 512, factors=(4, 16), edge_nm: float = 20.0,
                      ucell: int = 128, a_nm: float = 2.5, nbins: int = 1000, qlo: float = 0.01,
                      qhi: float = 150.0, seed: int = 0):
    """Three-level workload: ED-1 fills an n1^3 box with a cube of edge `edge_nm`; ED-2/ED-3 are
    block sums by `factors`, centred in n_low^3 boxes; all levels share `nbins` log edges."""
    dx1 = edge_nm / n1
    cell = mof_like_cell(ucell, a_nm, seed)
    c = float(n1 // 2)
    shape = Shape(SHAPE_CUBE, (c, c, c), float(n1 // 2))
    edges = log_edges(qlo, qhi, nbins)
    ed1 = Workload(f"cube{edge_nm:g}nm_ed1_{n1}", n1, dx1, cell, shape, edges, ed_dtype="f16")
    return ed1, [(f, n_low, dx1 * f) for f in factors]


def smooth_even_sizes(lo: int, hi: int) -> list[int]:
    out = []
    for v in range(lo, hi + 1):
        if v % 2:
            continue
        r = v
        for p in (2, 3, 5, 7):
            while r % p == 0:
                r //= p
        if r == 1:
            out.append(v)
    return out


@dataclass
class Particle:
    n: int
    shape: Shape


def batch_particles(count: int = 64, seed: int = 7, lo: int = 96, hi: int = 384) -> list[Particle]:
    """Uneven-size particle batch: N uniform over the even {2,3,5,7}-smooth sizes in [lo, hi],
    shape uniform over sphere/cube/octahedron, circumscribed diameter U[0.25, 0.5]*N voxels,
    uniformly random orientation."""
    sizes = smooth_even_sizes(lo, hi)
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        n = sizes[rng.randint(len(sizes))]
        kind = (SHAPE_SPHERE, SHAPE_CUBE, SHAPE_OCTAHEDRON)[rng.randint(3)]
        rc = 0.5 * rng.uniform_range(0.25, 0.5) * n
        rot = random_rotation(rng)
        if kind == SHAPE_SPHERE:
            size = rc
        elif kind == SHAPE_CUBE:
            size = rc / math.sqrt(3.0)
        else:
            size = rc
        c = float(n // 2)
        out.append(Particle(n, Shape(kind, (c, c, c), float(np.float32(size)), rot)))
    return out


def sphere_target_curve(q: np.ndarray, radius_nm: float, contrast_electrons: float) -> np.ndarray:
    """Closed-form uniform-sphere intensity N_e^2 [3 (sin qR - qR cos qR)/(qR)^3]^2 (target for a loss)."""
    x = np.asarray(q, dtype=np.float64) * radius_nm
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(x > 1e-8, 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3, 1.0 - x * x / 10.0)
    return contrast_electrons ** 2 * f * f


def random_density(n: int, seed: int, nz_planes: tuple | None = None) -> np.ndarray:
    """Uniform [0,1) float32 density [z][y][x]; planes outside nz_planes=(z0, count) are zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = rng.random((n, n, n), dtype=np.float64).astype(np.float32)
    if nz_planes is not None:
        z0, cnt = nz_planes
        rho[:z0] = 0
        rho[z0 + cnt:] = 0
    return rho
