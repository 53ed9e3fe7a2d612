"""Pins against the numbers the paper prints for its MOF demonstration.

tests/golden/paper_geometry.txt holds those numbers with the passage that
states each.  The tests check that the fixture is a consistent reading of the
paper, and that the oracle's Q arithmetic, its merge windows and its plane
range, with the library's level limit, reproduce the paper's statements on
that geometry.  The CUDA path is not involved.
"""
import math
import os

import numpy as np
import pytest

from oracle import density, merge, scatter
from paper_2303_13435_gb300 import api, inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_geometry.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, value = line.split()[:2]
            vals[key] = float(value)
    return vals


G = _golden()


def _levels():
    """(grid edge, voxel step in nm) of ED-1, ED-2 and ED-3 of the paper's demonstration."""
    dx1 = G["particle_diameter_nm"] / G["ed1_particle_voxels"]
    return [(int(G["ed1_box_voxels"]), dx1),
            (int(G["ed23_box_voxels"]), dx1 * G["ed2_zoom"]),
            (int(G["ed23_box_voxels"]), dx1 * G["ed3_zoom"])]


def test_fixture_is_a_consistent_reading_of_the_paper():
    # Sec. 2.3 para 1: 630 / 6 = 105 voxels, and 1.683 nm / 105 is the printed 0.16 Angstrom step
    assert G["unit_cell_voxels_dft"] / G["unit_cell_reduction"] == G["unit_cell_voxels"]
    step_a = 10.0 * G["unit_cell_edge_nm"] / G["unit_cell_voxels"]
    assert round(step_a, 2) == G["voxel_step_angstrom"]
    # the 64 nm particle over 4000 voxels is sampled at that step (0.2 % apart)
    dx1 = _levels()[0][1]
    assert abs(10.0 * dx1 - step_a) / step_a < 2e-3
    # Sec. 2.3 para 4: 4000 / 16 = 250 and 4000 / 125 = 32; the particle is 64 nm at every level
    assert G["ed1_particle_voxels"] / G["ed2_zoom"] == G["ed2_particle_voxels"]
    assert G["ed1_particle_voxels"] / G["ed3_zoom"] == G["ed3_particle_voxels"]
    for (n, dx), vox in zip(_levels(), ("ed1_particle_voxels", "ed2_particle_voxels", "ed3_particle_voxels")):
        assert G[vox] * dx == pytest.approx(G["particle_diameter_nm"], rel=1e-12)
        # the object fills at most half of each box edge (Sec. 2.3 para 4)
        assert 2 * G[vox] <= n
    # zeros not written: (8000 / 4000)^3
    assert (G["ed1_box_voxels"] / G["ed1_particle_voxels"]) ** 3 == G["io_saving_factor"]


def test_q_range_of_the_three_levels():
    """Abstract: the curve spans Q < 0.01 nm^-1 to about 150 nm^-1; Fig. 2 caption:
    artefacts appear beyond Q_max / 2."""
    (n1, dx1), (n2, dx2), (n3, dx3) = _levels()
    # the axis Nyquist |Q| of ED-1 from the oracle's Q of k^2 = (N/2)^2 is half the sampling
    # frequency 2 pi / dx, and it is the limit the library and the workloads use
    q_ny = float(scatter.q_of_k2(np.array([(n1 // 2) ** 2], dtype=np.int64), n1, dx1)[0])
    assert q_ny == pytest.approx(G["artefact_fraction_of_qmax"] * 2.0 * math.pi / dx1, rel=1e-12)
    assert api.level_qmax(dx1) == pytest.approx(q_ny, rel=1e-12)
    assert inputs.nyquist_q(dx1) == pytest.approx(q_ny, rel=1e-12)
    # the printed reach lies inside ED-1's trusted range, and not by a factor of 2 pi
    assert G["q_high_approx_per_nm"] < q_ny < 2.0 * G["q_high_approx_per_nm"]
    # the lowest nonzero |Q| (k^2 = 1): ED-3 reaches below 0.01 nm^-1, ED-2 does not
    q3 = float(scatter.q_of_k2(np.array([1], dtype=np.int64), n3, dx3)[0])
    q2 = float(scatter.q_of_k2(np.array([1], dtype=np.int64), n2, dx2)[0])
    assert q3 == pytest.approx(scatter.dq_of(n3, dx3), rel=1e-15)
    assert q3 < G["q_low_below_per_nm"] < q2


def test_merge_windows_on_the_paper_geometry():
    """Sec. 2.5: the level curves are merged; each level is trusted up to Q_max/2 = pi/dx."""
    lv = _levels()
    q = np.array([0.002, 0.005, 1.0, 5.0, 50.0, G["q_high_approx_per_nm"], 190.0, 250.0])
    edges = np.sort(np.concatenate([q / 1.001, q * 1.001]))
    nb = len(edges) - 1
    levels = [{"n": n, "dx": dx, "count": np.ones(nb, dtype=np.int64), "mean": np.zeros(nb),
               "sem": np.zeros(nb), "mean_q": np.zeros(nb)} for n, dx in lv]
    out = merge.merge_levels(levels, edges)
    src = out["source"][0::2]  # the bins centred on q
    # ED-3 below pi/dx3 = 1.57, ED-2 up to pi/dx2 = 12.3, ED-1 up to pi/dx1 = 196; beyond it none
    assert src.tolist() == [2, 2, 2, 1, 0, 0, 0, -1]


def test_nonzero_planes_of_a_half_box_sphere():
    """Sec. 2.4 para 3: transforming only the planes with density saves a factor of two
    when the particle spans half of the box edge (Sec. 2.3 para 4)."""
    n = 64
    sh = inputs.centred_sphere(n, n / 4)
    rho = density.shape_mask(n, sh.kind, sh.center, sh.size, sh.rot)
    z0, z1 = density.nonzero_plane_range(rho)
    planes = z1 - z0 + 1
    assert planes in (n // 2, n // 2 + 1)
    assert n / planes == pytest.approx(G["plane_saving_factor"], rel=0.05)
