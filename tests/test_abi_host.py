"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every function include/ur.h declares, and its host logic (bin thresholds,
integer division, argument validation, fault injection) is right."""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import scatter
from paper_2303_13435_gb300 import api, build, inputs


@pytest.fixture(scope="session", autouse=True)
def built_lib():
    build.build()
    return api.lib()


def test_exports_every_header_symbol():
    names = api.header_symbols()
    assert len(names) >= 15
    L = api.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) <= set(api.SIGNATURES)


def test_version_and_empty_error():
    assert b"sm_103a" in api.lib().ur_version()


def test_fastdiv_matches_integer_division():
    assert api.lib().ur_selftest_fastdiv() == 0


def test_butterflies_match_direct_dft():
    # radices 2..10, 16 and 32 of the FFT engines, forward and inverse, against a float64
    # direct DFT; FP32 butterflies with float64 twiddle constants stay within a
    # few ulp of the input norm
    err = api.lib().ur_selftest_dft()
    assert 0.0 <= err < 2e-6, err


@pytest.mark.parametrize("n,dx,kind", [(64, 0.0625, "lin"), (512, 0.040625, "log"), (96, 0.05, "log"),
                                       (16, 0.2, "tie")])
def test_thresholds_reproduce_oracle_bin_of_every_k2(n, dx, kind):
    """Sec. 2.5 bin assignment: the integer table gives, for every k^2 the grid has,
    exactly the bin the oracle's float64 |Q| comparison gives."""
    dq = 2 * math.pi / (n * dx)
    if kind == "lin":
        edges = inputs.linear_edges(inputs.nyquist_q(dx), 128)
    elif kind == "log":
        edges = inputs.log_edges(dq, inputs.nyquist_q(dx), 200)
    else:
        # edges exactly on lattice shells: q = dq * sqrt(s) for integer s (ties)
        edges = np.array([dq * math.sqrt(s) for s in (0, 1, 2, 3, 4, 5, 9, 16, 25, 50, 64)])
    t = api.bin_thresholds(n, dx, edges)
    smax = 3 * (n // 2) ** 2
    s = np.arange(smax + 1)
    want = scatter.bin_of_q(scatter.q_of_k2(s, n, dx), edges)
    nb = len(edges) - 1
    got = np.searchsorted(t, s, side="right") - 1
    got = np.where((got >= 0) & (got < nb), got, -1)
    assert np.array_equal(got, want)


def test_plan_create_rejects_bad_sizes_before_touching_the_gpu():
    for n in (7, 6, 22, 8192):
        with pytest.raises(api.UrError) as e:
            api.Plan(n, 0.1, np.array([0.0, 1.0]))
        assert e.value.status == 1
    with pytest.raises(api.UrError):
        api.Plan(64, 0.1, np.array([1.0, 1.0]))   # edges not increasing
    with pytest.raises(api.UrError):
        api.Plan(64, 0.1, np.array([0.0, 1.0]), z0=60, nz=10)   # slab outside the grid


def test_fault_injection_fires_on_the_host():
    code = (
        "import numpy as np\n"
        "from paper_2303_13435_gb300 import api\n"
        "try:\n"
        "    api.Plan(64, 0.1, np.array([0.0, 1.0]))\n"
        "except api.UrError as e:\n"
        "    print('STATUS', e.status)\n"
    )
    env = dict(os.environ, UR_FAULT="plan_create:1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert "STATUS 6" in r.stdout, r.stdout + r.stderr
