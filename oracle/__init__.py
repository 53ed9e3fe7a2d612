"""Plain, slow, CPU FP64 oracle for the wide-range scattering hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package.  The CUDA library never calls it
and shares no code with it.

Each function follows one passage of the paper (Pauw et al., "Ultima Ratio:
simulating wide-range X-ray scattering and diffraction", arXiv 2303.13435):

  density.py  Sec. 2.3 -- ED-1 by tiling the unit cell and masking it with the
              particle shape; ED-2/ED-3 by block integration and zero padding.
  scatter.py  Sec. 2.4 Eq. 1 -- the 3D DFT with 1/(MNL) normalisation, the
              intensity |F|^2; Sec. 2.5 -- isotropic averaging into Q bins.
  merge.py    Sec. 2.5 -- combining the level curves into one I(Q).
  adjoint.py  The gradient of a loss on binned I(Q) with respect to the unit
              cell and the mask weights (the plain chain rule through the above).

Readings of the paper where it is silent or ambiguous are stated in each
function's docstring.  Every function is pinned by the `not gpu` tests in
tests/test_oracle_pins.py to facts that do not come from the oracle itself.
"""
