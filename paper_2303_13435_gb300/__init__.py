"""GB300-native wide-range X-ray scattering hot path ("Ultima Ratio", arXiv 2303.13435).

The compute path is the CUDA C-ABI library built from csrc/ (libur.so); this
package holds its thin ctypes binding (`api`), the autograd wrapper (`autograd`)
and the seeded input generators (`inputs`).  Importing the package does not load
the library; `api` loads it on first use and raises if it is missing.
"""

__all__ = ["inputs", "api", "autograd"]
