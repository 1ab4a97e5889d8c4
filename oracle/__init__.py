"""FTLM oracle: a plain, slow, FP64 CPU implementation of the FTLM hot path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It shares no
code with the CUDA library and never imports it.

Parts:
  ftlm_oracle.c  basis, full lookup table, CLT arrays (Eq. 18), H.v (Eq. 12-14),
                 counter-based start vectors, Lanczos recurrence (FP64).
  ftlm.py        ctypes wrapper, tridiagonal eigenproblem (numpy eigh on the dense
                 T), thermodynamic sums (Eq. 4-9), the full FTLM driver.
  counting.py    index <-> label by the counting argument, and single rows of H.v,
                 for sectors too large to enumerate (sampled-row checks).
  spin.py        general local spin s: Eq. 15 dimensions, Eq. 10 N_nz, base-d
                 basis, H.v (Eq. 12-14), Lanczos and the FTLM driver.
  diagnostics.py FP32 diagnostics: Cullum-Willoughby ghosts and clusters (Eq. 25),
                 sigma_emp (Eq. 22).
"""
from .ftlm import *  # noqa: F401,F403
from . import counting  # noqa: F401
from . import spin  # noqa: F401
from . import diagnostics  # noqa: F401
