"""FP64 CPU oracle for the NUFFT Radon / MBIR hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  It shares no code with
the CUDA library under ``paper_2304_12934_gb300/`` and never imports it.

Contents
--------
``radon_oracle.c``  exact NUDFT forward/adjoint Radon (Sec. 2, Eqs. fourier_sum,
                    nufft, fourier_radon; Sec. 3 Eq. transpose), plus the
                    Dirichlet closed form used for sampled entries.
``core.py``         ctypes binding, the qGGMRF prior (Sec. 3 Eqs. reg2/reg3), the
                    data-fidelity gradient (Sec. 3 Eqs. objfn/gradient), power
                    iteration and the accelerated-gradient loop with restart
                    (Sec. 3, last paragraph).

Parity pins: every function here is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, exact special cases, brute force on tiny inputs and
invariants.  The iteration schedule of ``mbir_solve`` beyond those invariants
is "parity unpinned" by the paper (it prints no iterate values and leaves the
optimizer variant open), see ``core.mbir_solve``.
"""
from .core import *  # noqa: F401,F403
