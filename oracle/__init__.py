"""FP64 CPU oracle for the CheFSI hot path (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may
import this package. The CUDA library never loads it and shares no code with it.

Pinned functions and their pins are listed in tests/test_oracle_pins.py; no function
here is "parity unpinned".
"""
from .oracle import *  # noqa: F401,F403
from .oracle import (Hamiltonian, Projectors, NotSPD, lap_weights, lap_weights_exact,  # noqa: F401
                     laplacian, veff, projectors, lanczos_start, orth_rr, fix_signs,
                     chefsi_step, chefsi_solve, chefsi_first_bounds, chefsi_next_bounds, lib)
