"""FP64 CPU oracle for the Wilson-Dirac fermion matrix (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package. It shares no code with the CUDA library; both sides take their
inputs from the seeded generators in paper_1112_5280_gb300.synth.

Contents
  * ctypes bindings to the C oracle (wilson_oracle.c): hopping term, M, Mhat,
    CG on the normal equations, even-odd CG and BiCGStab.
  * dense.py: brute-force dense matrices for tiny lattices (pure Python loops),
    the free-field closed forms and the FFT solve of the free field.
  * contract.py: the meson correlator of eq. 4.1.
  * hmc.py: HMC for N_f = 2 (twisted-mass) Wilson fermions with even-odd
    preconditioning: actions, gauge and fermion forces, leapfrog and 2MN integrators.
  * gauge.py: bindings to heatbath.c, the SU(3) heatbath (Cabibbo-Marinari with
    Creutz's SU(2) draw, Philox4x64-10 random numbers) and the plaquette.
"""
from .wilson import (  # noqa: F401
    apply_M,
    apply_Mhat,
    get_threads,
    hop,
    hop_eo,
    hop_sites,
    set_threads,
    solve,
    true_residual,
    METHOD_CG_FULL,
    METHOD_CG_EO,
    METHOD_BICGSTAB_EO,
)
