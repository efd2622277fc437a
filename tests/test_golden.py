"""The oracle against its golden fixtures (tests/golden, written by make_golden.py).

The paper prints no worked example, so these fixtures are the oracle's own results on
seeded inputs: they freeze it, so that any later change to its arithmetic shows up here
(and must name the passage or reading that justifies it). Tolerances: the hopping term
and Mhat are site-local and deterministic (1e-14); the CG solution, the heatbath chain
and the trajectory go through reductions or libm calls whose last bits may differ across
thread counts and platforms, amplified by the updates (1e-9).
"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_golden as mg  # noqa: E402


@pytest.mark.parametrize("spec,fn,tol", [(mg.HOP, mg.hop_values, 1e-14), (mg.MHAT, mg.mhat_values, 1e-14),
                                         (mg.SOLVE, mg.solve_values, 1e-9),
                                         (mg.HEATBATH, mg.heatbath_values, 1e-9),
                                         (mg.HMC, mg.hmc_values, 1e-9)],
                         ids=["hop", "mhat_tm", "solve", "heatbath", "hmc"])
def test_oracle_matches_golden(spec, fn, tol):
    want = mg.read(spec[0])
    got = np.asarray(fn(), dtype=complex).ravel()
    assert got.shape == want.shape
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= tol * scale, np.abs(got - want).max() / scale
