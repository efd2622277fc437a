"""GPU meson correlators (paper Section 4, eq. 4.1) vs the oracle contraction.

The 12 point-source propagators come from the GPU multi-RHS solve; the GPU
contraction of those fields equals the oracle's contraction of the same
fields to 1e-12 (relative to the largest |C|), and the oracle's contraction of
its own solutions to 1e-8 (the solves' tolerance).
"""
import numpy as np
import pytest

import oracle
from oracle import contract
from paper_1112_5280_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(6, 6, 4, 6), (4, 4, 4, 8)])
def test_meson_correlator_matches_oracle(dims):
    ctx = lqcd.Context(0)
    U = synth.random_links(dims, 0.5, seed=11)
    kappa = 0.14
    site = synth.point_site(dims)
    g = ctx.gauge(dims, U, prec="f64")
    srcs_h = [synth.point_source(dims, site, s, c) for s in range(4) for c in range(3)]
    srcs = [ctx.field(dims, "f64", lqcd.FULL, data=b) for b in srcs_h]
    xs = [ctx.field(dims, "f64", lqcd.FULL) for _ in srcs]
    infos = lqcd.solve_multi(g, srcs, kappa, 1e-12, xs, lqcd.solve_opts(sloppy_prec="f32"))
    assert all(i["status"] == 0 for i in infos)
    codes = list(range(10))
    c_gpu = lqcd.meson_correlator(xs, codes)
    sols = [x.download() for x in xs]
    c_ref = contract.meson_correlator(dims, sols, codes)
    scale = np.abs(c_ref).max()
    assert np.abs(c_gpu - c_ref).max() < 1e-12 * scale
    osols = [oracle.solve(dims, U, kappa, b, tol=1e-12)[0] for b in srcs_h]
    c_or = contract.meson_correlator(dims, osols, codes)
    assert np.abs(c_gpu - c_or).max() < 1e-8 * scale
    ctx.close()
