"""The bounds-checked debug build (a sanitizer substitute; compute-sanitizer is not used).

Built with -DLQCD_DEBUG_BOUNDS, every spinor and link access of the batched kernels checks
its site index against the field and records the first index outside (no trap). The
debug build must give the oracle's results and record nothing on the library's own
workloads: ragged lattices with partial last tiles, coinciding neighbours (L = 2), batches
of mixed sizes, Mhat and mixed-precision solves. It runs in a child process, which loads
the debug library (LQCD_DEBUG_BOUNDS=1) and builds it first if needed. The normal build
refuses the query.
"""
import os
import subprocess
import sys
import textwrap

import pytest

from paper_1112_5280_gb300 import lqcd

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import numpy as np
    import oracle
    from paper_1112_5280_gb300 import lqcd, synth
    ctx = lqcd.Context(0)
    tol = {"f64": 1e-12, "f32": 1e-5, "f16": 4e-3, "df64": 1e-12}
    shapes = [(6, 6, 4, 10), (2, 2, 2, 2), (2, 4, 6, 4)]
    for prec in ("f64", "f32", "f16", "df64"):
        gs, fis, fos, refs = [], [], [], []
        for k, dims in enumerate(shapes):
            U = synth.random_links(dims, 0.5, seed=700 + k)
            psi = synth.gaussian_spinor(dims, seed=800 + k)
            g = ctx.gauge(dims, U, prec=prec, compress=12 if prec == "f16" else 18)
            fi = ctx.field(dims, prec, lqcd.FULL, data=psi)
            fo = ctx.field(dims, prec, lqcd.FULL)
            for p in (0, 1):
                lqcd.dslash_eo(g, fi, fo, p, dagger=(p == 1))
            ref = np.where((synth.parity_of_sites(dims) == 0)[:, None, None],
                           oracle.hop(dims, U, psi), oracle.hop(dims, U, psi, dagger=True))
            out = fo.download()
            assert np.abs(out - ref).max() / np.abs(ref).max() < tol[prec], (prec, dims)
            gs.append(g); fis.append(fi); fos.append(fo)
            refs.append((dims, U, psi))
        b = lqcd.DslashBatch(gs, fis, fos, 0)
        b.apply()
        for fo, (dims, U, psi) in zip(fos, refs):
            ev = synth.parity_of_sites(dims) == 0
            ref = oracle.hop(dims, U, psi)[ev]
            assert np.abs(fo.download()[ev] - ref).max() / np.abs(ref).max() < tol[prec]
        b.close()
        dims, U, psi = refs[0]
        me = ctx.field(dims, prec, lqcd.EVEN)
        lqcd.apply_Mhat(gs[0], 0.13, fis[0], me)
    dims = (6, 6, 4, 10)
    U = synth.random_links(dims, 0.5, seed=901)
    b = synth.gaussian_spinor(dims, seed=902)
    g = ctx.gauge(dims, U)
    for sp in ("f16", "f32"):
        x, info = lqcd.solve(g, b, 0.14, 1e-10, lqcd.solve_opts(sloppy_prec=sp))
        assert info["status"] == 0 and oracle.true_residual(dims, U, 0.14, b, x) <= 1e-10
    print("bounds", ctx.debug_bounds())
    ctx.close()
""")


def test_debug_build_records_nothing_and_matches_oracle():
    env = dict(os.environ, LQCD_DEBUG_BOUNDS="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1500)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "bounds None" in r.stdout, r.stdout[-2000:]


def test_normal_build_refuses_the_query():
    ctx = lqcd.Context(0)
    with pytest.raises(lqcd.LqcdError) as e:
        ctx.debug_bounds()
    assert e.value.code == lqcd.EINVAL and "LQCD_DEBUG_BOUNDS" in str(e.value)
    ctx.close()
