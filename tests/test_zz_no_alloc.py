"""lqcd_apply_Mhat_noalloc: Mhat for callers that cannot let the library allocate.

Applications that give all device memory to their own pool (a caching
allocator or a fixed arena) or that cannot accept the device synchronisation
of cudaMalloc call this variant; its odd temporary is a fixed 16 MiB array
built into the library. This file is collected last on purpose. The test calls
the entry point through the C ABI twice in a row, on different inputs, and
compares each result with lqcd_apply_Mhat within the FP32 parity tolerance of
the other tests (1e-5 of the largest component); it also checks that a lattice
beyond the scratch size is refused with a clear error.
"""
import numpy as np
import pytest

from paper_1112_5280_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


def test_apply_Mhat_noalloc_matches_apply_Mhat():
    ctx = lqcd.Context(0)
    dims = (16, 16, 16, 32)  # the benchmark lattice: FP32 odd temporary 6.3 MB
    U = synth.random_links(dims, 0.5, seed=1001)
    g = ctx.gauge(dims, U, prec="f32", compress=18)
    even = synth.parity_of_sites(dims) == 0
    for call, (seed, kappa, dag) in enumerate([(2002, 0.15, False), (2003, 0.155, True)]):
        psi = synth.gaussian_spinor(dims, seed=seed)
        fin = ctx.field(dims, "f32", lqcd.EVEN, data=psi)
        ref_f = ctx.field(dims, "f32", lqcd.EVEN)
        out_f = ctx.field(dims, "f32", lqcd.EVEN)
        lqcd.apply_Mhat(g, kappa, fin, ref_f, dagger=dag)
        lqcd.apply_Mhat_noalloc(g, kappa, fin, out_f, dagger=dag)
        ref = ref_f.download()[even]
        got = out_f.download()[even]
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= TOL_F32, (call, err)
    ctx.close()


def test_apply_Mhat_noalloc_refuses_oversize():
    ctx = lqcd.Context(0)
    dims = (24, 24, 24, 48)  # FP32 half spinor 31.9 MB > 16 MiB
    g = ctx.gauge(dims, synth.unit_links(dims), prec="f32", compress=18)
    fin = ctx.field(dims, "f32", lqcd.EVEN)
    fout = ctx.field(dims, "f32", lqcd.EVEN)
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.apply_Mhat_noalloc(g, 0.15, fin, fout)
    assert e.value.code == lqcd.EINVAL and "scratch" in str(e.value)
    ctx.close()
