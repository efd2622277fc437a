"""lqcd_apply_Mhat_noalloc: Mhat for callers that cannot let the library allocate.

Applications that give all device memory to their own pool (a caching
allocator or a fixed arena) or that cannot accept the device synchronisation
of cudaMalloc call this variant; its odd temporary is a fixed 16 MiB array
built into the library. This file is collected last on purpose. The entry
point launches the same kernels with the same coefficients as lqcd_apply_Mhat,
so each result must equal lqcd_apply_Mhat's bit for bit: checked through the C
ABI on two calls in a row (different inputs, kappa and dagger) for every
spinor precision with 18- and 12-real gauge fields, including double-float
fields of a 12-real gauge (whose links keep 18 reals). Oversized lattices and a
non-finite kappa are refused with clear errors.
"""
import numpy as np
import pytest

from paper_1112_5280_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu

DIMS = (16, 16, 16, 32)  # the benchmark lattice: FP64 odd temporary 12.6 MB of the 16 MiB


@pytest.fixture(scope="module")
def links():
    return synth.random_links(DIMS, 0.5, seed=1001)


@pytest.mark.parametrize("prec,compress", [("f32", 18), ("f32", 12), ("f64", 18), ("f64", 12),
                                           ("f16", 12), ("bf16", 12), ("df64", 18), ("df64", 12)])
def test_apply_Mhat_noalloc_matches_apply_Mhat(links, prec, compress):
    ctx = lqcd.Context(0)
    g = ctx.gauge(DIMS, links, prec=prec, compress=compress)
    even = synth.parity_of_sites(DIMS) == 0
    for call, (seed, kappa, dag) in enumerate([(2002, 0.15, False), (2003, 0.155, True)]):
        psi = synth.gaussian_spinor(DIMS, seed=seed)
        fin = ctx.field(DIMS, prec, lqcd.EVEN, data=psi)
        ref_f = ctx.field(DIMS, prec, lqcd.EVEN)
        out_f = ctx.field(DIMS, prec, lqcd.EVEN)
        lqcd.apply_Mhat(g, kappa, fin, ref_f, dagger=dag)
        lqcd.apply_Mhat_noalloc(g, kappa, fin, out_f, dagger=dag)
        ref = ref_f.download()[even]
        got = out_f.download()[even]
        assert np.abs(ref).max() > 0.5, (call, "reference is not a real result")
        assert np.array_equal(got, ref), (prec, compress, call, np.abs(got - ref).max())
        for f_ in (fin, ref_f, out_f):
            f_.close()
    g.close()
    ctx.close()


def test_apply_Mhat_noalloc_refuses_bad_arguments():
    ctx = lqcd.Context(0)
    dims = (24, 24, 24, 48)  # FP32 half spinor 31.9 MB > 16 MiB
    g = ctx.gauge(dims, synth.unit_links(dims), prec="f32", compress=18)
    fin = ctx.field(dims, "f32", lqcd.EVEN)
    fout = ctx.field(dims, "f32", lqcd.EVEN)
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.apply_Mhat_noalloc(g, 0.15, fin, fout)
    assert e.value.code == lqcd.EINVAL and "scratch" in str(e.value)
    small = (4, 4, 4, 4)
    g2 = ctx.gauge(small, synth.unit_links(small), prec="f32", compress=18)
    a = ctx.field(small, "f32", lqcd.EVEN)
    b = ctx.field(small, "f32", lqcd.EVEN)
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.apply_Mhat_noalloc(g2, float("nan"), a, b)
    assert e.value.code == lqcd.EINVAL and "kappa" in str(e.value)
    ctx.close()
