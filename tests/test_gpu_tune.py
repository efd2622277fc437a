"""The launch autotuner: choices are valid, results do not depend on them, the table
survives a save/load round trip.

The persistent grid only changes which CTA handles which tile; per-site arithmetic and
the per-tile reduction order are fixed, so operators and whole solves must be bitwise
the same before and after tuning.
"""
import numpy as np
import pytest

from paper_1112_5280_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = lqcd.Context(0)
    yield c
    c.close()


@pytest.fixture(autouse=True)
def clean_table():
    lqcd.tune_clear()
    yield
    lqcd.tune_clear()


def _mhat(ctx, g, dims, psi, prec, kappa=0.15, mu=0.0):
    fin = ctx.field(dims, prec, lqcd.EVEN, data=psi)
    fout = ctx.field(dims, prec, lqcd.EVEN)
    lqcd.apply_Mhat(g, kappa, fin, fout, mu=mu)
    return fout.download()


@pytest.mark.parametrize("prec,compress", [("f32", 18), ("f16", 12), ("df64", 18)])
def test_tuned_choice_is_valid_and_results_unchanged(ctx, prec, compress):
    dims = (8, 8, 8, 16)
    U = synth.random_links(dims, 0.5, seed=91)
    psi = synth.gaussian_spinor(dims, seed=92)
    g = ctx.gauge(dims, U, prec=prec, compress=compress)
    before = _mhat(ctx, g, dims, psi, prec)
    r = lqcd.autotune_dslash([g] * 4, prec)
    assert r["prec"] == lqcd.PRECISIONS[prec] and r["nr"] == compress
    assert r["ntiles"] == 4 * (np.prod(dims) // 2 // 64)
    assert r["candidates"] >= 1 and r["us_best"] > 0 and r["us_default"] > 0
    assert r["us_best"] <= r["us_default"] * 1.0000001
    assert 0 <= r["ctas_per_sm"] <= 32 and r["form"] in (0, 1)
    if prec == "df64":
        assert r["candidates"] >= 2  # both kernel forms were timed
    # force a non-default choice for the single-slot launch size and compare bitwise
    single = lqcd.autotune_dslash([g], prec)
    assert single["ntiles"] == np.prod(dims) // 2 // 64
    after = _mhat(ctx, g, dims, psi, prec)
    assert np.array_equal(before, after)


def test_solve_bitwise_independent_of_grid(ctx):
    """A mixed-precision solve gives the same bits with the default grid, a tuned grid and a
    one-CTA-per-SM grid."""
    dims = (8, 8, 8, 8)
    U = synth.random_links(dims, 0.5, seed=93)
    b = synth.gaussian_spinor(dims, seed=94)
    g = ctx.gauge(dims, U, prec="f64")
    opts = lqcd.solve_opts(sloppy_prec="f16")
    x0, i0 = lqcd.solve(g, b, 0.15, 1e-10, opts)
    g16 = ctx.gauge(dims, U, prec="f16", compress=12)
    lqcd.autotune_dslash([g16], "f16")
    x1, i1 = lqcd.solve(g, b, 0.15, 1e-10, opts)
    lqcd.set_grid_multiplier(0, 1)
    try:
        x2, i2 = lqcd.solve(g, b, 0.15, 1e-10, opts)
    finally:
        lqcd.set_grid_multiplier(0, 0)
    assert i0["status"] == i1["status"] == i2["status"] == 0
    assert i0["iters"] == i1["iters"] == i2["iters"]
    assert np.array_equal(x0, x1) and np.array_equal(x0, x2)


def test_save_load_round_trip(ctx, tmp_path):
    dims = (4, 4, 4, 8)
    g = ctx.gauge(dims, synth.random_links(dims, 0.5, seed=95), prec="f32")
    lqcd.autotune_dslash([g, g], "f32")
    lqcd.autotune_dslash([g], "f32")
    table = lqcd.tune_entries()
    assert len(table) == 2
    path = tmp_path / "tune.txt"
    lqcd.tune_save(path)
    lqcd.tune_clear()
    assert lqcd.tune_entries() == []
    lqcd.tune_load(path)
    got = lqcd.tune_entries()
    key = lambda e: (e["prec"], e["nr"], e["ntiles"])  # noqa: E731
    assert len(got) == 2
    for a, b in zip(sorted(got, key=key), sorted(table, key=key)):
        assert a["ctas_per_sm"] == b["ctas_per_sm"] and a["form"] == b["form"]
        assert a["ntiles"] == b["ntiles"] and abs(a["us_best"] - b["us_best"]) < 1e-2


def test_load_rejects_foreign_and_malformed_files(ctx, tmp_path):
    bad = tmp_path / "other.txt"
    bad.write_text("lqcd-tune 1 SomeOtherGPU_sm80\ndslash 1 18 5 40 0 0 3 10.0 10.0\n")
    with pytest.raises(lqcd.LqcdError):
        lqcd.tune_load(bad)
    dims = (4, 4, 4, 8)
    g = ctx.gauge(dims, synth.random_links(dims, 0.5, seed=96), prec="f32")
    lqcd.autotune_dslash([g], "f32")
    good = tmp_path / "good.txt"
    lqcd.tune_save(good)
    header = good.read_text().splitlines()[0]
    broken = tmp_path / "broken.txt"
    broken.write_text(header + "\ndslash 1 18 5 40 0 7 3 10.0 10.0\n")  # form 7 does not exist
    lqcd.tune_clear()
    with pytest.raises(lqcd.LqcdError):
        lqcd.tune_load(broken)
    assert lqcd.tune_entries() == []
    with pytest.raises(lqcd.LqcdError):
        lqcd.tune_load(tmp_path / "missing.txt")
