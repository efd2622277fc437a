"""The launch autotuner: choices are valid, results do not depend on them, the table
survives a save/load round trip.

The persistent grid only changes which CTA handles which tile; per-site arithmetic and
the per-tile reduction order are fixed, so operators and whole solves must be bitwise
the same before and after tuning.
"""
import json

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
    assert 0 <= r["ctas_per_sm"] <= 32 and r["form"] in ((0, 3) if prec == "f32" else (0, 1))
    if prec in ("df64", "f32"):
        assert r["candidates"] >= 2  # both kernel forms (register budgets) were timed
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
    lqcd.autotune_dslash([g, g], "f32")  # own-link entry of 2 slots and the shared-link entry
    lqcd.autotune_dslash([g], "f32")
    table = lqcd.tune_entries()
    assert len(table) == 3 and sum(e["nrhs"] == 2 for e in table) == 1
    path = tmp_path / "tune.json"
    lqcd.tune_save(path)
    doc = json.loads(path.read_text())
    assert doc["format"] == "lqcd-tune" and doc["version"] == 2 and len(doc["entries"]) == 3
    lqcd.tune_clear()
    assert lqcd.tune_entries() == []
    lqcd.tune_load(path)
    got = lqcd.tune_entries()
    key = lambda e: (e["prec"], e["nr"], e["nrhs"], e["ntiles"])  # noqa: E731
    assert len(got) == 3
    for a, b in zip(sorted(got, key=key), sorted(table, key=key)):
        assert a["ctas_per_sm"] == b["ctas_per_sm"] and a["form"] == b["form"] and a["group"] == b["group"]
        assert a["ntiles"] == b["ntiles"] and abs(a["us_best"] - b["us_best"]) < 1e-2


def _device_tag(ctx, tmp_path):
    dims = (4, 4, 4, 8)
    g = ctx.gauge(dims, synth.unit_links(dims), prec="f32")
    lqcd.autotune_dslash([g], "f32")
    p = tmp_path / "tag.json"
    lqcd.tune_save(p)
    lqcd.tune_clear()
    return json.loads(p.read_text())["device"]


def _entry(**kw):
    e = {"prec": 1, "nr": 18, "nrhs": 0, "bucket": 5, "ntiles": 40, "ctas_per_sm": 0, "form": 0,
         "group": 0, "candidates": 3, "us_best": 10.0, "us_default": 10.0}
    e.update(kw)
    return e


@pytest.mark.parametrize("compress", [12, 18])
def test_second_register_budget_is_bitwise_the_default(ctx, tmp_path, compress):
    """Form 3 (the FP32 Dslash compiled for 8 CTAs per SM) runs the same site arithmetic in
    the same order: M-hat and a whole solve are bitwise those of the default form."""
    dims = (8, 8, 8, 16)  # 64 tiles per half lattice: bucket 6
    U = synth.random_links(dims, 0.5, seed=93)
    psi = synth.gaussian_spinor(dims, seed=94)
    g = ctx.gauge(dims, U, prec="f32", compress=compress)
    g64 = ctx.gauge(dims, U, prec="f64")
    b = ctx.field(dims, "f64", lqcd.FULL, data=psi)
    o = lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=compress)

    def run():
        x = ctx.field(dims, "f64", lqcd.FULL)
        info = lqcd.solve_fields(g64, b, 0.15, 1e-10, x, o)
        out = x.download()
        x.close()
        return _mhat(ctx, g, dims, psi, "f32"), out, info["iters"]

    ref = run()
    tag = _device_tag(ctx, tmp_path)
    p = tmp_path / "hi.json"
    p.write_text(json.dumps({"format": "lqcd-tune", "version": 2, "device": tag, "entries": [
        _entry(prec=1, nr=compress, bucket=6, ntiles=64, form=3)]}))
    lqcd.tune_load(p)
    assert [e["form"] for e in lqcd.tune_entries()] == [3]
    got = run()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]) and ref[2] == got[2]


def test_load_rejects_foreign_and_malformed_files(ctx, tmp_path):
    tag = _device_tag(ctx, tmp_path)

    def doc(entries, device=tag, version=2):
        return json.dumps({"format": "lqcd-tune", "version": version, "device": device, "entries": entries})

    cases = {
        "other_device": doc([_entry()], device="SomeOtherGPU_sm80"),
        "old_version": doc([_entry()], version=1),
        "no_such_form": doc([_entry(form=7)]),
        "shared_form_without_rhs": doc([_entry(form=2, group=2)]),
        "group_beyond_rhs": doc([_entry(nrhs=4, bucket=3, form=2, group=6)]),
        "second_budget_not_fp32": doc([_entry(prec=2, nr=12, form=3)]),
        "missing_field": doc([{k: v for k, v in _entry().items() if k != "ctas_per_sm"}]),
        "truncated": doc([_entry()])[:-3],
        "text_format": "lqcd-tune 1 " + tag + "\ndslash 1 18 5 40 0 0 3 10.0 10.0\n",
    }
    ok = tmp_path / "ok.json"
    ok.write_text(doc([_entry(), _entry(nrhs=4, bucket=3, form=2, group=2)]))
    lqcd.tune_load(ok)
    assert len(lqcd.tune_entries()) == 2
    for name, text in cases.items():
        lqcd.tune_clear()
        p = tmp_path / f"{name}.json"
        p.write_text(text)
        with pytest.raises(lqcd.LqcdError):
            lqcd.tune_load(p)
        assert lqcd.tune_entries() == [], name
    with pytest.raises(lqcd.LqcdError):
        lqcd.tune_load(tmp_path / "missing.json")


def test_shared_link_group_size_does_not_change_results(ctx, tmp_path):
    """12 point sources on one gauge field: the solutions are the same bit for bit whether
    every source loads its own links, or the tuner's (or a loaded table's) group of sources
    shares each site block's link loads, whatever the group size."""
    dims = (8, 8, 8, 16)  # 64 site blocks: the engine's own rule keeps own links here
    U = synth.random_links(dims, 0.5, seed=97)
    g = ctx.gauge(dims, U, prec="f64")
    site = synth.point_site(dims)
    srcs = [ctx.field(dims, "f64", lqcd.FULL, data=synth.point_source(dims, site, s_, c_))
            for s_ in range(4) for c_ in range(3)]
    opts = lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=12)

    def run():
        xs = [ctx.field(dims, "f64", lqcd.FULL) for _ in srcs]
        infos = lqcd.solve_multi(g, srcs, 0.15, 1e-10, xs, opts)
        assert all(i["status"] == 0 for i in infos)
        out = [x.download() for x in xs]
        for x in xs:
            x.close()
        return out

    ref = run()
    tag = _device_tag(ctx, tmp_path)
    for group in (2, 5, 12):
        p = tmp_path / f"g{group}.json"
        p.write_text(json.dumps({"format": "lqcd-tune", "version": 2, "device": tag, "entries": [
            _entry(prec=1, nr=12, nrhs=12, bucket=6, ntiles=768, form=2, group=group)]}))
        lqcd.tune_clear()
        lqcd.tune_load(p)
        got = run()
        assert all(np.array_equal(a, b) for a, b in zip(ref, got)), group
    lqcd.tune_clear()
    res = lqcd.autotune_dslash([g] * 12, "f32", 12)
    assert res["nrhs"] == 12 and (res["group"] == 0 or 2 <= res["group"] <= 12)
    assert res["form"] == 2 if res["group"] else res["form"] in (0, 3)
    got = run()
    assert all(np.array_equal(a, b) for a, b in zip(ref, got))
