"""Host-side logic of bench.py without a GPU: clock-record parsing, peaks, the source digest that
invalidates stale ncu traffic records, the forms table, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import bench
import paper_2103_00571_gb300 as su3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_clock_summary_parses_nvidia_smi_rows():
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 812.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "0, 1965, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = []
    assert c.summary()["samples"] == 0


def test_peaks_and_digest():
    hbm, smax, src = bench.peaks()
    assert hbm > 1000 and smax > 1000 and src in ("measured", "fallback")
    d1 = bench.source_digest()
    assert len(d1) == 16 and d1 == bench.source_digest()


def test_forms_table_is_valid():
    names = set()
    for name, dt, ri, ro, lay, *ar in bench.FORMS:
        assert name not in names
        names.add(name)
        arith = ar[0] if ar else su3.NATIVE
        assert su3.check_desc(su3.Desc(dt, ri, lay, 10, 0, arith)) == 0
        assert su3.check_desc(su3.Desc(dt, ro, lay, 10, 0, arith)) == 0


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--L", "8",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, check=True, cwd=ROOT)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["metric"] == bench.METRIC and line["steps"] == 2 and line["higher_is_better"] is True


def test_best_layout_from_tuning_cache():
    """The tuner's layout pick reads the committed cache: for each tuned (dtype, repr, arith) the
    layout with the highest GB/s, None where nothing was tuned."""
    from paper_2103_00571_gb300 import tune
    key = "NVIDIA GB300/152"
    forms = tune.load_cache()[key]["forms"]
    for dt in (su3.F64, su3.F32, su3.F16):
        got = tune.best_layout(dt, su3.FULL18, su3.NATIVE, key=key)
        rates = {tune.parse_form(n).layout: r["GBps"] for n, r in forms.items()
                 if (tune.parse_form(n).dtype, tune.parse_form(n).repr, tune.parse_form(n).arith,
                     tune.parse_form(n).site_stride_bytes) == (dt, su3.FULL18, su3.NATIVE, 0)}
        assert got == max(rates, key=rates.get)
    assert tune.best_layout(su3.F32, su3.TWOROW12, su3.F32PAIR, key=key) is None
    assert tune.best_layout(su3.F64, key="no such GPU") is None


def test_parse_launch():
    assert bench.parse_launch("block=256, tile_sites=64,threads_per_link=3") == {
        "block": 256, "tile_sites": 64, "threads_per_link": 3}
    assert bench.parse_launch("") == {}
    import pytest
    with pytest.raises(SystemExit):
        bench.parse_launch("warps=8")


def test_form_names_round_trip():
    from paper_2103_00571_gb300 import tune
    for name in tune.ALL_FORMS:
        d = tune.parse_form(name)
        assert tune.parse_form(tune.form_name(d)).key() == d.key()
        a, c = tune.parse_pair(name)
        assert a.key() == d.key()
        assert (c.repr != a.repr) == tune.is_pair_name(name)
    a, c = tune.parse_pair("f64-2to18-aos-f32pair")
    assert (a.repr, c.repr, a.arith) == (su3.TWOROW12, su3.FULL18, su3.F32PAIR)
    assert any(tune.is_pair_name(n) for n in tune.ALL_FORMS)
    d = tune.parse_form("f64-full-aos-f32pair-p640")
    assert (d.site_stride_bytes, d.arith) == (640, su3.F32PAIR) and tune.form_name(d) == "f64-full-aos-f32pair-p640"


def test_summary_ends_the_line_and_stays_short():
    """The compact digest holds the headline, the FP64-accurate form, every form, the batch and the
    end-to-end figure, and fits in the last kilobyte and a half of the printed line."""
    form = {"GBps": 5963.1, "site_updates_per_s": 5.18e9, "max_err": 3.3e-14, "ok": True}
    line = {"value": 1589.2, "site_updates_per_s": 1.38e9, "config": {"form": "f64-full18-aos-native"},
            "roofline": {"bound": "alu", "frac": 0.947, "hbm": {"frac": 0.239}},
            "fp64_accurate": {"form": "f64-f32pair-aos", "GBps": 5963.1, "max_err": 3.3e-14, "tol": 1e-13,
                              "ok": True, "roofline": {"frac": 0.8956}},
            "forms": {name: dict(form) for name, *_ in bench.FORMS},
            "batched": {k: {"ms": 1.27, "site_updates_per_s": 2.34e9, "ok": True}
                        for k in ("graph_persistent", "graph_persistent_f64_as_f32pair", "per_lattice_loop")},
            "e2e": {"value": 333.1, "path": "direct", "vs_copies_only": 1.9}, "cpu_baseline": {"value": 31.1},
            "paper_site640": {"native": {"site_updates_per_s": 1.38e9}, "f32pair": {"site_updates_per_s": 5.09e9}}}
    s = bench.summary(line)
    assert s["headline"]["hbm_frac"] == 0.239 and s["fp64_accurate"]["hbm_frac"] == 0.8956
    assert set(s["forms"]) == {name for name, *_ in bench.FORMS}
    assert s["forms"]["f64-f32pair-aos"] == [5963, 5.18, 3.3e-14] and s["forms_within_tol"] is True
    assert s["site640_Gsite_per_s"] == {"native": 1.38, "f32pair": 5.09}
    assert s["e2e"]["GBps"] == 333.1 and s["batched"]["graph_persistent"][2] is True
    assert len(json.dumps({"summary": s})) < 1400


def test_digest_ignores_comments_only():
    """The traffic records' digest follows the code: comments and layout do not change it, while a
    change in code, string literals included, does."""
    base = 'int a = 1; // x\n/* y */ const char* s = "// kept"; char q = \'"\';\n'
    assert bench.code_only(base) == bench.code_only(base.replace("// x", "// other words").replace("/* y */", "\n\n"))
    assert bench.code_only(base) != bench.code_only(base.replace("a = 1", "a = 2"))
    assert bench.code_only(base) != bench.code_only(base.replace("// kept", "// changed"))
    assert "// kept" in bench.code_only(base) and "x" not in bench.code_only(base).replace("// kept", "")
