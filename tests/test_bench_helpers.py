"""Host-side arithmetic of bench.py's roofline report (no GPU): unit counts
against their closed forms, the algorithmic bytes of the contractions against
a hand count, and the roofline entries' internal consistency for each
recursion the bench can report."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PK = {"hbm_gbs": 6794.8, "bf16_tflops": 1899.0, "fp64_tflops": 0.993, "src": "measured"}
ISSUE = 152 * 128 * 2070e6


@pytest.mark.parametrize("L", [1, 2, 7, 64, 2048])
def test_unit_counts(L):
    # sum_{l<L} (l+1)^2 = L (L+1) (2L+1) / 6
    assert bench.tn_units(L) == L * (L + 1) * (2 * L + 1) // 6
    # Risbo: half plane l(l+1)/2 plus integer plane (l+1)(l+2)/2 = (l+1)^2 per l >= 1
    assert bench.risbo_units(L) == bench.tn_units(L) - 1
    assert bench.risbo_ff_instructions(L) == sum(
        52 * (l * (l + 1) // 2) + 59 * ((l + 1) * (l + 2) // 2) for l in range(1, L))


def test_contraction_bytes_by_hand():
    L, B = 2048, 16
    M = 2 * L - 1
    planes = 4 * L * (L + 1) * (2 * L + 1) // 6
    want = 2 * planes + B * M * L * 8 + B * L * L * 16 + B * L * L * 8 + B * M * L * 16
    assert bench.contraction_bytes(L, B, "mixed") == want
    assert abs(want - 27.754e9) < 1e7
    # FP64: planes and operands twice as wide
    assert bench.contraction_bytes(L, B, "fp64") > want


@pytest.mark.parametrize("rec", ["tn", "risbo_ff", "risbo_f64"])
def test_delta_roofline_consistent(rec):
    L, sec = 2048, 0.0118
    d = bench.delta_roofline(rec, L, sec, PK, ISSUE, 152, 2070.0)
    assert d["bound"] in ("alu", "hbm")
    assert d["floor_ms"] > 0
    if rec == "tn":
        # the bound is the larger floor, and frac = floor / measured time
        fi = d["fp32_issue"]["frac"] * sec
        fb = d["hbm"]["frac"] * sec
        assert abs(1e3 * max(fi, fb) - d["floor_ms"]) < 1e-9
        assert abs(d["frac"] - d["floor_ms"] / 1e3 / sec) < 1e-12
        assert abs(fi - 25 * bench.tn_units(L) * 2 / ISSUE) < 1e-12  # 3 + 7 + 15 FP32 instructions per element
    else:
        assert abs(d["achieved"] - 2 * 7 * bench.risbo_units(L) / sec / 1e12) < 1e-9
        if rec == "risbo_ff":
            assert "fp32_issue" in d


def test_fp64_rate_formula_and_job_value():
    L = 2048
    tc = 2 * bench.contraction_units(L, [0] * 8 + [2] * 8) * 4
    cb = bench.contraction_bytes(L, 16, "mixed")
    r = bench.fp64_rate_delta_stage(L, 0.0564, PK["fp64_tflops"], tc, PK["bf16_tflops"], cb, PK["hbm_gbs"])
    rec_oct = 2 * 7 * bench.risbo_units(L) / (PK["fp64_tflops"] * 1e12)
    assert abs(r["roofline_ms"] - 1e3 * rec_oct) < 1e-9
    assert r["frac_quarter_plane_units"] > r["frac"]
    # whole-job transforms/s: 2 B transforms per rank and step
    assert bench.whole_job_value(2, 16, 10, 1.0) == 2 * 2 * 16 * 10


def test_error_report_on_host_tensors():
    torch = pytest.importorskip("torch")
    L = 16
    g = torch.Generator().manual_seed(0)
    ref = torch.randn(3, L * L, dtype=torch.complex128, generator=g)
    x = ref.clone()
    # perturb one coefficient in band l = 9 (index l*l + l + m)
    x[1, 9 * 9 + 9 + 2] += 1e-3
    rep = bench.error_report(x, ref, L, n_bands=4)
    assert abs(rep["rel_max"] - 1e-3 / float(ref.abs().max())) < 1e-12
    assert abs(rep["rel_rms"] - 1e-3 / float(ref.norm())) < 1e-12
    assert [b["l"] for b in rep["bands"]] == [[0, 4], [4, 8], [8, 12], [12, 16]]
    for b in rep["bands"]:
        if b["l"] == [8, 12]:
            sel = torch.tensor([8 <= int(i ** 0.5) < 12 for i in range(L * L)])
            assert abs(b["rel_max"] - 1e-3 / float(ref[:, sel].abs().max())) < 1e-12
        else:
            assert b["rel_max"] == 0.0
    # exact copies give zeros everywhere
    z = bench.error_report(ref, ref, L)
    assert z["rel_max"] == 0.0 and z["rel_rms"] == 0.0 and all(b["rel_max"] == 0.0 for b in z["bands"])
