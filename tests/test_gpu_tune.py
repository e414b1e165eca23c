"""The autotuner on the GPU: a plan made with MW_FLAG_AUTOTUNE records its
choice in the cache named by MW_TUNE_CACHE, a second plan of the same key
takes the cached choice without a search, a plain plan given the same values
produces bitwise the same results, and the tuned plan is no slower than the
fixed defaults (chunk 512, two groups per pass, 256 columns per block) at
L = 512 and at the benchmark's L = 2048, B = 16."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1110_6298_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def mw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6298_gb300 import build
    build.build()
    from paper_1110_6298_gb300 import mw as m
    m.lib()
    return m


def round_trip_ms(plan, flm, maps, out, n=3):
    plan.inverse(flm, out=maps)
    plan.forward(maps, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(n):
        plan.inverse(flm, out=maps)
        plan.forward(maps, out=out)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n


@pytest.mark.parametrize("L,spins", [(512, [0] * 8 + [2] * 8), (2048, [0] * 8 + [2] * 8)])
def test_autotuned_plan(mw, tmp_path, monkeypatch, L, spins):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("MW_TUNE_CACHE", str(cache))
    g = wl.rng(600 + L)
    flm = torch.from_numpy(np.stack([wl.gaussian_flm(g, L, s, wl.cl_red) for s in spins])).cuda()
    tuned = mw.Plan(L, spins, precision="mixed", autotune=True)
    t = tuned.tuning
    assert t["ms"] > 0 and t["chunk"] in (128, 256, 512) and t["groups"] in (1, 2) and t["tn_threads"] in (128, 256)
    dev = torch.cuda.get_device_name()
    key = mw.tune_key([L] * len(spins), spins, mw.PRECISIONS["mixed"] | mw.FLAG_AUTOTUNE, dev)
    rec = mw.tune_cache_lookup(cache, key)
    assert rec is not None and {k: rec[k] for k in ("chunk", "groups", "tn_threads")} == \
        {k: t[k] for k in ("chunk", "groups", "tn_threads")}
    # a second plan of the same key reads the cache (no search: same ms, quick)
    again = mw.Plan(L, spins, precision="mixed", autotune=True)
    ta = again.tuning
    assert {k: ta[k] for k in ("chunk", "groups", "tn_threads")} == {k: t[k] for k in ("chunk", "groups", "tn_threads")}
    assert abs(ta["ms"] - t["ms"]) < 1e-5  # the recorded time, not a new search
    again.close()
    # the same values on a plain plan give bitwise the same results
    static = mw.Plan(L, spins, precision="mixed")
    static.set_tuning(t["chunk"], t["groups"], t["tn_threads"])
    m1, m2 = tuned.inverse(flm), static.inverse(flm)
    assert torch.equal(m1, m2)
    f1, f2 = tuned.forward(m1), static.forward(m1)
    assert torch.equal(f1, f2)
    assert float((f1 - flm).abs().max() / flm.abs().max()) < 1e-6
    # no slower than the fixed defaults (best of two measurements each, 10% noise margin)
    default = mw.Plan(L, spins, precision="mixed")
    maps, out = torch.empty_like(m1), torch.empty_like(flm)
    td = min(round_trip_ms(default, flm, maps, out) for _ in range(2))
    tt = min(round_trip_ms(tuned, flm, maps, out) for _ in range(2))
    assert tt <= 1.10 * td, (tt, td, t)
    for p in (tuned, static, default):
        p.close()
