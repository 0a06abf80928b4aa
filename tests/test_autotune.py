"""Autotuner: candidate schedules are valid factorisations (CPU), and every
schedule the tuner can pick computes the same action (GPU)."""
import numpy as np
import pytest

from paper_1601_07378_gb300 import autotune, synth, vloc
from paper_1601_07378_gb300.build import build
from helpers import TOL, make_case, oracle_apply, rel_l2_per_band

torch = pytest.importorskip("torch")


def test_factorizations_are_valid_and_complete():
    for n in (2, 24, 96, 120, 125, 144, 256):
        fs = autotune.factorizations(n)
        assert fs and all(int(np.prod(f)) == n and set(f) <= set(autotune.RADICES) and len(f) <= 3 for f in fs)
        assert len({tuple(f) for f in fs}) == len(fs)
    assert [12, 8] in autotune.factorizations(96) and [8, 12] in autotune.factorizations(96)


def test_set_schedule_validation_host_only():
    build()
    g = synth.sphere_glist(24, 24, 24, 6)
    plan = vloc.VlocPlan((24, 24, 24), g, host_only=True)
    plan.set_schedule(0, [4, 6])
    assert plan.info()["radix"][0] == [4, 6] and not plan.info()["compile_time_kernels"]
    for axis, rad in [(0, [5, 5]), (3, [24]), (1, [7, 2]), (2, [2, 2, 2, 3, 1])]:
        with pytest.raises(vloc.VlocError):
            plan.set_schedule(axis, rad)


@pytest.mark.gpu
def test_every_schedule_of_an_axis_matches_oracle():
    n, R = (24, 20, 30), 5
    g, c, V = make_case(n, R, 2, seed=70, order="shuffled", prec="f32")
    ref = oracle_apply(n, g, c, V)
    ct = torch.from_numpy(c).cuda()
    Vt = torch.from_numpy(V).cuda()
    for a in range(3):
        for rad in autotune.factorizations(n[a]):
            plan = vloc.VlocPlan(n, g, torch.complex64)
            plan.set_schedule(a, rad)
            out = plan.apply(ct, Vt)
            torch.cuda.synchronize()
            assert rel_l2_per_band(out.cpu().numpy(), ref).max() < TOL["f32"], (a, rad)


@pytest.mark.gpu
def test_tuner_returns_a_working_configuration(tmp_path, monkeypatch):
    monkeypatch.setenv("VLOC_TUNE_CACHE", str(tmp_path / "tune.json"))
    n, R, nb = (32, 32, 32), 8, 16
    g, c, V = make_case(n, R, nb, seed=71, prec="f32")
    cfg = autotune.tune(n, g, torch.complex64, nb, reps=1, chunks=(8, 16))
    assert cfg["candidates"] > 4 and cfg["ms"] > 0
    assert autotune.tune(n, g, torch.complex64, nb) == cfg          # served from the cache
    plan, cfg2 = autotune.tuned_plan(n, g, torch.complex64, nb)
    out = plan.apply(torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda())
    torch.cuda.synchronize()
    assert rel_l2_per_band(out.cpu().numpy(), oracle_apply(n, g, c, V)).max() < TOL["f32"]
