"""Host logic of bench.py (no GPU): the algorithmic byte and FLOP counts that
the roofline divides by, and the clock record.

The expected sizes are the hot-path scope table's, counted from the sphere
definition h^2 + k^2 + l^2 <= R^2 independently of this library; the plan's
stick and plane counts (host-only plans, no device memory) must reproduce
them exactly, and bench.path_counts must turn them into the stated per-band
bytes (B5: 2 npw + 4 cylinder + 4 slab complex values) and 5 n log2 n FLOPs.
"""
import importlib.util
import os

import numpy as np
import pytest

from paper_1601_07378_gb300 import synth, vloc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_07378_gb300.build import build
    build()
    return vloc.load()


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


# grid, R, npw, sticks, cylinder points, slab points, MFLOP per band (compact)
TABLE = [
    ((24, 24, 24), 6, 925, 113, 2712, 7488, 1.1),
    ((64, 64, 64), 16, 17077, 797, 51008, 135168, 27.4),
    ((96, 96, 120), 24, 57777, 1793, 215160, 564480, 127.1),
    ((96, 96, 96), 24, 57777, 1793, 172128, 451584, 101.1),
]


@pytest.mark.parametrize("n,R,npw,S,cyl,slab,mflop", TABLE)
def test_plan_sizes_and_counts_match_the_scope_table(bench, n, R, npw, S, cyl, slab, mflop):
    torch = pytest.importorskip("torch")
    g = synth.sphere_glist(*n, R)
    assert len(g) == npw
    plan = vloc.VlocPlan(n, g, torch.complex64, host_only=True)
    info = plan.info()
    assert (info["npw"], info["nsticks"]) == (npw, S)
    assert info["nsticks"] * n[2] == cyl
    assert info["nplanes"] * n[1] * n[2] == slab
    per_band, flops, B5, B3 = bench.path_counts(info, n)
    assert round(flops / 1e6, 1) == mflop
    e = 8
    assert B5 == 2 * npw * e + 4 * cyl * e + 4 * slab * e
    assert B3 == 2 * npw * e + 4 * slab * e
    # the five kernels' bytes add up to B5
    assert sum(per_band.values()) == B5


def test_b5_and_b3_at_the_headline_and_config_2(bench):
    torch = pytest.importorskip("torch")
    out = {}
    for n in ((96, 96, 96), (96, 96, 120)):
        plan = vloc.VlocPlan(n, synth.sphere_glist(*n, 24), torch.complex64, host_only=True)
        _, _, B5, B3 = bench.path_counts(plan.info(), n)
        out[n] = (round(B5 / 1e6, 2), round(B3 / 1e6, 2))
    assert out[(96, 96, 96)] == (20.88, 15.38)
    assert out[(96, 96, 120)] == (25.87, 18.99)
    plan64 = vloc.VlocPlan((96, 96, 96), synth.sphere_glist(96, 96, 96, 24), torch.complex128, host_only=True)
    assert round(bench.path_counts(plan64.info(), (96, 96, 96))[2] / 1e6, 2) == 41.77


def test_flops_count_by_hand_on_a_small_grid(bench):
    # 5 n log2 n per line over the pruned line sets, both directions, plus
    # 2N for the product with V, written out for a 4 x 8 x 16 grid
    info = {"nsticks": 3, "nplanes": 2, "npw": 10, "precision": 1}
    _, flops, _, _ = bench.path_counts(info, (4, 8, 16))
    f = lambda m: 5 * m * np.log2(m)
    by_hand = 2 * (3 * f(16) + 2 * 16 * f(8) + 8 * 16 * f(4)) + 2 * 4 * 8 * 16
    assert flops == pytest.approx(by_hand)


def test_clock_summary(bench):
    def line(sm, smax, hw="Not Active", therm="Not Active", swth="Not Active", cap="Not Active"):
        return f"0, {sm}, {smax}, 900.00, 0x0, {hw}, {therm}, {swth}, {cap}"
    got = bench.summarize_clocks([line(2070, 2070), line(1980, 2070, cap="Active"), line(2070, 2070),
                                  "garbage", "0, [N/A], 2070, 1, 0, a, b, c, d"])
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    got = bench.summarize_clocks([line(1500, 2070, therm="Active"), line(1400, 2070, hw="Active")])
    assert got["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and got["sm_mhz"] == 1500.0
    assert bench.summarize_clocks([])["samples"] == 0
