"""vloc_apply_noalloc: the apply for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: code that runs while another runtime
owns the GPU's memory (a framework that reserves it up front and forbids
outside allocations), or a process that must not allocate after start-up.
vloc_apply_noalloc uses a fixed scratch array built into the library instead
of the plan's workspace, and accepts host-only plans, which make no CUDA
call.  These tests call it through the C ABI, twice in a row, and compare it
with vloc_apply and with the FP64 oracle on sampled bands, within the parity
tolerances (2e-6 FP32, 1e-12 FP64, relative L2 per band).  The plan's own
kernel family is used: compile-time-length (default), runtime-radix
(generic) and double-float plans are each covered.  This file is collected
last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

from helpers import TOL, make_case, oracle_apply, rel_l2_per_band
from paper_1601_07378_gb300 import synth, vloc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f32": (torch.complex64, torch.float32), "f64": (torch.complex128, torch.float64)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1601_07378_gb300.build import build
    build()


def _noalloc(plan, c, V, out):
    lib = vloc.load()
    nb = c.numel() // plan.npw
    return lib.vloc_apply_noalloc(plan.handle, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(V.data_ptr()), nb,
                                  ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec,n,R,nb,kind", [("f32", (96, 96, 96), 24, 20, "ct"),    # several scratch chunks
                                              ("f64", (64, 64, 64), 16, 7, "ct"),
                                              ("f32", (30, 45, 27), 7, 3, "ct"),
                                              ("f64", (24, 24, 24), 6, 1, "ct"),
                                              ("f32", (48, 40, 36), 10, 5, "generic"),
                                              ("f64", (48, 40, 36), 10, 4, "generic"),
                                              ("f64", (64, 64, 64), 16, 6, "double_float"),
                                              ("f64", (96, 96, 96), 24, 3, "double_float")])
@pytest.mark.parametrize("host_only", [False, True])
def test_noalloc_matches_apply_and_oracle_two_calls(prec, n, R, nb, kind, host_only):
    cd, rd = DT[prec]
    g, c, V = make_case(n, R, nb, seed=31, order="shuffled", prec=prec)
    opts = {"generic": kind == "generic", "double_float": kind == "double_float"}
    ref_plan = vloc.VlocPlan(n, g, cd, **opts)
    plan = vloc.VlocPlan(n, g, cd, host_only=True, **opts) if host_only else ref_plan
    if kind == "double_float":
        assert plan.info()["double_float"]
    Vt = torch.from_numpy(V).to("cuda", rd)
    sample = sorted({0, nb - 1, nb // 2})
    want_oracle = oracle_apply(n, g, c, V, bands=sample)
    for call in range(2):
        scale = 1.0 + call
        ct = torch.from_numpy(c).to("cuda", cd) * scale
        want = ref_plan.apply(ct, Vt)
        got = torch.full_like(ct, float("nan"))
        assert _noalloc(plan, ct, Vt, got) == vloc.VLOC_OK
        torch.cuda.synchronize()
        g_np = got.cpu().numpy()
        err = rel_l2_per_band(g_np, want.cpu().numpy().astype(np.complex128))
        assert err.max() < TOL[prec], (call, err.max())
        err_o = rel_l2_per_band(g_np[sample] / scale, want_oracle)
        assert err_o.max() < TOL[prec], (call, err_o.max())


def test_noalloc_refuses_gamma_plans():
    n = (32, 32, 32)
    gh = synth.half_sphere(synth.sphere_glist(*n, 8))
    for host_only in (True, False):
        plan = vloc.VlocPlan(n, gh, torch.complex64, host_only=host_only, gamma=True)
        c = torch.zeros((2, len(gh)), dtype=torch.complex64, device="cuda")
        V = torch.zeros(n, dtype=torch.float32, device="cuda")
        out = torch.zeros_like(c)
        assert _noalloc(plan, c, V, out) == vloc.VLOC_ERR_STATE
    torch.cuda.synchronize()


def test_noalloc_rejects_problems_beyond_its_scratch():
    # 256^3 FP64 with R = 60: one band's workspace alone exceeds the 48 MiB.
    n = (256, 256, 256)
    g = synth.sphere_glist(*n, 60)
    plan = vloc.VlocPlan(n, g, torch.complex128, host_only=True)
    c = torch.zeros((1, len(g)), dtype=torch.complex128, device="cuda")
    V = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(c)
    assert _noalloc(plan, c, V, out) == vloc.VLOC_ERR_SIZE
    assert _noalloc(plan, c, V, out) == vloc.VLOC_ERR_SIZE
