"""vloc_apply_noalloc: the apply for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (another runtime owns the GPU's memory,
or the process must not allocate after start-up).  vloc_apply_noalloc uses a
fixed scratch array built into the library instead of the plan's workspace,
and accepts host-only plans, which make no CUDA call.  These tests call it
through the C ABI, twice in a row, and compare with vloc_apply within the
parity tolerances (2e-6 FP32, 1e-12 FP64, relative L2 per band).  This file
is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

from helpers import TOL, make_case, rel_l2_per_band
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


@pytest.mark.parametrize("prec,n,R,nb", [("f32", (96, 96, 96), 24, 20),    # several scratch chunks
                                         ("f64", (64, 64, 64), 16, 7),
                                         ("f32", (30, 45, 27), 7, 3),
                                         ("f64", (24, 24, 24), 6, 1)])
@pytest.mark.parametrize("host_only", [False, True])
def test_noalloc_matches_apply_two_calls(prec, n, R, nb, host_only):
    cd, rd = DT[prec]
    g, c, V = make_case(n, R, nb, seed=31, order="shuffled", prec=prec)
    ref_plan = vloc.VlocPlan(n, g, cd)
    plan = vloc.VlocPlan(n, g, cd, host_only=True) if host_only else ref_plan
    Vt = torch.from_numpy(V).to("cuda", rd)
    for call in range(2):
        ct = torch.from_numpy(c).to("cuda", cd) * (1.0 + call)
        want = ref_plan.apply(ct, Vt)
        got = torch.full_like(ct, float("nan"))
        assert _noalloc(plan, ct, Vt, got) == vloc.VLOC_OK
        torch.cuda.synchronize()
        err = rel_l2_per_band(got.cpu().numpy(), want.cpu().numpy().astype(np.complex128))
        assert err.max() < TOL[prec], (call, err.max())


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
