"""Correctness aids of the pruned passes, on the GPU.

* Poisoned workspace: with VLOC_POISON_WORKSPACE the cylinder and slab are
  filled with NaN before every chunk, so a pruned pass that reads a cell its
  chunk never wrote turns the result non-finite.  Every entry point that
  uses the workspace must still match the FP64 oracle.
* Allocation failures: VLOC_FAULT=alloc:K fails the K-th allocation of
  vloc_plan_create; the call must return VLOC_ERR_ALLOC and free what it had
  allocated.
* Bounded waits: VLOC_FAULT=tma_wait makes the first block of the TMA x-pass
  skip its first tile load; its bounded wait must run out, the kernel must
  return, and vloc_device_status must report VLOC_ERR_TIMEOUT once, with the
  context still usable.
* Arithmetic-rate probes: each kind runs and reports a plausible rate.
"""
import numpy as np
import pytest

from helpers import TOL, make_case, oracle_apply, rel_l2_per_band
from oracle import oracle as O
from paper_1601_07378_gb300 import synth, vloc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f32": (torch.complex64, torch.float32), "f64": (torch.complex128, torch.float64)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1601_07378_gb300.build import build
    build()


@pytest.mark.parametrize("prec,kind", [("f32", "ct"), ("f32", "generic"), ("f64", "ct"), ("f64", "generic"),
                                       ("f64", "double_float")])
@pytest.mark.parametrize("n,R,nb,chunk", [((24, 24, 24), 6, 3, 0), ((40, 36, 50), 8, 7, 3),
                                          ((48, 48, 25), 6, 5, 2), ((96, 96, 96), 24, 4, 3)])
def test_poisoned_workspace_apply_matches_oracle(prec, kind, n, R, nb, chunk):
    cd, rd = DT[prec]
    g, c, V = make_case(n, R, nb, seed=71, order="shuffled", prec=prec)
    plan = vloc.VlocPlan(n, g, cd, chunk=chunk, poison=True, generic=kind == "generic",
                         double_float=kind == "double_float")
    out = plan.apply(torch.from_numpy(c).to("cuda", cd), torch.from_numpy(V).to("cuda", rd))
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.isfinite(o.view(np.float64 if prec == "f64" else np.float32)).all()
    err = rel_l2_per_band(o, oracle_apply(n, g, c, V))
    assert err.max() < TOL[prec], err.max()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_poisoned_workspace_backward_halves_density_match_oracle(prec):
    cd, rd = DT[prec]
    n, R, nb = (32, 48, 30), 7, 5
    g, c, V = make_case(n, R, nb, seed=72, order="shuffled", prec=prec)
    rng = np.random.default_rng(73)
    gout = (rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).astype(c.dtype)
    plan = vloc.VlocPlan(n, g, cd, chunk=4, poison=True)
    ct = torch.from_numpy(c).to("cuda", cd)
    Vt = torch.from_numpy(V).to("cuda", rd)
    gc, gV = plan.backward(ct, torch.from_numpy(gout).to("cuda", cd), Vt)
    psi = plan.to_real(ct)
    back = plan.to_recip(psi)
    rho = plan.density(ct)
    torch.cuda.synchronize()
    dc_ref, dV_ref = O.grads(n, g, c.astype(np.complex128), V.astype(np.float64), gout.astype(np.complex128))
    assert rel_l2_per_band(gc.cpu().numpy(), dc_ref).max() < TOL[prec]
    dV = gV.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(dV - dV_ref) / np.linalg.norm(dV_ref) < TOL[prec]
    psi_ref = O.to_real(n, g, c.astype(np.complex128))
    assert rel_l2_per_band(psi.cpu().numpy().reshape(nb, -1), psi_ref.reshape(nb, -1)).max() < TOL[prec]
    back_ref = O.to_recip(n, g, psi_ref)
    assert rel_l2_per_band(back.cpu().numpy(), back_ref).max() < TOL[prec]
    rho_ref = O.density(n, g, c.astype(np.complex128))
    r = rho.cpu().numpy().astype(np.float64)
    assert np.isfinite(r).all()
    assert np.linalg.norm(r - rho_ref) / np.linalg.norm(rho_ref) < TOL[prec]


def test_allocation_failures_return_alloc_error_and_free_everything(monkeypatch):
    n = (48, 48, 48)
    g = synth.sphere_glist(*n, 12)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seen = 0
    for k in range(1, 30):
        monkeypatch.setenv("VLOC_FAULT", f"alloc:{k}")
        try:
            p = vloc.VlocPlan(n, g, torch.complex128, double_float=True, chunk=16)
        except vloc.VlocError as e:
            assert e.code == vloc.VLOC_ERR_ALLOC, (k, e.code)
            seen += 1
            continue
        p.close()      # k past the last allocation: the plan was made
        break
    monkeypatch.delenv("VLOC_FAULT")
    assert seen >= 8   # tables, 3 twiddles, error flag, 3 + 1 double-float, workspace, ...
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < (8 << 20), (free0, free1)
    # a plan made afterwards works
    gg, c, V = make_case(n, 12, 2, seed=74, prec="f64")
    plan = vloc.VlocPlan(n, gg, torch.complex128, double_float=True, chunk=16)
    out = plan.apply(torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda())
    assert rel_l2_per_band(out.cpu().numpy(), oracle_apply(n, gg, c, V)).max() < TOL["f64"]


def test_tma_wait_that_runs_out_reports_timeout(monkeypatch):
    n, R, nb = (64, 64, 64), 16, 6
    g, c, V = make_case(n, R, nb, seed=75, prec="f32")
    ct = torch.from_numpy(c).cuda()
    Vt = torch.from_numpy(V).cuda()
    monkeypatch.setenv("VLOC_FAULT", "tma_wait")
    plan = vloc.VlocPlan(n, g, torch.complex64, x_tma=True)
    monkeypatch.delenv("VLOC_FAULT")
    assert plan.info()["x_tma"]
    plan.apply(ct, Vt)
    assert plan.device_status() == vloc.VLOC_ERR_TIMEOUT
    assert plan.device_status() == vloc.VLOC_OK          # the flag was cleared
    # the context stays usable: a plan without the fault runs and is right
    good = vloc.VlocPlan(n, g, torch.complex64, x_tma=True)
    out = good.apply(ct, Vt)
    assert good.device_status() == vloc.VLOC_OK
    assert rel_l2_per_band(out.cpu().numpy(), oracle_apply(n, g, c, V)).max() < TOL["f32"]


@pytest.mark.parametrize("kind", sorted(vloc.PEAK_KINDS))
def test_alu_peak_probes_run(kind):
    r = vloc.alu_peak(kind, 2000)
    assert r["ms"] > 0 and r["flops"] > 0
    # far below any plausible ceiling and far above a broken launch
    assert 1.0 < r["gflops"] < 1e6, r
