"""The quarter-sphere x-pass (Sec. 4.3, Fig. 5: the cuboid of a sphere of
radius n1/4 occupies x = 0..n1/4 and n1 - n1/4 .. n1 - 1).

For that plane set the x-pass kernels take each row's plane at compile time,
skip the rows known to be zero in the first inverse stage and never form the
outputs of rows outside the cuboid in the last forward stage.  Skipping a
known zero changes no rounding (x + 0 = x).  The results must match the FP64
oracle within the usual gates, and the general x-pass (selected by creating
the plan with VLOC_NO_XQ set) within a few units of the last place.
"""
import numpy as np
import pytest

from helpers import TOL, make_case, oracle_apply, rel_l2_per_band
from oracle import oracle as O
from paper_1601_07378_gb300 import synth, vloc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# every compiled x length, with y/z lengths that hold the sphere of radius n1/4
CASES = [(24, 16), (32, 18), (48, 30), (60, 32), (64, 36), (72, 40), (80, 48), (96, 50), (100, 54),
         (120, 64), (128, 72), (144, 80)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1601_07378_gb300.build import build
    build()


def _plans(n, g, dtype, monkeypatch, **kw):
    q = vloc.VlocPlan(n, g, dtype, **kw)
    monkeypatch.setenv("VLOC_NO_XQ", "1")
    ref = vloc.VlocPlan(n, g, dtype, **kw)
    monkeypatch.delenv("VLOC_NO_XQ")
    assert q.info()["x_quarter"] and not ref.info()["x_quarter"]
    return q, ref


@pytest.mark.parametrize("n1,m", CASES)
def test_quarter_x_pass_fp32_bit_identical_and_matches_oracle(n1, m, monkeypatch):
    n = (n1, m, m)
    g, c, V = make_case(n, n1 / 4, 3, seed=81, order="shuffled", prec="f32")
    q, ref = _plans(n, g, torch.complex64, monkeypatch)
    ct = torch.from_numpy(c).cuda()
    Vt = torch.from_numpy(V).cuda()
    out = q.apply(ct, Vt)
    out_ref = ref.apply(ct, Vt)
    torch.cuda.synchronize()
    o, o_ref = out.cpu().numpy(), out_ref.cpu().numpy()
    assert rel_l2_per_band(o, oracle_apply(n, g, c, V)).max() < TOL["f32"]
    assert rel_l2_per_band(o, o_ref.astype(np.complex128)).max() < 3e-7


@pytest.mark.parametrize("double_float", [False, True])
@pytest.mark.parametrize("n1,m", [(24, 24), (48, 32), (96, 60), (144, 80)])
def test_quarter_x_pass_fp64_bit_identical_and_matches_oracle(n1, m, double_float, monkeypatch):
    n = (n1, m, m)
    g, c, V = make_case(n, n1 / 4, 2, seed=82, order="shuffled", prec="f64")
    q, ref = _plans(n, g, torch.complex128, monkeypatch, double_float=double_float)
    assert q.info()["double_float"] == double_float
    ct = torch.from_numpy(c).cuda()
    Vt = torch.from_numpy(V).cuda()
    out = q.apply(ct, Vt)
    out_ref = ref.apply(ct, Vt)
    torch.cuda.synchronize()
    assert rel_l2_per_band(out.cpu().numpy(), oracle_apply(n, g, c, V)).max() < TOL["f64"]
    assert rel_l2_per_band(out.cpu().numpy(), out_ref.cpu().numpy()).max() < 1e-14


def test_quarter_x_pass_backward_chunks_and_poison(monkeypatch):
    # the backward's dL/dc runs the same x-pass; poisoned workspace, chunks
    n = (64, 36, 36)
    g, c, V = make_case(n, 16, 7, seed=83, prec="f32")
    rng = np.random.default_rng(84)
    gout = (rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).astype(np.complex64)
    q, ref = _plans(n, g, torch.complex64, monkeypatch, chunk=3, poison=True)
    ct, Vt, gt = torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(gout).cuda()
    gc, gV = q.backward(ct, gt, Vt)
    gc0, gV0 = ref.backward(ct, gt, Vt)
    out = q.apply(ct, Vt)
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy().view(np.float32)).all()
    assert rel_l2_per_band(gc.cpu().numpy(), gc0.cpu().numpy().astype(np.complex128)).max() < 3e-7
    assert torch.equal(gV, gV0)   # dL/dV does not use the forward x-pass
    assert rel_l2_per_band(out.cpu().numpy(), oracle_apply(n, g, c, V)).max() < TOL["f32"]


@pytest.mark.parametrize("n1,m,nb", [(48, 30, 5), (96, 50, 3), (144, 80, 2)])
def test_quarter_density_matches_oracle(n1, m, nb, monkeypatch):
    # the density's x-pass reads only the cuboid's rows in its first stage
    n = (n1, m, m)
    g, c, _ = make_case(n, n1 / 4, nb, seed=85, order="shuffled", prec="f32")
    occ = np.linspace(2.0, 0.5, nb).astype(np.float32)
    q, ref = _plans(n, g, torch.complex64, monkeypatch, chunk=2)
    ct, ot = torch.from_numpy(c).cuda(), torch.from_numpy(occ).cuda()
    rho = q.density(ct, ot).cpu().numpy().astype(np.float64)
    rho0 = ref.density(ct, ot).cpu().numpy().astype(np.float64)
    want = O.density(n, g, c.astype(np.complex128), occ.astype(np.float64))
    assert np.linalg.norm(rho - want) / np.linalg.norm(want) < TOL["f32"]
    assert np.linalg.norm(rho - rho0) / np.linalg.norm(rho0) < 3e-7


@pytest.mark.parametrize("n3,m", CASES)
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_quarter_band_z_pass_matches_oracle(n3, m, prec, monkeypatch):
    # every |l| <= n3/4: K1 clears and reads only the band's rows, K4's last
    # forward stage forms only them (FP32 kernels; FP64 plans take the
    # general z-pass and are checked alongside)
    n = (m, m, n3)
    g, c, V = make_case(n, n3 / 4, 3, seed=86, order="shuffled", prec=prec)
    dt = torch.complex64 if prec == "f32" else torch.complex128
    q = vloc.VlocPlan(n, g, dt)
    monkeypatch.setenv("VLOC_NO_XQ", "1")
    ref = vloc.VlocPlan(n, g, dt)
    monkeypatch.delenv("VLOC_NO_XQ")
    assert q.info()["z_quarter"] and not ref.info()["z_quarter"]
    ct, Vt = torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda()
    out, out_ref = q.apply(ct, Vt), ref.apply(ct, Vt)
    h = torch.from_numpy(np.linspace(0.5, 2.0, len(g))).to("cuda", Vt.dtype)   # a diagonal added in the gather
    outh = q.apply_h(ct, Vt, h)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    want = oracle_apply(n, g, c, V)
    assert rel_l2_per_band(o, want).max() < TOL[prec]
    assert rel_l2_per_band(o, out_ref.cpu().numpy().astype(np.complex128)).max() < (3e-7 if prec == "f32" else 1e-14)
    want_h = want + np.asarray(h.cpu().numpy(), np.float64)[None, :] * c.astype(np.complex128)
    assert rel_l2_per_band(outh.cpu().numpy(), want_h).max() < TOL[prec]
