"""The warp-register z-passes (VLOC_Z_WARP; n3 = 32 C, C = 1..4; plain FP32
plans).

K1 and K4 split each length-n3 stick into C residue classes of 32 elements
and run the 32-point DFTs across a warp's lanes (Sec. 2's 1-D FFT sets along
z, Cooley-Tukey over the classes).  The results must match the FP64 oracle
within the FP32 gate, and the tile z-passes (the same plan without the flag)
within FP32 rounding: a different summation order, so closeness, not bit
identity.
"""
import numpy as np
import pytest

from helpers import TOL, make_case, oracle_apply, rel_l2_per_band
from paper_1601_07378_gb300 import vloc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1601_07378_gb300.build import build
    build()


def _plans(n, g, **kw):
    w = vloc.VlocPlan(n, g, torch.complex64, z_warp=True, **kw)
    ref = vloc.VlocPlan(n, g, torch.complex64, **kw)
    assert w.info()["z_warp"] and not ref.info()["z_warp"]
    return w, ref


# n3 of every class count; radii inside the quarter band (|l| <= n3/4) and
# beyond it (all three classes' rows occupied), odd and even stick counts
CASES = [((20, 18, 32), 8.0), ((20, 18, 32), 9.5), ((24, 30, 64), 16.0), ((30, 24, 64), 11.0),
         ((36, 40, 96), 24.0), ((40, 36, 96), 17.5), ((36, 36, 128), 32.0), ((24, 20, 128), 9.0)]


@pytest.mark.parametrize("n,R", CASES)
@pytest.mark.parametrize("order", ["canonical", "shuffled"])
def test_warp_z_pass_matches_oracle_and_tile_form(n, R, order):
    g, c, V = make_case(n, R, 5, seed=91, order=order, prec="f32")
    w, ref = _plans(n, g)
    ct, Vt = torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda()
    out, out_ref = w.apply(ct, Vt), ref.apply(ct, Vt)
    adj = w.apply(ct, Vt, adjoint=True)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    want = oracle_apply(n, g, c, V)
    assert rel_l2_per_band(o, want).max() < TOL["f32"]
    assert rel_l2_per_band(adj.cpu().numpy(), want).max() < TOL["f32"]   # V real: the adjoint is the same map
    assert rel_l2_per_band(o, out_ref.cpu().numpy().astype(np.complex128)).max() < 1e-6


def test_warp_z_pass_h_apply_in_place_and_chunks():
    # H = diag + V_loc with the result written over the input (each lane
    # reads its input coefficient before it writes the result there), over
    # several workspace chunks with a ragged last one
    n = (36, 40, 96)
    g, c, V = make_case(n, 24.0, 7, seed=92, order="shuffled", prec="f32")
    w, _ = _plans(n, g, chunk=3)
    h = np.linspace(0.5, 2.0, len(g)).astype(np.float32)
    want = oracle_apply(n, g, c, V) + h.astype(np.float64)[None, :] * c.astype(np.complex128)
    ct, Vt, ht = torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(h).cuda()
    out = w.apply_h(ct, Vt, ht)
    torch.cuda.synchronize()
    assert rel_l2_per_band(out.cpu().numpy(), want).max() < TOL["f32"]
    w.apply_h(ct, Vt, ht, out=ct)
    torch.cuda.synchronize()
    assert rel_l2_per_band(ct.cpu().numpy(), want).max() < TOL["f32"]


def test_warp_z_pass_full_size_sampled():
    # the full-size workload (96^3, R = 24, 1024 bands) in one workspace
    # chunk, 8 sampled bands against the oracle
    n = (96, 96, 96)
    g, c, V = make_case(n, 24.0, 1024, seed=93, order="canonical", prec="f32")
    plan = vloc.VlocPlan(n, g, torch.complex64, z_warp=True)
    assert plan.info()["z_warp"] and plan.info()["chunk_bands"] >= 1024
    out = plan.apply(torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda())
    torch.cuda.synchronize()
    pick = np.array([0, 1, 255, 511, 512, 777, 1022, 1023])
    o = out.cpu().numpy()[pick]
    assert rel_l2_per_band(o, oracle_apply(n, g, c[pick], V)).max() < TOL["f32"]
