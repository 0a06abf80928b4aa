"""The inverse z-pass for caller lists in stick order (FP32, |l| <= n3/4):
inputs addressed from each stick's run (the default), or staged by bulk
copies (VLOC_Z_BULK).

Each stick of a z-pass tile is one contiguous run of the band's
coefficients; one lane stages it in shared memory by a 1-D bulk copy of its
16-byte-aligned interior plus plain loads of its unaligned ends, completing
on an mbarrier with a bounded wait.  The first stage then reads the same
values the direct form loads one by one, so the two forms agree bit for bit
(the direct form is the same plan without the flag), and both match the
FP64 oracle.
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
    q = vloc.VlocPlan(n, g, torch.complex64, z_bulk=True, **kw)
    ref = vloc.VlocPlan(n, g, torch.complex64, **kw)
    assert q.info()["z_bulk"] and not ref.info()["z_bulk"]
    return q, ref


# n3 of two-stage schedules, quarter-band spheres; odd and even npw (the
# bands' runs start on and off the 16-byte grid)
CASES = [((20, 18, 24), 6.0), ((24, 30, 48), 12.0), ((36, 40, 64), 16.0), ((40, 36, 72), 18.0),
         ((48, 48, 96), 24.0), ((30, 36, 96), 13.0), ((40, 40, 120), 20.0), ((36, 36, 128), 32.0)]


@pytest.mark.parametrize("n,R", CASES)
def test_bulk_staged_z_pass_bit_identical_and_matches_oracle(n, R):
    g, c, V = make_case(n, R, 5, seed=101, prec="f32")
    q, ref = _plans(n, g)
    ct, Vt = torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda()
    out, out_ref = q.apply(ct, Vt), ref.apply(ct, Vt)
    # a view one band in: every run moves by npw elements (a change of
    # 16-byte phase when npw is odd)
    out1 = q.apply(ct[1:], Vt)
    torch.cuda.synchronize()
    assert torch.equal(out, out_ref)
    assert torch.equal(out1, out[1:])
    assert rel_l2_per_band(out.cpu().numpy(), oracle_apply(n, g, c, V)).max() < TOL["f32"]
    assert q.device_status() == 0


def test_bulk_staged_z_pass_chunks_poison_h_alias():
    n = (96, 96, 96)
    g, c, V = make_case(n, 24.0, 7, seed=102, prec="f32")
    assert len(g) % 2 == 1
    q, ref = _plans(n, g, chunk=3, poison=True)
    h = np.linspace(0.5, 2.0, len(g)).astype(np.float32)
    ct, Vt, ht = torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(h).cuda()
    out, out_ref = q.apply_h(ct, Vt, ht), ref.apply_h(ct, Vt, ht)
    torch.cuda.synchronize()
    assert torch.equal(out, out_ref)
    want = oracle_apply(n, g, c, V) + h.astype(np.float64)[None, :] * c.astype(np.complex128)
    assert rel_l2_per_band(out.cpu().numpy(), want).max() < TOL["f32"]
    q.apply_h(ct, Vt, ht, out=ct)
    torch.cuda.synchronize()
    assert torch.equal(ct, out)
    assert q.device_status() == 0


@pytest.mark.parametrize("n,R", [((48, 48, 96), 24.0), ((36, 40, 64), 16.0), ((40, 40, 120), 20.0)])
def test_run_addressed_k1_matches_dense_table_bit_for_bit(n, R):
    # a caller list in stick order lets K1 address its inputs from each
    # stick's run; the same plane waves in a shuffled order go through the
    # dense z-band table.  Each element of the transform sees
    # the same values and the same arithmetic, so the results agree bit for
    # bit, for the action and for H = diag + V_loc written over its input.
    g, c, V = make_case(n, R, 5, seed=103, prec="f32")
    perm = np.random.default_rng(104).permutation(len(g))
    pt = torch.from_numpy(perm).cuda()
    p_run = vloc.VlocPlan(n, g, torch.complex64)
    p_tab = vloc.VlocPlan(n, np.ascontiguousarray(g[perm]), torch.complex64)
    Vt = torch.from_numpy(V).cuda()
    c_run, c_tab = torch.from_numpy(c).cuda(), torch.from_numpy(np.ascontiguousarray(c[:, perm])).cuda()
    out_run, out_tab = p_run.apply(c_run, Vt), p_tab.apply(c_tab, Vt)
    h = np.linspace(0.5, 2.0, len(g)).astype(np.float32)
    h_run, h_tab = torch.from_numpy(h).cuda(), torch.from_numpy(np.ascontiguousarray(h[perm])).cuda()
    p_run.apply_h(c_run, Vt, h_run, out=c_run)
    p_tab.apply_h(c_tab, Vt, h_tab, out=c_tab)
    torch.cuda.synchronize()
    assert torch.equal(out_tab, out_run[:, pt])
    assert torch.equal(c_tab, c_run[:, pt])
    assert rel_l2_per_band(out_run.cpu().numpy(), oracle_apply(n, g, c, V)).max() < TOL["f32"]
    want = oracle_apply(n, g, c, V) + h.astype(np.float64)[None, :] * c.astype(np.complex128)
    assert rel_l2_per_band(c_run.cpu().numpy(), want).max() < TOL["f32"]
