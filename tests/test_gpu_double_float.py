"""GPU parity of the double-float FP64 apply (VLOC_DOUBLE_FLOAT): FP64 data
in and out, transforms in hi + lo FP32 pairs on the FP32 pipes.  The gate is
the FP64 one, 1e-12 relative L2 per band against the FP64 oracle."""
import numpy as np
import pytest

from helpers import TOL, make_case, oracle_apply, rel_l2_per_band
from oracle import oracle as O
from paper_1601_07378_gb300 import synth, vloc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1601_07378_gb300.build import build
    build()


def run(n, g, c, V, **kw):
    plan = vloc.VlocPlan(n, g, torch.complex128, double_float=True, **kw)
    ct = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    Vt = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    out = plan.apply(ct, Vt)
    torch.cuda.synchronize()
    return plan, ct, Vt, out


@pytest.mark.parametrize("n,R,nb,order", [
    ((24, 24, 24), 6, 1, "canonical"),
    ((24, 24, 24), 6, 5, "shuffled"),
    ((48, 60, 72), 11, 3, "shuffled"),      # three different lengths
    ((64, 64, 64), 16, 4, "canonical"),
    ((80, 32, 100), 8, 2, "shuffled"),
    ((96, 96, 25), 6, 2, "canonical"),      # odd z length: native FP64 fallback
])
def test_double_float_matches_oracle(n, R, nb, order):
    g, c, V = make_case(n, R, nb, seed=12, order=order, prec="f64")
    plan, _, _, out = run(n, g, c, V)
    inf = plan.info()
    assert inf["double_float"] == (n[2] != 25)
    err = rel_l2_per_band(out.cpu().numpy(), oracle_apply(n, g, c, V))
    assert err.max() < TOL["f64"], err.max()


@pytest.mark.parametrize("n", [(96, 96, 96), (96, 96, 120), (128, 128, 128), (144, 144, 144)])
def test_double_float_full_size_sampled(n):
    R, nb = n[0] // 4, (1024 if n == (96, 96, 96) else 64)
    g, c, V = make_case(n, R, nb, seed=2, prec="f64")
    plan, _, _, out = run(n, g, c, V)
    assert plan.info()["double_float"]
    chunk = plan.info()["chunk_bands"]
    bands = sorted({b for b in (0, chunk - 1, chunk, nb // 2, nb - 1) if b < nb})
    err = rel_l2_per_band(out.cpu().numpy()[bands], oracle_apply(n, g, c, V, bands))
    assert err.max() < TOL["f64"], err.max()


def test_double_float_chunks_alias_adjoint_h_graph():
    n, R, nb = (24, 32, 48), 6, 7
    g, c, V = make_case(n, R, nb, seed=3, order="shuffled", prec="f64")
    ref = oracle_apply(n, g, c, V)
    for chunk in (1, 3, 100):
        plan, ct, Vt, out = run(n, g, c, V, chunk=chunk)
        assert rel_l2_per_band(out.cpu().numpy(), ref).max() < TOL["f64"]
        adj = plan.apply(ct, Vt, adjoint=True)
        torch.cuda.synchronize()
        assert torch.equal(adj, out)
        plan.apply(ct, Vt, out=ct)
        torch.cuda.synchronize()
        assert torch.equal(ct, out)
    T = O.kinetic(g, (9.0, 9.5, 10.0))
    plan, ct, Vt, _ = run(n, g, c, V, graph=True)
    for _ in range(2):
        h = plan.apply_h(ct, Vt, torch.from_numpy(T).cuda())
        torch.cuda.synchronize()
        assert rel_l2_per_band(h.cpu().numpy(), T[None, :] * c + ref).max() < TOL["f64"]


def test_double_float_gamma():
    n = (48, 48, 48)
    gh = synth.half_sphere(synth.sphere_glist(*n, 12))
    c = synth.coefficients(gh, 5, seed=4)
    V, _ = synth.potential(*n, "smooth", seed=5)
    plan = vloc.VlocPlan(n, gh, torch.complex128, gamma=True, double_float=True)
    out = plan.apply(torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda())
    torch.cuda.synchronize()
    ref = O.gamma_apply(n, gh, c, V)
    assert rel_l2_per_band(out.cpu().numpy(), ref).max() < TOL["f64"]


def test_double_float_flag_needs_fp64():
    g = synth.sphere_glist(24, 24, 24, 6)
    with pytest.raises(vloc.VlocError):
        vloc.VlocPlan((24, 24, 24), g, torch.complex64, double_float=True)


def test_double_float_batched_graph():
    # two double-float plans of different grids in one graph-captured batch
    n1, n2 = (24, 24, 24), (48, 60, 72)
    g1, c1, V1 = make_case(n1, 6, 3, seed=7, prec="f64")
    g2, c2, V2 = make_case(n2, 11, 2, seed=8, prec="f64")
    p1 = vloc.VlocPlan(n1, g1, torch.complex128, double_float=True, graph=True)
    p2 = vloc.VlocPlan(n2, g2, torch.complex128, double_float=True, graph=True)
    cs = [torch.from_numpy(c1).cuda(), torch.from_numpy(c2).cuda()]
    Vs = [torch.from_numpy(V1).cuda(), torch.from_numpy(V2).cuda()]
    for _ in range(2):
        outs = vloc.apply_batched([p1, p2], cs, Vs)
        torch.cuda.synchronize()
        assert rel_l2_per_band(outs[0].cpu().numpy(), oracle_apply(n1, g1, c1, V1)).max() < TOL["f64"]
        assert rel_l2_per_band(outs[1].cpu().numpy(), oracle_apply(n2, g2, c2, V2)).max() < TOL["f64"]


@pytest.mark.parametrize("df", [True, False])
@pytest.mark.parametrize("n,R", [((36, 40, 48), 12.0), ((36, 40, 48), 14.0), ((30, 24, 72), 18.0), ((40, 36, 96), 24.0)])
def test_fp64_direct_z_pass_h_in_place(df, n, R):
    # |l| <= n3/4 for every plane wave (R <= n3/4): the inverse z-pass loads
    # the caller's band through the dense z-band table; R = 14 at n3 = 48
    # leaves the band and takes the tile z-pass.  Both FP64 forms, H = diag +
    # V_loc written over its input, chunks of 3 bands.
    g, c, V = make_case(n, R, 7, seed=31, order="shuffled", prec="f64")
    plan = vloc.VlocPlan(n, g, torch.complex128, double_float=df, chunk=3)
    h = np.linspace(0.5, 2.0, len(g))
    want = oracle_apply(n, g, c, V) + h[None, :] * c
    ct = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    Vt, ht = torch.from_numpy(V).cuda(), torch.from_numpy(h).cuda()
    out = plan.apply_h(ct, Vt, ht)
    plan.apply_h(ct, Vt, ht, out=ct)
    torch.cuda.synchronize()
    assert rel_l2_per_band(out.cpu().numpy(), want).max() < TOL["f64"]
    assert torch.equal(ct, out)
