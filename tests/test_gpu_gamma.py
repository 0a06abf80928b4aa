"""GPU parity of the Gamma-point real mode (Sec. 4.3, last paragraph) against
the FP64 oracle, through the C ABI.

The caller stores each real band on half of the sphere; the CUDA path packs
two bands into one complex transform and separates the results.  The oracle
completes each band with c(-G) = conj c(G), applies the plain definition and
reads the half back.  Same tolerances as the complex path (relative L2 per
band: 2e-6 FP32, 1e-12 FP64).
"""
import numpy as np
import pytest

from helpers import TOL, rel_l2_per_band
from oracle import oracle as O
from paper_1601_07378_gb300 import synth, vloc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f32": (torch.complex64, torch.float32), "f64": (torch.complex128, torch.float64)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1601_07378_gb300.build import build
    build()


def gamma_case(n, R, nb, seed, order="canonical", prec="f32"):
    g = synth.sphere_glist(*n, R, order=order, seed=seed)
    gh = synth.half_sphere(g)
    c = synth.coefficients(gh, nb, seed=seed)
    V, _ = synth.potential(*n, "smooth", seed=seed + 1000)
    if prec == "f32":
        c, V = c.astype(np.complex64), V.astype(np.float32)
    return gh, c, V


def oracle_gamma(n, gh, c, V, bands=None):
    cc = np.asarray(c, dtype=np.complex128)
    if bands is not None:
        cc = cc[bands]
    return O.gamma_apply(n, gh, cc, np.asarray(V, dtype=np.float64))


def run(n, gh, c, V, prec, **kw):
    cd, rd = DT[prec]
    plan = vloc.VlocPlan(n, gh, cd, gamma=True, **kw)
    ct = torch.from_numpy(np.ascontiguousarray(c)).to("cuda", cd)
    Vt = torch.from_numpy(np.ascontiguousarray(V)).to("cuda", rd)
    out = plan.apply(ct, Vt)
    torch.cuda.synchronize()
    return plan, ct, Vt, out


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,R,nb,order", [
    ((24, 24, 24), 6, 1, "canonical"),       # one band: its pair partner is zero
    ((24, 24, 24), 6, 5, "shuffled"),        # odd band count
    ((4, 6, 5), 2.2, 3, "shuffled"),
    ((8, 8, 8), 2.5, 4, "canonical"),
    ((40, 36, 50), 8, 3, "canonical"),
    ((30, 45, 27), 7, 6, "shuffled"),
    ((64, 64, 64), 16, 4, "canonical"),
])
def test_gamma_matches_oracle(prec, n, R, nb, order):
    gh, c, V = gamma_case(n, R, nb, seed=21, order=order, prec=prec)
    plan, _, _, out = run(n, gh, c, V, prec)
    inf = plan.info()
    assert inf["gamma"] and inf["npw"] == len(gh)
    err = rel_l2_per_band(out.cpu().numpy(), oracle_gamma(n, gh, c, V))
    assert err.max() < TOL[prec], err.max()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_gamma_full_size_sampled(prec):
    # 96^3, R = 24: 28 889 half-sphere plane waves, 1024 real bands (bench size)
    n, nb = (96, 96, 96), 1024
    gh, c, V = gamma_case(n, 24, nb, seed=2, prec=prec)
    plan, _, _, out = run(n, gh, c, V, prec)
    pairs = plan.info()["chunk_bands"]
    bands = sorted({b for b in (0, 1, 2 * pairs - 1, 2 * pairs, nb // 2 + 1, nb - 1) if b < nb})
    err = rel_l2_per_band(out.cpu().numpy()[bands], oracle_gamma(n, gh, c, V, bands))
    assert err.max() < TOL[prec], err.max()


def test_gamma_chunks_and_alias():
    n, nb = (24, 20, 30), 7
    gh, c, V = gamma_case(n, 5, nb, seed=3, order="shuffled", prec="f64")
    ref = oracle_gamma(n, gh, c, V)
    for chunk in (1, 2, 3, 100):
        plan, ct, Vt, out = run(n, gh, c, V, "f64", chunk=chunk)
        assert rel_l2_per_band(out.cpu().numpy(), ref).max() < TOL["f64"]
        plan.apply(ct, Vt, out=ct)
        torch.cuda.synchronize()
        assert torch.equal(ct, out)


def test_gamma_results_are_real_bands():
    # completing the result with conj at -G gives a real function: its G = 0
    # entry is real and the complex path on the completed list agrees
    n = (20, 18, 25)
    gh, c, V = gamma_case(n, 4, 4, seed=8, prec="f64")
    _, _, _, out = run(n, gh, c, V, "f64")
    z = int(np.flatnonzero(~np.any(gh != 0, axis=1))[0])
    assert torch.all(out[:, z].imag == 0)
    gf, cf = O.gamma_complete(gh, c)
    full = vloc.VlocPlan(n, gf, torch.complex128)
    of = full.apply(torch.from_numpy(cf).cuda(), torch.from_numpy(V).cuda())
    torch.cuda.synchronize()
    assert rel_l2_per_band(out.cpu().numpy(), of[:, :len(gh)].cpu().numpy()).max() < 1e-12


def test_gamma_graph_and_batched():
    n = (24, 24, 24)
    gh, c, V = gamma_case(n, 6, 9, seed=4, prec="f32")
    ref = oracle_gamma(n, gh, c, V)
    plan, ct, Vt, _ = run(n, gh, c, V, "f32", graph=True, chunk=2)
    for _ in range(2):
        out = plan.apply(ct, Vt)
        torch.cuda.synchronize()
        assert rel_l2_per_band(out.cpu().numpy(), ref).max() < TOL["f32"]
    g2 = synth.sphere_glist(*n, 5)
    c2 = synth.coefficients(g2, 3, seed=6).astype(np.complex64)
    p2 = vloc.VlocPlan(n, g2, torch.complex64)
    c2t = torch.from_numpy(c2).cuda()
    outs = vloc.apply_batched([plan, p2], [ct, c2t], [Vt, Vt])
    torch.cuda.synchronize()
    assert rel_l2_per_band(outs[0].cpu().numpy(), ref).max() < TOL["f32"]
    ref2 = O.apply(n, g2, c2.astype(np.complex128), V.astype(np.float64))
    assert rel_l2_per_band(outs[1].cpu().numpy(), ref2).max() < TOL["f32"]


def test_gamma_rejects():
    n = (16, 16, 16)
    g = synth.sphere_glist(*n, 4)
    gh = synth.half_sphere(g)
    # both G and -G present
    with pytest.raises(vloc.VlocError) as e:
        vloc.VlocPlan(n, np.concatenate([gh, -gh[1:2]]), torch.complex64, gamma=True)
    assert e.value.code == -3
    # -G outside the grid's index range (h = -n1/2 has no +n1/2)
    with pytest.raises(vloc.VlocError) as e:
        vloc.VlocPlan(n, np.array([[0, 0, 0], [-8, 0, 0]], dtype=np.int32), torch.complex64, gamma=True)
    assert e.value.code == -3
    plan = vloc.VlocPlan(n, gh, torch.complex64, gamma=True)
    c = torch.from_numpy(synth.coefficients(gh, 2, seed=1).astype(np.complex64)).cuda()
    V = torch.ones(n, dtype=torch.float32, device="cuda")
    with pytest.raises(vloc.VlocError) as e:
        plan.backward(c, c, V)
    assert e.value.code == -7
    assert np.array_equal(plan.index_map(), O.index_map(n, gh))


@pytest.mark.parametrize("n,R,nb,chunk", [((24, 24, 24), 6, 1, 0), ((24, 24, 24), 6, 7, 2), ((40, 36, 50), 8, 5, 0),
                                          ((30, 45, 27), 7, 6, 0), ((96, 96, 96), 24, 9, 4),
                                          ((48, 48, 60), 11, 4, 1)])
def test_gamma_pairs_formed_in_the_z_passes(n, R, nb, chunk, monkeypatch):
    # FP32 compile-time plans form each pair a + i b as K1 reads the half
    # list and separate the results as K4 writes them (no pack or unpack
    # pass); against the oracle and against the plan with the separate passes
    gh, c, V = gamma_case(n, R, nb, seed=23, order="shuffled", prec="f32")
    plan = vloc.VlocPlan(n, gh, torch.complex64, gamma=True, chunk=chunk, poison=True)
    monkeypatch.setenv("VLOC_GAMMA_PACK", "1")
    ref_plan = vloc.VlocPlan(n, gh, torch.complex64, gamma=True, chunk=chunk)
    monkeypatch.delenv("VLOC_GAMMA_PACK")
    fused = all(x in (24, 32, 48, 60, 64, 72, 80, 96, 100, 120, 128, 144) for x in n[2:])
    assert plan.info()["gamma_fused"] == fused and not ref_plan.info()["gamma_fused"]
    ct = torch.from_numpy(c).cuda()
    Vt = torch.from_numpy(V).cuda()
    out = plan.apply(ct, Vt)
    out_ref = ref_plan.apply(ct, Vt)
    d = torch.from_numpy(np.linspace(0.25, 3.0, len(gh)).astype(np.float32)).cuda()
    outh = plan.apply_h(ct, Vt, d)
    torch.cuda.synchronize()
    want = oracle_gamma(n, gh, c, V)
    assert rel_l2_per_band(out.cpu().numpy(), want).max() < TOL["f32"]
    assert rel_l2_per_band(out.cpu().numpy(), out_ref.cpu().numpy().astype(np.complex128)).max() < 3e-7
    want_h = want + d.cpu().numpy().astype(np.float64)[None, :] * c.astype(np.complex128)
    assert rel_l2_per_band(outh.cpu().numpy(), want_h).max() < TOL["f32"]
    # out == coeffs
    ca = ct.clone()
    plan.apply(ca, Vt, out=ca)
    torch.cuda.synchronize()
    assert torch.equal(ca, out)


def test_gamma_pair_forming_needs_mirrors_in_one_tile():
    # the row/column partitions of Sec. 4.1 / 4.2 do not keep a stick and its
    # mirror together, so their Gamma plans keep the separate passes
    n = (32, 32, 32)
    gh = synth.half_sphere(synth.sphere_glist(*n, 8))
    assert vloc.VlocPlan(n, gh, torch.complex64, gamma=True).info()["gamma_fused"]
    assert not vloc.VlocPlan(n, gh, torch.complex64, gamma=True, partition="basic").info()["gamma_fused"]
    assert not vloc.VlocPlan(n, gh, torch.complex128, gamma=True).info()["gamma_fused"]
    assert not vloc.VlocPlan(n, gh, torch.complex64, gamma=True, generic=True).info()["gamma_fused"]
