"""GPU parity of the two halves of the chain on their own and of the charge
density (through the C ABI) against the FP64 oracle.

vloc_to_real: psi = F+ S c (Sec. 2, the G -> r FFT); vloc_to_recip: the
r -> G FFT with 1/N and the gather; vloc_density: rho(r) = sum_n f_n
|psi_n(r)|^2 (Sec. 3.1), also for Gamma-point plans.  Tolerances as the
apply tests: relative L2 2e-6 (FP32) and 1e-12 (FP64).
"""
import numpy as np
import pytest

from helpers import TOL, make_case, rel_l2_per_band
from oracle import oracle as O
from paper_1601_07378_gb300 import synth, vloc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f32": (torch.complex64, torch.float32), "f64": (torch.complex128, torch.float64)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1601_07378_gb300.build import build
    build()


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


CASES = [
    ((24, 24, 24), 6, 3, "canonical"),
    ((4, 6, 5), 2.2, 2, "shuffled"),
    ((40, 36, 50), 8, 3, "shuffled"),
    ((48, 48, 25), 6, 2, "shuffled"),     # compile-time x length, odd z length
    ((30, 45, 27), 7, 2, "canonical"),
    ((64, 64, 64), 16, 3, "canonical"),
]


@pytest.mark.parametrize("generic", [False, True])
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,R,nb,order", CASES)
def test_to_real_and_to_recip(prec, n, R, nb, order, generic):
    cd, rd = DT[prec]
    g, c, _ = make_case(n, R, nb, seed=31, order=order, prec=prec)
    plan = vloc.VlocPlan(n, g, cd, generic=generic)
    ct = torch.from_numpy(c).cuda()
    psi = plan.to_real(ct)
    torch.cuda.synchronize()
    ref = O.to_real(n, g, c.astype(np.complex128))
    assert rel_l2_per_band(psi.cpu().numpy(), ref).max() < TOL[prec]
    # r -> G of an arbitrary grid (not only of a band-limited one)
    rng = np.random.default_rng(5)
    u = (rng.standard_normal((nb, *n)) + 1j * rng.standard_normal((nb, *n))).astype(c.dtype)
    got = plan.to_recip(torch.from_numpy(u).cuda())
    torch.cuda.synchronize()
    assert rel_l2_per_band(got.cpu().numpy(), O.to_recip(n, g, u.astype(np.complex128))).max() < TOL[prec]
    # round trip on the device
    back = plan.to_recip(psi)
    torch.cuda.synchronize()
    assert rel_l2_per_band(back.cpu().numpy(), c.astype(np.complex128)).max() < TOL[prec]


@pytest.mark.parametrize("generic", [False, True])
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,R,nb,order", CASES + [((32, 32, 32), 8, 37, "canonical")])
def test_density(prec, n, R, nb, order, generic):
    cd, rd = DT[prec]
    g, c, _ = make_case(n, R, nb, seed=41, order=order, prec=prec)
    f = np.random.default_rng(2).uniform(0.0, 2.0, nb).astype(np.float32 if prec == "f32" else np.float64)
    plan = vloc.VlocPlan(n, g, cd, generic=generic)
    ct = torch.from_numpy(c).cuda()
    rho = plan.density(ct, torch.from_numpy(f).cuda())
    rho1 = plan.density(ct)
    torch.cuda.synchronize()
    assert _rel(rho.cpu().numpy(), O.density(n, g, c.astype(np.complex128), f.astype(np.float64))) < TOL[prec]
    assert _rel(rho1.cpu().numpy(), O.density(n, g, c.astype(np.complex128))) < TOL[prec]


@pytest.mark.parametrize("generic", [False, True])
def test_density_chunks_groups_and_determinism(generic):
    # chunks of 3 and 64 bands and one of all 70, several groups of 16 bands;
    # the compile-time FP32 kernels keep their group sums in FP32 (one x-pass
    # launch takes a whole chunk), the runtime-radix ones in FP64 (a chunk
    # of 64 or 70 bands takes two launches); bit-identical on repeat
    n, R, nb = (24, 20, 30), 5, 70
    g, c, _ = make_case(n, R, nb, seed=7, order="shuffled", prec="f32")
    ref = O.density(n, g, c.astype(np.complex128))
    for chunk in (3, 64, 0):
        plan = vloc.VlocPlan(n, g, torch.complex64, chunk=chunk, generic=generic)
        ct = torch.from_numpy(c).cuda()
        a = plan.density(ct)
        b = plan.density(ct)
        torch.cuda.synchronize()
        assert _rel(a.cpu().numpy(), ref) < TOL["f32"]
        assert torch.equal(a, b)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_gamma_density(prec):
    cd, rd = DT[prec]
    for n, R, nb in (((24, 24, 24), 6, 5), ((40, 36, 50), 8, 4), ((8, 8, 8), 2.5, 1)):
        gh = synth.half_sphere(synth.sphere_glist(*n, R, order="shuffled", seed=3))
        c = synth.coefficients(gh, nb, seed=9)
        f = np.linspace(0.5, 2.0, nb)
        if prec == "f32":
            c, f = c.astype(np.complex64), f.astype(np.float32)
        plan = vloc.VlocPlan(n, gh, cd, gamma=True, chunk=2)
        rho = plan.density(torch.from_numpy(c).cuda(), torch.from_numpy(f).cuda())
        torch.cuda.synchronize()
        want = O.gamma_density(n, gh, c.astype(np.complex128), f.astype(np.float64))
        assert _rel(rho.cpu().numpy(), want) < TOL[prec], n


def test_density_full_size_matches_sampled_oracle():
    # 96^3, R = 24, 256 bands (FP32, default chunk): the oracle's density on
    # a sample of 16 bands equals the device density of the same 16 bands,
    # and the 256-band density obeys Parseval
    n, R, nb = (96, 96, 96), 24, 256
    g, c, _ = make_case(n, R, nb, seed=2, prec="f32")
    plan = vloc.VlocPlan(n, g, torch.complex64)
    ct = torch.from_numpy(c).cuda()
    rho = plan.density(ct).double().cpu().numpy()
    N = np.prod(n)
    assert abs(rho.sum() - N * (np.abs(c.astype(np.complex128)) ** 2).sum()) < 1e-5 * rho.sum()
    s = [0, 100, 255] + list(range(1, 14))
    sub = plan.density(ct[s].contiguous())
    torch.cuda.synchronize()
    assert _rel(sub.cpu().numpy(), O.density(n, g, c[s].astype(np.complex128))) < TOL["f32"]


def test_half_errors():
    n = (16, 16, 16)
    g, c, _ = make_case(n, 4, 2, seed=1, prec="f32")
    plan = vloc.VlocPlan(n, g, torch.complex64)
    ct = torch.from_numpy(c).cuda()
    z = plan.density(ct[:0])
    torch.cuda.synchronize()
    assert torch.count_nonzero(z) == 0
    gp = vloc.VlocPlan(n, synth.half_sphere(synth.sphere_glist(*n, 4)), torch.complex64, gamma=True)
    cg = torch.zeros(2, gp.npw, dtype=torch.complex64, device="cuda")
    with pytest.raises(vloc.VlocError) as e:
        gp.to_real(cg)
    assert e.value.code == -7
    buf = torch.zeros(2 * int(np.prod(n)) + 2 * plan.npw, dtype=torch.complex64, device="cuda")
    with pytest.raises(vloc.VlocError) as e:  # psi overlapping the coefficients
        vloc._check(plan.lib.vloc_to_real(plan.handle, vloc._ptr(buf), 2, vloc._ptr(buf[plan.npw:]), None), "x")
    assert e.value.code == -1
