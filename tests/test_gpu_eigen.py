"""Second workload: lowest eigenpairs of H = |G|^2/2 + V_loc (Eq. 1 at the
Gamma point, local potential only) by Chebyshev-filtered subspace iteration
whose matrix-vector product is the GPU H apply (vloc_apply_h), against the
oracle's dense Hamiltonian (columns = the oracle's action on unit vectors)
diagonalised by numpy."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_07378_gb300 import eigensolver as E
from paper_1601_07378_gb300 import synth, vloc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f32": (torch.complex64, torch.float32), "f64": (torch.complex128, torch.float64)}
CELL = (9.0, 9.5, 10.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1601_07378_gb300.build import build
    build()


def _potential(n):
    V, _ = synth.potential(*n, "smooth", seed=17)
    return -4.0 * (V - V.min())          # wells of a few hartree


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_apply_h_matches_oracle(prec):
    cd, rd = DT[prec]
    n = (24, 20, 30)
    g = synth.sphere_glist(*n, 5, order="shuffled", seed=1)
    c = synth.coefficients(g, 5, seed=2).astype(np.complex64 if prec == "f32" else np.complex128)
    V = _potential(n).astype(np.float32 if prec == "f32" else np.float64)
    T = O.kinetic(g, CELL)
    plan = vloc.VlocPlan(n, g, cd, chunk=2)
    ct = torch.from_numpy(c).cuda()
    out = plan.apply_h(ct, torch.from_numpy(V).cuda(), torch.from_numpy(T).to("cuda", rd))
    torch.cuda.synchronize()
    cc = c.astype(np.complex128)
    ref = T[None, :] * cc + O.apply(n, g, cc, V.astype(np.float64))
    err = np.linalg.norm(out.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() < {"f32": 2e-6, "f64": 1e-12}[prec]
    # exact alias out == c
    out2 = plan.apply_h(ct, torch.from_numpy(V).cuda(), torch.from_numpy(T).to("cuda", rd), out=ct)
    torch.cuda.synchronize()
    assert torch.equal(out2, out)


def test_gamma_apply_h_matches_oracle():
    n = (24, 24, 24)
    gh = synth.half_sphere(synth.sphere_glist(*n, 6))
    c = synth.coefficients(gh, 5, seed=3)
    V = _potential(n)
    T = O.kinetic(gh, CELL)
    plan = vloc.VlocPlan(n, gh, torch.complex128, gamma=True)
    out = plan.apply_h(torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(T).cuda())
    torch.cuda.synchronize()
    g0 = ~np.any(gh != 0, axis=1)
    creal = c.copy()
    creal[:, g0] = creal[:, g0].real
    ref = T[None, :] * creal + O.gamma_apply(n, gh, c, V)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 2e-4)])
@pytest.mark.parametrize("gamma", [False, True])
def test_chfsi_lowest_eigenvalues(prec, tol, gamma):
    cd, rd = DT[prec]
    n, R, nev = (24, 24, 24), 6, 12
    g = synth.sphere_glist(*n, R)
    V = _potential(n)
    want = O.lowest_eigs(n, g, V, O.kinetic(g, CELL), nev)
    gl = synth.half_sphere(g) if gamma else g
    plan = vloc.VlocPlan(n, gl, cd, gamma=gamma)
    H = E.Hamiltonian(plan, torch.from_numpy(V).to("cuda", rd), cell=CELL)
    res = E.chfsi(H, nev, tol=tol, maxiter=60, seed=1)
    torch.cuda.synchronize()
    lam = res.eigenvalues.double().cpu().numpy()
    assert res.history[-1] < tol, res.history
    assert np.abs(lam - want).max() < {"f64": 1e-8, "f32": 5e-4}[prec] * max(1.0, np.abs(want).max()), (lam, want)
    # eigenvectors orthonormal in the plan's inner product
    X = res.vectors
    S = H.gram(X, X)
    eye = torch.eye(nev, dtype=S.dtype, device=S.device)
    assert (S - eye).abs().max() < {"f64": 1e-10, "f32": 1e-4}[prec]
