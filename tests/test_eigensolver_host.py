"""The eigensolver's host algebra on CPU (no GPU): Chebyshev filter, QR
orthonormalisation, Rayleigh-Ritz and the Gamma-point inner products.

The H apply is a stand-in plan whose ``apply_h`` is the FP64 oracle's action
plus the kinetic diagonal, so the only code under test is the solver; its
lowest eigenvalues must equal numpy's dense eigenvalues of the oracle's H
(Eq. 1 at the Gamma point with a local potential only).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_07378_gb300 import eigensolver as E, synth

torch = pytest.importorskip("torch")

N3, R, CELL, NEV = (24, 24, 24), 6, (9.0, 9.5, 10.0), 12


class OraclePlan:
    """The plan interface the solver uses, acting through the oracle (FP64)."""

    def __init__(self, n, g, gamma=False):
        self.n, self.glist, self.npw, self.gamma = n, np.asarray(g), len(g), gamma
        self.dtype, self.real_dtype = torch.complex128, torch.float64

    def apply_h(self, X, V, T, out=None):
        x, v, t = X.numpy(), V.numpy(), T.numpy()
        a = O.gamma_apply(self.n, self.glist, x, v) if self.gamma else O.apply(self.n, self.glist, x, v)
        y = a + t[None, :] * x
        if self.gamma:      # a real band's c(0) is real: its imaginary part is not part of the band
            z = ~np.any(self.glist != 0, axis=1)
            y[:, z] = t[None, z] * x[:, z].real + a[:, z]
        return torch.from_numpy(y)


@pytest.fixture(scope="module")
def case():
    O.build()
    g = synth.sphere_glist(*N3, R)
    V, _ = synth.potential(*N3, "smooth", seed=17)
    V = -4.0 * (V - V.min())
    return g, V, O.lowest_eigs(N3, g, V, O.kinetic(g, CELL), NEV)


@pytest.mark.parametrize("gamma", [False, True])
def test_chfsi_finds_the_dense_lowest_eigenvalues(case, gamma):
    g, V, want = case
    gl = synth.half_sphere(g) if gamma else g
    H = E.Hamiltonian(OraclePlan(N3, gl, gamma), torch.from_numpy(V), cell=CELL)
    res = E.chfsi(H, NEV, tol=1e-9, maxiter=60, seed=1)
    assert np.abs(res.eigenvalues.numpy() - want).max() < 1e-8
    assert res.history[-1] < 1e-9
    # Ritz vectors orthonormal in H's inner product (weights 2 for G != 0 on the half)
    Gm = H.gram(res.vectors, res.vectors).numpy()
    assert np.abs(Gm - np.eye(NEV)).max() < 1e-10
    if gamma:
        assert np.isrealobj(Gm) or np.abs(np.imag(Gm)).max() == 0.0


def test_orthonormalize_in_the_gamma_inner_product(case):
    g, V, _ = case
    gl = synth.half_sphere(g)
    H = E.Hamiltonian(OraclePlan(N3, gl, True), torch.from_numpy(V), cell=CELL)
    rng = np.random.default_rng(3)
    X = torch.from_numpy(rng.standard_normal((10, len(gl))) + 1j * rng.standard_normal((10, len(gl))))
    Q = E._orthonormalize(H, X)
    assert np.abs(H.gram(Q, Q).numpy() - np.eye(10)).max() < 1e-12
    # same span: Q's rows reproduce X's rows exactly in that inner product
    C = H.gram(Q, X).numpy()                        # coefficients <q_i, x_j>
    back = C.T @ Q.numpy()
    w = H.w.numpy()
    err = np.sqrt((np.abs(back - X.numpy()) ** 2 * w).sum()) / np.sqrt((np.abs(X.numpy()) ** 2 * w).sum())
    assert err < 1e-12
