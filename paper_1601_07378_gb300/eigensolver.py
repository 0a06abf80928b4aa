"""Lowest eigenpairs of H = |k+G|^2/2 + V_loc by Chebyshev-filtered subspace
iteration, with the V_loc action as the matrix-vector product.

Sec. 2 of the paper: the Hamiltonian is never assembled; iterative
diagonalisation applies it to blocks of trial bands, and each application
costs the two 3-D FFTs of the V_loc action.  Here the block apply is
``VlocPlan.apply_h`` (one pass of the GPU chain with the kinetic term added
in the gather), and the small dense steps (Gram matrices, QR
orthonormalisation, the Rayleigh-Ritz eigenproblem) are cuBLAS / cuSOLVER
calls through torch on the same device.

Filter: the scaled three-term Chebyshev recurrence of degree m damps the
spectrum above the block's largest Ritz value a towards the upper bound b
(lambda_max <= max T + max V, since ||A|| <= max |V|) and amplifies the
wanted part below a (Zhou, Saad, Tiago and Chelikowsky, J. Comput. Phys.
219 (2006) 172).

For Gamma-point plans (real bands on half of the sphere) inner products
count every G != 0 twice and take the real part, so the subspace matrices
are real symmetric.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field


@dataclass
class EigResult:
    eigenvalues: "object"          # torch real [nev]
    vectors: "object"              # torch complex [nev, npw]
    residuals: "object"            # torch real [nev], ||H x - lambda x||
    iterations: int
    h_applies: int                 # band applies of H (bands x calls)
    history: list = field(default_factory=list)


class Hamiltonian:
    """H = diag(T) + A on one plan: T = |k+G|^2 / 2 for an orthorhombic cell
    of side lengths ``cell`` (k = 0), or any real diagonal given as ``T``."""

    def __init__(self, plan, V, *, cell=None, T=None):
        import numpy as np
        import torch
        self.plan, self.V = plan, V
        if T is None:
            g = np.asarray(plan_glist(plan), dtype=np.float64)
            gg = 2.0 * math.pi * g / np.asarray(cell, dtype=np.float64)[None, :]
            T = torch.from_numpy(0.5 * (gg ** 2).sum(axis=1))
        self.T = T.to(device=V.device, dtype=plan.real_dtype).contiguous()
        self.gamma = bool(getattr(plan, "gamma", False))
        if self.gamma:
            g = np.asarray(plan_glist(plan))
            w = np.where(np.any(g != 0, axis=1), 2.0, 1.0)
            self.w = torch.from_numpy(w).to(device=V.device, dtype=plan.real_dtype)
        else:
            self.w = None
        self.applies = 0

    def __call__(self, X, out=None):
        self.applies += X.shape[0]
        return self.plan.apply_h(X, self.V, self.T, out)

    def upper_bound(self) -> float:
        return float(self.T.max()) + float(self.V.max())

    # inner products: [nb, npw] x [nb', npw] -> [nb, nb'] (real for Gamma-point
    # bands: every combination of real bands must stay real)
    def gram(self, X, Y):
        if self.w is None:
            return X.conj() @ Y.transpose(0, 1)
        return ((X.conj() * self.w) @ Y.transpose(0, 1)).real

    def combine(self, M, X):
        """Rows M X for a coefficient matrix M (real for Gamma-point bands)."""
        return M.to(X.dtype) @ X

    def norms(self, X):
        if self.w is None:
            return X.abs().pow(2).sum(dim=1).sqrt()
        return (X.abs().pow(2) * self.w).sum(dim=1).sqrt()


def plan_glist(plan):
    """The plan's G-list as given by the caller (kept on the Python side)."""
    g = getattr(plan, "glist", None)
    if g is None:
        raise ValueError("plan has no G-list attached")
    return g


def _orthonormalize(H: Hamiltonian, X):
    """Rows of X made orthonormal in H's inner product by a Householder QR of
    the bands as columns (stable for the badly conditioned filtered blocks;
    Gamma-point bands as real vectors [sqrt(w) Re x, sqrt(w) Im x])."""
    import torch
    if H.w is None:
        Q, _ = torch.linalg.qr(X.transpose(0, 1))
        return Q.transpose(0, 1).contiguous()
    sw = H.w.sqrt()
    M = torch.cat([(X.real * sw).transpose(0, 1), (X.imag * sw).transpose(0, 1)], dim=0)
    Q, _ = torch.linalg.qr(M)
    npw = X.shape[1]
    re = Q[:npw].transpose(0, 1) / sw
    im = Q[npw:].transpose(0, 1) / sw
    return torch.complex(re, im).to(X.dtype).contiguous()


def _rayleigh_ritz(H: Hamiltonian, X, HX):
    import torch
    Hs = H.gram(X, HX)
    Hs = 0.5 * (Hs + Hs.conj().transpose(0, 1))
    lam, Q = torch.linalg.eigh(Hs)
    # Hs[i, j] = <x_i|H|x_j>, so Ritz vector k is sum_j Q[j, k] x_j: as rows,
    # X' = Q^T X (and the same rotation of H X)
    Qt = Q.transpose(0, 1)
    return lam, H.combine(Qt, X), H.combine(Qt, HX)


def chebyshev_filter(H: Hamiltonian, X, degree: int, a: float, b: float, a0: float):
    """p_m(H) X for the scaled Chebyshev polynomial that is small on [a, b]
    and grows below a (normalised at a0 < a)."""
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    sigma = e / (a0 - c)
    sigma1 = sigma
    Y = (H(X) - c * X) * (sigma1 / e)
    for _ in range(2, degree + 1):
        sigma2 = 1.0 / (2.0 / sigma1 - sigma)
        Ynew = (H(Y) - c * Y) * (2.0 * sigma2 / e) - (sigma * sigma2) * X
        X, Y = Y, Ynew
        sigma = sigma2
    return Y


def chfsi(H: Hamiltonian, nev: int, *, nblock: int | None = None, degree: int = 12, tol: float = 1e-6,
          maxiter: int = 100, seed: int = 0, X0=None) -> EigResult:
    """Lowest ``nev`` eigenpairs of H by Chebyshev-filtered subspace iteration
    on a block of ``nblock`` bands (default nev + max(8, nev // 4)).
    Converged when every wanted residual ||H x - lambda x|| < tol * max(1, |lambda|)."""
    import torch
    plan = H.plan
    npw = plan.npw
    nb = nblock or nev + max(8, nev // 4)
    if nb > npw:
        raise ValueError("block larger than the basis")
    dev = H.V.device
    if X0 is None:
        # seeded random start, drawn on the device; smooth bands (large |G| damped)
        gen = torch.Generator(device=dev).manual_seed(seed)
        rdt = plan.real_dtype
        X = torch.complex(torch.randn(nb, npw, generator=gen, dtype=rdt, device=dev),
                          torch.randn(nb, npw, generator=gen, dtype=rdt, device=dev))
        X = (X / (1.0 + H.T)[None, :]).to(plan.dtype)
    else:
        X = X0.to(device=dev, dtype=plan.dtype).clone()
    if H.gamma:
        g = plan_glist(plan)
        import numpy as np
        z = np.flatnonzero(~np.any(np.asarray(g) != 0, axis=1))
        if len(z):
            X[:, int(z[0])] = X[:, int(z[0])].real.to(X.dtype)
    X = _orthonormalize(H, X)
    HX = H(X)
    lam, X, HX = _rayleigh_ritz(H, X, HX)
    b_up = H.upper_bound()
    hist = []
    res = None
    it = 0
    for it in range(1, maxiter + 1):
        R = HX - lam.to(X.dtype)[:, None] * X
        res = H.norms(R)
        scale = torch.clamp(lam.abs(), min=1.0)
        hist.append(float((res[:nev] / scale[:nev]).max()))
        if hist[-1] < tol:
            break
        a = float(lam[-1])
        a0 = float(lam[0])
        if a >= b_up:
            b_up = a + 1.0
        Y = chebyshev_filter(H, X, degree, a, b_up, a0)
        X = _orthonormalize(H, Y)
        HX = H(X)
        lam, X, HX = _rayleigh_ritz(H, X, HX)
    R = HX - lam.to(X.dtype)[:, None] * X
    res = H.norms(R)
    return EigResult(lam[:nev], X[:nev], res[:nev], it, H.applies, hist)
