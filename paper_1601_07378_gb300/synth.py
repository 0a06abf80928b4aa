"""Seeded synthetic inputs shaped like plane-wave DFT workloads.

This module only *generates inputs*: G-vector lists, plane-wave coefficients
and a real local potential V(r).  It holds none of the V_loc action's
arithmetic (no scatter, no FFT, no multiply-by-V, no gather) and is the one
module shared by the CUDA path's tests/bench and by the CPU oracle.

Workload recipe (the paper's own 500-atom Al run is not available, so these
stand in for it; the shapes follow the paper's setting: a grid about four
times the cut-off radius, a full cut-off sphere and about 10^3 bands):

* G-list: every integer Miller triple (h, k, l) with h^2 + k^2 + l^2 <= R^2
  (cut-off sphere of Eq. 3 in integer grid units; the configs use "<=").
  Canonical order: sorted by (h mod n1, k mod n2), then l ascending from -L
  to L, so each (h, k) stick is one contiguous run.
* Coefficients: c(G) = (a + i b) / (1 + |G|^2), a, b ~ N(0, 1), NumPy PCG64,
  band-major [nbands][npw].
* Potential: real V(r) = sum_q v_q exp(+2 pi i q.r / n) with v_{-q} = conj(v_q)
  ("few": v_0 = 1 plus three random modes and their conjugates, |q|_inf <= 3;
  "smooth": every q with |q|_inf <= 4, amplitude 0.25 exp(-|q|^2 / 8)).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "sphere_glist",
    "half_sphere",
    "canonical_order",
    "coefficients",
    "potential_modes",
    "potential_on_grid",
    "potential",
    "WORKLOADS",
]


def _valid_range(n: int) -> tuple[int, int]:
    """Miller index range that maps one-to-one onto 0..n-1 by h mod n."""
    return -(n // 2), (n + 1) // 2 - 1


def canonical_order(g: np.ndarray, n1: int, n2: int, n3: int) -> np.ndarray:
    """Permutation that sorts a G-list by (h mod n1, k mod n2, l)."""
    g = np.asarray(g)
    return np.lexsort((g[:, 2], g[:, 1] % n2, g[:, 0] % n1))


def sphere_glist(n1: int, n2: int, n3: int, R: float, *, strict: bool = False,
                 order: str = "canonical", seed: int = 0, R2: int | None = None) -> np.ndarray:
    """Integer Miller triples inside the cut-off sphere, int32 [npw, 3].

    ``strict`` selects ``<`` (Eq. 3 as printed) instead of ``<=``; ``R2``
    (an integer squared radius) overrides ``R * R`` in the test.
    ``order`` is "canonical" (stick-contiguous) or "shuffled" (a seeded
    random permutation, to exercise arbitrary caller orderings).
    """
    if R2 is None:
        R2 = R * R
    else:
        R = float(np.sqrt(R2))
    r = int(np.floor(R))
    lo = [max(-r, _valid_range(n)[0]) for n in (n1, n2, n3)]
    hi = [min(r, _valid_range(n)[1]) for n in (n1, n2, n3)]
    h, k, l = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                          np.arange(lo[2], hi[2] + 1), indexing="ij")
    d2 = h * h + k * k + l * l
    keep = d2 < R2 if strict else d2 <= R2
    g = np.stack([h[keep], k[keep], l[keep]], axis=1).astype(np.int32)
    g = g[canonical_order(g, n1, n2, n3)]
    if order == "shuffled":
        g = g[np.random.default_rng(seed + 77).permutation(len(g))]
    elif order != "canonical":
        raise ValueError(order)
    return np.ascontiguousarray(g)


def half_sphere(g: np.ndarray) -> np.ndarray:
    """One of each pair {G, -G} of a G -> -G symmetric list, plus G = 0, in
    the list's order: h > 0, or h = 0 and k > 0, or h = k = 0 and l >= 0.
    The input list of the Gamma-point real mode (Sec. 4.3)."""
    g = np.asarray(g)
    h, k, l = g[:, 0], g[:, 1], g[:, 2]
    keep = (h > 0) | ((h == 0) & (k > 0)) | ((h == 0) & (k == 0) & (l >= 0))
    return np.ascontiguousarray(g[keep])


def coefficients(g: np.ndarray, nbands: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """c(G) = (a+ib)/(1+|G|^2), a,b ~ N(0,1) from PCG64(seed), [nbands][npw]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    npw = len(g)
    a = rng.standard_normal((nbands, npw))
    b = rng.standard_normal((nbands, npw))
    g2 = (np.asarray(g, dtype=np.float64) ** 2).sum(axis=1)
    c = (a + 1j * b) / (1.0 + g2)[None, :]
    return np.ascontiguousarray(c.astype(dtype))


def potential_modes(kind: str, seed: int) -> list[tuple[tuple[int, int, int], complex]]:
    """Fourier modes {q: v_q} of a real potential (Hermitian: v_{-q} = conj v_q)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    modes: dict[tuple[int, int, int], complex] = {(0, 0, 0): 1.0 + 0j}
    if kind == "few":
        while len(modes) < 7:
            q = tuple(int(x) for x in rng.integers(-3, 4, size=3))
            mq = (-q[0], -q[1], -q[2])
            if q == (0, 0, 0) or q in modes or mq in modes:
                continue
            v = complex(rng.normal(0.0, np.sqrt(0.125)), rng.normal(0.0, np.sqrt(0.125)))
            modes[q] = v
            modes[mq] = v.conjugate()
    elif kind == "smooth":
        K = 4
        for q1 in range(-K, K + 1):
            for q2 in range(-K, K + 1):
                for q3 in range(-K, K + 1):
                    q = (q1, q2, q3)
                    mq = (-q1, -q2, -q3)
                    if q == (0, 0, 0) or q in modes:
                        continue
                    amp = 0.25 * np.exp(-(q1 * q1 + q2 * q2 + q3 * q3) / 8.0)
                    v = amp * complex(rng.standard_normal(), rng.standard_normal()) / np.sqrt(2.0)
                    modes[q] = v
                    modes[mq] = v.conjugate()
    elif kind == "constant":
        pass
    else:
        raise ValueError(kind)
    return sorted(modes.items())


def potential_on_grid(modes, n1: int, n2: int, n3: int) -> np.ndarray:
    """Evaluate V(j) = sum_q v_q exp(+2 pi i q.j/n) on the grid, float64 [n1,n2,n3].

    Separable evaluation over the (small) set of mode components; the
    imaginary part cancels by Hermitian symmetry and is dropped.
    """
    qs = np.array([q for q, _ in modes], dtype=np.int64)
    vs = np.array([v for _, v in modes], dtype=np.complex128)
    K = int(np.abs(qs).max()) if len(qs) else 0
    span = 2 * K + 1
    cube = np.zeros((span, span, span), dtype=np.complex128)
    for (q1, q2, q3), v in zip(qs, vs):
        cube[q1 + K, q2 + K, q3 + K] += v
    def phases(n):
        q = np.arange(-K, K + 1)[:, None]
        j = np.arange(n)[None, :]
        return np.exp(2j * np.pi * ((q * j) % n) / n)
    E1, E2, E3 = phases(n1), phases(n2), phases(n3)
    V = np.einsum("abc,ai,bj,ck->ijk", cube, E1, E2, E3, optimize=True)
    return np.ascontiguousarray(V.real)


def potential(n1: int, n2: int, n3: int, kind: str, seed: int):
    """(V on the grid, modes)."""
    modes = potential_modes(kind, seed)
    return potential_on_grid(modes, n1, n2, n3), modes


# Workloads: grid, cut-off radius (grid units), bands, potential kind, seed.
WORKLOADS = {
    "c0_24": dict(grid=(24, 24, 24), R=6, nbands=1, vkind="few", seed=0),
    "c1_64": dict(grid=(64, 64, 64), R=16, nbands=256, vkind="smooth", seed=1),
    "c2_96x96x120": dict(grid=(96, 96, 120), R=24, nbands=1024, vkind="smooth", seed=2),
    "head_96": dict(grid=(96, 96, 96), R=24, nbands=1024, vkind="smooth", seed=2),
    "c4_96": dict(grid=(96, 96, 96), R=24, nbands=512, vkind="smooth", seed=4),
    "fd_32": dict(grid=(32, 32, 32), R=8, nbands=2, vkind="smooth", seed=4),
}

# Uneven multi-instance batch: grids n^3 with R = n/4 and 64*(i+1) bands.
BATCH_GRIDS = [48, 60, 72, 96, 100, 120, 128, 144]
