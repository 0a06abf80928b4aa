"""FP64 CPU oracle for the V_loc|psi> hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline (``cpu_baseline`` and ``--impl reference``) may import this module.
It shares no code with the CUDA path (``paper_1601_07378_gb300``) and imports
nothing from it; its inputs come from the seeded generators in
``paper_1601_07378_gb300.synth`` via the caller.

Contents, each citing the passage of Gao, Mo, Fang & Wang (arXiv:1601.07378)
it follows:

* ``apply`` / ``to_real`` / ``grad_V`` / ``axis_dft``: the plain C oracle
  (``vloc_oracle.c``): scatter, naive per-axis DFTs, multiply by V, naive
  inverse, gather (Sec. 2, Eqs. 2-3 and the two-FFT recipe after them).
* ``np_*``: a NumPy restatement of the same definition with an explicit sign
  argument (DFT matrices per axis), and ``bf_*``: the plane-wave sums of
  Eq. 2 written out point by point (brute force, tiny grids only).
* ``closed_form_apply``: for a potential with few Fourier modes the action is
  the convolution out(G) = sum_q v_q c(G - q) (no FFT at all), valid while
  every n_a > 2R + K (no wrap-around, Fig. 1).
* ``gamma_complete`` / ``gamma_apply``: the Gamma-point real mode (Sec. 4.3,
  last paragraph): a band stored on half of the sphere is completed with
  c(-G) = conj c(G) (c(0) real), acted on by ``apply`` and read back on the
  half; ``bf_real_apply`` writes the same action with real plane-wave sums
  (cosines and sines, brute force, tiny grids).
* ``to_recip`` (the r -> G half of the recipe after Eq. 3: naive DFT passes,
  1/N, gather) with its brute force ``bf_to_recip``; ``density`` /
  ``gamma_density``: rho(r) = sum_n f_n |psi_n(r)|^2 (Sec. 3.1, first
  paragraph), from ``to_real``.
* ``kinetic`` / ``dense_h`` / ``lowest_eigs``: the Kohn-Sham Hamiltonian of
  Eq. 1 at the Gamma point with a local potential only, H = |G|^2 / 2 + V_loc,
  as a dense matrix whose columns are ``apply`` on unit vectors plus the
  kinetic diagonal, and its lowest eigenvalues by numpy's dense solver (the
  reference for the iterative eigensolver, Sec. 2: H is applied, never
  assembled, in production).
* ``sticks`` / ``greedy_partition`` (Sec. 3.2, Fig. 2), ``basic_partition``
  (Sec. 4.1, Fig. 3-4) and ``improved_partition`` (Sec. 4.2).

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` except the basic/improved partitions' exact
layouts, whose worked example (Fig. 4) is missing from the paper: parity
unpinned for those two (their invariants and the Tab. 2 ordering are tested).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vloc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


# --------------------------------------------------------------------------
# build / load the plain C oracle
# --------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile vloc_oracle.c with gcc (-O2, OpenMP, IEEE arithmetic)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_index_map.argtypes = [ctypes.c_int] * 3 + [i32p, ctypes.c_int64, i64p]
            lib.oracle_to_real.argtypes = [ctypes.c_int] * 3 + [i32p, ctypes.c_int64, dp, ctypes.c_int64, dp, ctypes.c_int]
            lib.oracle_apply.argtypes = [ctypes.c_int] * 3 + [i32p, ctypes.c_int64, dp, dp, ctypes.c_int64, dp, ctypes.c_int]
            lib.oracle_grad_V.argtypes = [ctypes.c_int] * 3 + [i32p, ctypes.c_int64, dp, dp, ctypes.c_int64, dp, ctypes.c_int]
            lib.oracle_axis_dft.argtypes = [ctypes.c_int] * 3 + [dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_max_threads.argtypes = []
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _glist(g):
    return np.ascontiguousarray(np.asarray(g, dtype=np.int32).reshape(-1, 3))


def _cplx(c):
    c = np.ascontiguousarray(np.asarray(c, dtype=np.complex128))
    return c


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError({-2: "bad size", -3: "bad G-list", -5: "out of memory"}.get(rc, str(rc)))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def index_map(n, g) -> np.ndarray:
    """Grid index ((h mod n1)*n2 + (k mod n2))*n3 + (l mod n3) per G (Eqs. 2-3)."""
    g = _glist(g)
    out = np.empty(len(g), dtype=np.int64)
    _check(_load().oracle_index_map(n[0], n[1], n[2], _p(g, ctypes.c_int32), len(g), _p(out, ctypes.c_int64)))
    return out


def to_real(n, g, c, nthreads: int = 0) -> np.ndarray:
    """psi = F+ S c on the full grid, complex128 [nb, n1, n2, n3]."""
    g = _glist(g)
    c = _cplx(c).reshape(-1, len(g))
    nb = c.shape[0]
    psi = np.empty((nb, n[0], n[1], n[2]), dtype=np.complex128)
    _check(_load().oracle_to_real(n[0], n[1], n[2], _p(g, ctypes.c_int32), len(g),
                                  _p(c.view(np.float64), ctypes.c_double), nb,
                                  _p(psi.view(np.float64), ctypes.c_double), nthreads))
    return psi


def apply(n, g, c, V, nthreads: int = 0) -> np.ndarray:
    """out = (1/N) S^T F- diag(V) F+ S c, complex128 [nb, npw]."""
    g = _glist(g)
    c = _cplx(c).reshape(-1, len(g))
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
    assert V.size == n[0] * n[1] * n[2]
    nb = c.shape[0]
    out = np.empty_like(c)
    _check(_load().oracle_apply(n[0], n[1], n[2], _p(g, ctypes.c_int32), len(g),
                                _p(c.view(np.float64), ctypes.c_double), _p(V, ctypes.c_double), nb,
                                _p(out.view(np.float64), ctypes.c_double), nthreads))
    return out


def grad_V(n, g, c, gout, nthreads: int = 0) -> np.ndarray:
    """dL/dV = (1/N) sum_b Re(conj(F+ S gout_b) * F+ S c_b), float64 [n1, n2, n3]."""
    g = _glist(g)
    c = _cplx(c).reshape(-1, len(g))
    gout = _cplx(gout).reshape(-1, len(g))
    assert c.shape == gout.shape
    dV = np.empty(n[0] * n[1] * n[2], dtype=np.float64)
    _check(_load().oracle_grad_V(n[0], n[1], n[2], _p(g, ctypes.c_int32), len(g),
                                 _p(c.view(np.float64), ctypes.c_double),
                                 _p(gout.view(np.float64), ctypes.c_double), c.shape[0],
                                 _p(dV, ctypes.c_double), nthreads))
    return dV.reshape(n)


def grads(n, g, c, V, gout, nthreads: int = 0):
    """(dL/dc, dL/dV) for out = A c: dL/dc = A^H gout = A gout (V real)."""
    return apply(n, g, gout, V, nthreads), grad_V(n, g, c, gout, nthreads)


def axis_dft(n, grids, axis: int, sign: int, nthreads: int = 0) -> np.ndarray:
    """One naive DFT pass along an axis of full grids (copy returned)."""
    # C order whatever the input's strides: the C side reads the buffer as [nb][n1][n2][n3]
    a = np.array(grids, dtype=np.complex128, order="C", copy=True).reshape(-1, n[0], n[1], n[2])
    _check(_load().oracle_axis_dft(n[0], n[1], n[2], _p(a.view(np.float64), ctypes.c_double),
                                   a.shape[0], axis, sign, nthreads))
    return a


# --------------------------------------------------------------------------
# NumPy restatement (explicit sign) and brute force
# --------------------------------------------------------------------------
def _miller_ok(h, n):
    return (h >= -(n // 2)) & (h <= (n + 1) // 2 - 1)


def np_index_map(n, g) -> np.ndarray:
    g = _glist(g)
    for a in range(3):
        if not np.all(_miller_ok(g[:, a], n[a])):
            raise OracleError("bad G-list")
    idx = ((g[:, 0] % n[0]).astype(np.int64) * n[1] + g[:, 1] % n[1]) * n[2] + g[:, 2] % n[2]
    if len(np.unique(idx)) != len(idx):
        raise OracleError("bad G-list")
    return idx


def _dft_matrix(m: int, sign: int) -> np.ndarray:
    j = np.arange(m)
    t = np.outer(j, j) % m
    return np.exp(sign * 2j * np.pi * t / m)


def np_to_real(n, g, c, sign: int = +1) -> np.ndarray:
    """psi(j) = sum_m Z(m) exp(sign 2 pi i m.j/n), per-axis DFT matrices."""
    g = _glist(g)
    c = _cplx(c).reshape(-1, len(g))
    nb = c.shape[0]
    Z = np.zeros((nb, n[0] * n[1] * n[2]), dtype=np.complex128)
    Z[:, np_index_map(n, g)] = c
    Z = Z.reshape(nb, *n)
    Z = np.einsum("bijk,xi->bxjk", Z, _dft_matrix(n[0], sign))
    Z = np.einsum("bxjk,yj->bxyk", Z, _dft_matrix(n[1], sign))
    Z = np.einsum("bxyk,zk->bxyz", Z, _dft_matrix(n[2], sign))
    return Z


def np_apply(n, g, c, V, sign: int = +1) -> np.ndarray:
    """(1/N) gather(F_{-sign} (V * F_{sign} scatter(c)))."""
    g = _glist(g)
    N = n[0] * n[1] * n[2]
    psi = np_to_real(n, g, c, sign) * np.asarray(V, dtype=np.float64).reshape(n)[None]
    U = np.einsum("bijk,xi->bxjk", psi, _dft_matrix(n[0], -sign))
    U = np.einsum("bxjk,yj->bxyk", U, _dft_matrix(n[1], -sign))
    U = np.einsum("bxyk,zk->bxyz", U, _dft_matrix(n[2], -sign))
    return U.reshape(U.shape[0], -1)[:, np_index_map(n, g)] / N


def bf_to_real(n, g, c) -> np.ndarray:
    """Eq. 2 summed plane wave by plane wave at every grid point (tiny grids)."""
    g = _glist(g)
    c = _cplx(c).reshape(-1, len(g))
    j1, j2, j3 = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    J = np.stack([j1.ravel(), j2.ravel(), j3.ravel()], axis=1)  # [N, 3]
    out = np.zeros((c.shape[0], J.shape[0]), dtype=np.complex128)
    for p in range(len(g)):
        ph = sum(((int(g[p, a]) * J[:, a]) % n[a]) / n[a] for a in range(3))
        out += c[:, p:p + 1] * np.exp(2j * np.pi * ph)[None, :]
    return out.reshape(c.shape[0], *n)


def bf_apply(n, g, c, V) -> np.ndarray:
    """Brute-force action: Eq. 2 sums, times V, projected back on each G."""
    g = _glist(g)
    N = n[0] * n[1] * n[2]
    u = bf_to_real(n, g, c).reshape(-1, N) * np.asarray(V, dtype=np.float64).reshape(1, N)
    j1, j2, j3 = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    J = np.stack([j1.ravel(), j2.ravel(), j3.ravel()], axis=1)
    out = np.zeros((u.shape[0], len(g)), dtype=np.complex128)
    for p in range(len(g)):
        ph = sum(((int(g[p, a]) * J[:, a]) % n[a]) / n[a] for a in range(3))
        out[:, p] = (u * np.exp(-2j * np.pi * ph)[None, :]).sum(axis=1) / N
    return out


def closed_form_apply(g, c, modes) -> np.ndarray:
    """out(G) = sum_q v_q c(G - q), both G and G - q on the list (no FFT)."""
    g = _glist(g)
    c = _cplx(c).reshape(-1, len(g))
    pos = {tuple(int(x) for x in row): i for i, row in enumerate(g)}
    out = np.zeros_like(c)
    for i, row in enumerate(g):
        G = tuple(int(x) for x in row)
        for q, v in modes:
            j = pos.get((G[0] - q[0], G[1] - q[1], G[2] - q[2]))
            if j is not None:
                out[:, i] += v * c[:, j]
    return out


# --------------------------------------------------------------------------
# sticks and the three partitions (Sec. 3.2, 4.1, 4.2)
# --------------------------------------------------------------------------
def gamma_complete(g_half, c_half):
    """Sec. 4.3: Psi(G) = conj Psi(-G).  Full list = the half list followed by
    -G for each G != 0 of it; coefficients completed the same way, with the
    G = 0 coefficient taken real.  Returns (g_full, c_full)."""
    g_half = np.asarray(g_half, dtype=np.int64).reshape(-1, 3)
    c_half = np.asarray(c_half, dtype=np.complex128).reshape(-1, len(g_half))
    nz = np.any(g_half != 0, axis=1)
    g_full = np.concatenate([g_half, -g_half[nz]])
    c0 = c_half.copy()
    c0[:, ~nz] = c0[:, ~nz].real
    c_full = np.concatenate([c0, np.conj(c0[:, nz])], axis=1)
    return g_full.astype(np.int32), c_full


def gamma_apply(n, g_half, c_half, V, nthreads: int = 0) -> np.ndarray:
    """A applied to real bands given on half of the sphere (Sec. 4.3):
    complete, apply (Sec. 2), keep the half list's entries."""
    g_full, c_full = gamma_complete(g_half, c_half)
    return apply(n, g_full, c_full, V, nthreads)[:, :len(g_half)]


def bf_real_psi(n, g_half, c_half) -> np.ndarray:
    """Real bands of the Gamma-point mode summed in real arithmetic (tiny grids):
    psi(r) = Re c(0) + 2 sum_{G != 0 in half} [Re c(G) cos(th) - Im c(G) sin(th)],
    th = 2 pi G.r / n.  float64 [nb, N]."""
    n1, n2, n3 = n
    g_half = np.asarray(g_half, dtype=np.float64).reshape(-1, 3)
    c_half = np.asarray(c_half, dtype=np.complex128).reshape(-1, len(g_half))
    r = np.stack(np.meshgrid(np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3,
                             indexing="ij"), axis=-1).reshape(-1, 3)
    th = 2.0 * np.pi * (r @ g_half.T)                     # [N, nh]
    nz = np.any(g_half != 0, axis=1)
    wc = np.where(nz, 2.0, 1.0)                           # G = 0 counted once
    ws = np.where(nz, 2.0, 0.0)
    return np.stack([np.cos(th) @ (wc * cb.real) - np.sin(th) @ (ws * cb.imag) for cb in c_half])


def bf_real_apply(n, g_half, c_half, V) -> np.ndarray:
    """Real-arithmetic brute force of the Gamma-point action (tiny grids):
    psi from ``bf_real_psi``, then out(G) = (1/N) sum_r V(r) psi(r) (cos(th) - i sin(th))."""
    n1, n2, n3 = n
    N = n1 * n2 * n3
    gh = np.asarray(g_half, dtype=np.float64).reshape(-1, 3)
    r = np.stack(np.meshgrid(np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3,
                             indexing="ij"), axis=-1).reshape(-1, 3)
    th = 2.0 * np.pi * (r @ gh.T)
    f = bf_real_psi(n, g_half, c_half) * np.asarray(V, dtype=np.float64).reshape(1, -1)
    return (f @ np.cos(th) - 1j * (f @ np.sin(th))) / N


# ---- the two halves of the action on their own, and the charge density
def to_recip(n, g, u, nthreads: int = 0) -> np.ndarray:
    """The r -> G half of Sec. 2's two-FFT recipe: out(G) = (1/N) sum_r u(r)
    exp(-2 pi i G.r / n) at the list's G (three naive DFT passes of the C
    oracle, then the gather), complex128 [nb, npw] from u [nb, n1, n2, n3]."""
    N = n[0] * n[1] * n[2]
    a = np.asarray(u, dtype=np.complex128).reshape(-1, n[0], n[1], n[2])
    for axis in range(3):
        a = axis_dft(n, a, axis, -1, nthreads)
    return a.reshape(a.shape[0], N)[:, index_map(n, g)] / N


def bf_to_recip(n, g, u) -> np.ndarray:
    """(1/N) sum_r u(r) exp(-2 pi i G.r / n) summed point by point (tiny grids)."""
    n1, n2, n3 = n
    r = np.stack(np.meshgrid(np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3,
                             indexing="ij"), axis=-1).reshape(-1, 3)
    E = np.exp(-2j * np.pi * (r @ np.asarray(g, dtype=np.float64).T))   # [N, npw]
    return np.asarray(u, dtype=np.complex128).reshape(-1, n1 * n2 * n3) @ E / (n1 * n2 * n3)


def density(n, g, c, occ=None, nthreads: int = 0) -> np.ndarray:
    """Charge density of Sec. 3.1: rho(r) = sum_n f_n |psi_n(r)|^2 with
    psi_n = F+ S c_n (the unnormalised G -> r transform) and f_n = occ[n]
    (1 when occ is None).  float64 [n1, n2, n3]."""
    psi = to_real(n, g, c, nthreads)
    f = np.ones(psi.shape[0]) if occ is None else np.asarray(occ, dtype=np.float64)
    assert f.shape == (psi.shape[0],)
    return np.tensordot(f, psi.real ** 2 + psi.imag ** 2, axes=1)


def gamma_density(n, g_half, c_half, occ=None, nthreads: int = 0) -> np.ndarray:
    """Density of real bands given on half of the sphere (Sec. 4.3): complete, then ``density``."""
    g_full, c_full = gamma_complete(g_half, c_half)
    return density(n, g_full, c_full, occ, nthreads)


def kinetic(g, cell) -> np.ndarray:
    """|G|^2 / 2 with G = 2 pi (h / L1, k / L2, l / L3) for an orthorhombic
    cell of side lengths ``cell`` (Eq. 1's kinetic term at k = 0)."""
    gg = 2.0 * np.pi * np.asarray(g, dtype=np.float64) / np.asarray(cell, dtype=np.float64)[None, :]
    return 0.5 * (gg ** 2).sum(axis=1)


def dense_h(n, g, V, T, nthreads: int = 0) -> np.ndarray:
    """H[:, j] = T_j e_j + A e_j over the plane-wave basis (complex128 [npw, npw])."""
    npw = len(np.asarray(g).reshape(-1, 3))
    cols = apply(n, g, np.eye(npw, dtype=np.complex128), V, nthreads)   # row j = A e_j
    H = cols.T.copy()
    H[np.arange(npw), np.arange(npw)] += np.asarray(T, dtype=np.float64)
    return H


def lowest_eigs(n, g, V, T, k: int, nthreads: int = 0) -> np.ndarray:
    """The k lowest eigenvalues of ``dense_h`` (numpy's Hermitian solver)."""
    return np.linalg.eigvalsh(dense_h(n, g, V, T, nthreads))[:k]


def sticks(n, g):
    """Occupied z-sticks: sorted linear ids (h mod n1)*n2 + (k mod n2) and #PW each."""
    g = _glist(g)
    sid = (g[:, 0] % n[0]).astype(np.int64) * n[1] + (g[:, 1] % n[1])
    ids, counts = np.unique(sid, return_counts=True)
    return ids, counts


def greedy_partition(ids, weights, P: int) -> np.ndarray:
    """Sec. 3.2 / Fig. 2: sort columns by workload descending (ties: ascending
    column id), deal the k-th sorted column to part k mod P.  Returns the part
    of each column, in the order of ``ids``."""
    order = sorted(range(len(ids)), key=lambda i: (-int(weights[i]), int(ids[i])))
    part = np.empty(len(ids), dtype=np.int32)
    for rank, i in enumerate(order):
        part[i] = rank % P
    return part


def process_grid(p: int) -> tuple[int, int]:
    """Sec. 4.1: p = m x n with |m - n| minimal, m the larger (m rows, n columns)."""
    m = next(d for d in range(int(np.ceil(np.sqrt(p))), p + 1) if p % d == 0)
    return m, p // m


def basic_partition(n, g, p: int) -> np.ndarray:
    """Sec. 4.1 basic algorithm on the z-stick (reciprocal) layout, cyclic:
    a stick with first-pass coordinates (a, b) = (h mod n1, k mod n2) goes to
    row a mod m, column b mod n; rank = row * n + col.  Per stick in the order
    of ``sticks``."""
    m, ncol = process_grid(p)
    ids, _ = sticks(n, g)
    a = ids // n[1]
    b = ids % n[1]
    return ((a % m) * ncol + (b % ncol)).astype(np.int32)


def improved_partition(n, g, p: int) -> np.ndarray:
    """Sec. 4.2: plane weights = #PW per plane; planes sorted by weight
    (descending, ties ascending index) and dealt round-robin: planes of
    constant b = k mod n2 to column groups, planes of constant a = h mod n1 to
    row groups.  rank = row * n + col, per stick in the order of ``sticks``."""
    m, ncol = process_grid(p)
    ids, w = sticks(n, g)
    a = ids // n[1]
    b = ids % n[1]
    wa = np.bincount(a, weights=w, minlength=n[0])
    wb = np.bincount(b, weights=w, minlength=n[1])
    row_of = np.empty(n[0], dtype=np.int64)
    for rank, i in enumerate(sorted(range(n[0]), key=lambda i: (-wa[i], i))):
        row_of[i] = rank % m
    col_of = np.empty(n[1], dtype=np.int64)
    for rank, i in enumerate(sorted(range(n[1]), key=lambda i: (-wb[i], i))):
        col_of[i] = rank % ncol
    return (row_of[a] * ncol + col_of[b]).astype(np.int32)


def part_loads(part: np.ndarray, weights: np.ndarray, P: int) -> np.ndarray:
    return np.bincount(part, weights=weights, minlength=P).astype(np.int64)
