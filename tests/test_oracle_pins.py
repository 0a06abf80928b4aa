"""Pins of the FP64 CPU oracle to things other than itself (CPU only).

Each test fixes the oracle against the mathematics or the paper: brute-force
plane-wave sums (Eq. 2), single plane waves, constant V, the few-mode closed
form (Fig. 1 without wrap-around), Parseval, Hermiticity, the library FFT,
the sign reading of Eq. 2, the compact-FFT support claims (Sec. 4.3,
Fig. 5), finite-difference gradients and the partitions of Sec. 3.2 / 4.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_07378_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _inner(a, b):
    return np.vdot(a.ravel(), b.ravel())


TINY = [((4, 6, 5), 2.2), ((6, 5, 4), 2.0), ((8, 8, 8), 2.5)]


# ---------------------------------------------------------------- index map
def test_index_map_definition():
    n = (6, 5, 4)
    g = synth.sphere_glist(*n, 2.0, order="shuffled", seed=3)
    idx = O.index_map(n, g)
    for p, (h, k, l) in enumerate(g):
        assert idx[p] == ((h % n[0]) * n[1] + (k % n[1])) * n[2] + (l % n[2])
    assert np.array_equal(idx, O.np_index_map(n, g))


@pytest.mark.parametrize("bad", [
    [[0, 0, 0], [1, 1, 1], [0, 0, 0]],   # duplicate G
    [[0, 3, 0]],                          # k = 3 outside [-2, 2] for n2 = 5
    [[-4, 0, 0]],                         # h = -4 outside [-3, 2] for n1 = 6
    [[0, 0, 2]],                          # l = 2 outside [-2, 1] for n3 = 4
])
def test_index_map_rejects(bad):
    n = (6, 5, 4)
    g = np.array(bad, dtype=np.int32)
    with pytest.raises(O.OracleError):
        O.index_map(n, g)
    with pytest.raises(O.OracleError):
        O.np_index_map(n, g)


def test_sphere_counts():
    # Exact counts of h^2+k^2+l^2 <= R^2 and of occupied (h, k) sticks.
    for n, R, npw, S in [((24, 24, 24), 6, 925, 113), ((64, 64, 64), 16, 17077, 797),
                         ((96, 96, 120), 24, 57777, 1793), ((96, 96, 96), 24, 57777, 1793)]:
        g = synth.sphere_glist(*n, R)
        ids, w = O.sticks(n, g)
        assert len(g) == npw and len(ids) == S and w.sum() == npw


def test_paper_workload_is_context_only():
    d = json.load(open(os.path.join(GOLDEN, "paper_workload.json")))
    counts = {r2: len(synth.sphere_glist(80, 80, 80, 0, R2=r2)) for r2 in (411, 412, 413)}
    assert counts == {411: 35033, 412: 35033, 413: 35273}
    assert d["npw"] not in counts.values()


# ---------------------------------------------------------------- transforms
def test_hand_worked_1x1x4():
    d = json.load(open(os.path.join(GOLDEN, "hand_1x1x4.json")))
    n = tuple(d["grid"])
    g = np.array(d["glist"], dtype=np.int32)
    c = (np.array(d["coeffs_re"]) + 1j * np.array(d["coeffs_im"]))[None]
    psi = O.to_real(n, g, c).ravel()
    np.testing.assert_allclose(psi, np.array(d["psi_re"]) + 1j * np.array(d["psi_im"]), atol=1e-15)
    out = O.apply(n, g, c, np.array(d["V"]))
    np.testing.assert_allclose(out.ravel(), np.array(d["out_re"]) + 1j * np.array(d["out_im"]), atol=1e-15)


@pytest.mark.parametrize("n,R", TINY)
def test_bruteforce_to_real(n, R):
    g = synth.sphere_glist(*n, R, order="shuffled", seed=1)
    c = synth.coefficients(g, 2, seed=5)
    ref = O.bf_to_real(n, g, c)
    assert _rel(O.to_real(n, g, c), ref) < 1e-13
    assert _rel(O.np_to_real(n, g, c), ref) < 1e-13


@pytest.mark.parametrize("n,R", TINY[:2])
def test_bruteforce_apply(n, R):
    g = synth.sphere_glist(*n, R, order="shuffled", seed=2)
    c = synth.coefficients(g, 2, seed=6)
    V, _ = synth.potential(*n, "smooth", seed=7)
    ref = O.bf_apply(n, g, c, V)
    assert _rel(O.apply(n, g, c, V), ref) < 1e-13


def test_single_plane_wave():
    n = (8, 6, 10)
    g = synth.sphere_glist(*n, 2.5)
    j1, j2, j3 = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    for p in [0, 7, len(g) // 2, len(g) - 1]:
        c = np.zeros((1, len(g)), dtype=np.complex128)
        c[0, p] = 1.0
        h, k, l = (int(x) for x in g[p])
        ph = ((h * j1) % n[0]) / n[0] + ((k * j2) % n[1]) / n[1] + ((l * j3) % n[2]) / n[2]
        assert np.abs(O.to_real(n, g, c)[0] - np.exp(2j * np.pi * ph)).max() < 1e-14


def test_constant_potential_is_scalar_multiply():
    n = (12, 10, 9)
    g = synth.sphere_glist(*n, 3.0, order="shuffled", seed=4)
    c = synth.coefficients(g, 3, seed=8)
    out = O.apply(n, g, c, np.full(n, 1.75))
    assert np.abs(out - 1.75 * c).max() < 1e-14


@pytest.mark.parametrize("n,R,kind", [((24, 24, 24), 6, "few"), ((32, 32, 32), 8, "smooth"),
                                      ((20, 18, 22), 4, "smooth")])
def test_closed_form_convolution(n, R, kind):
    # n_a > 2R + K (K = 3 or 4): the periodic product has no wrap-around on
    # the sphere, so out(G) = sum_q v_q c(G - q) exactly (Fig. 1 discussion).
    g = synth.sphere_glist(*n, R, order="shuffled", seed=9)
    c = synth.coefficients(g, 2, seed=10)
    V, modes = synth.potential(*n, kind, seed=11)
    assert min(n) > 2 * R + max(max(abs(x) for x in q) for q, _ in modes)
    assert _rel(O.apply(n, g, c, V), O.closed_form_apply(g, c, modes)) < 1e-13


def test_wraparound_appears_when_grid_too_small():
    # Negative control for the closed form: n < 2R + K folds terms back (Fig. 1).
    n = (10, 10, 10)
    g = synth.sphere_glist(*n, 4)
    c = synth.coefficients(g, 1, seed=12)
    V, modes = synth.potential(*n, "smooth", seed=13)
    assert _rel(O.apply(n, g, c, V), O.closed_form_apply(g, c, modes)) > 1e-6


def test_parseval():
    n = (16, 12, 15)
    g = synth.sphere_glist(*n, 5)
    c = synth.coefficients(g, 2, seed=14)
    psi = O.to_real(n, g, c)
    N = np.prod(n)
    lhs = (np.abs(psi) ** 2).reshape(2, -1).sum(1)
    rhs = N * (np.abs(c) ** 2).sum(1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)


def test_hermiticity_and_definiteness():
    n = (16, 15, 12)
    g = synth.sphere_glist(*n, 5, order="shuffled", seed=15)
    c = synth.coefficients(g, 2, seed=16)
    V, _ = synth.potential(*n, "smooth", seed=17)
    phi, psi = c[0], c[1]
    A_psi = O.apply(n, g, psi, V)[0]
    A_phi = O.apply(n, g, phi, V)[0]
    lhs, rhs = _inner(phi, A_psi), _inner(A_phi, psi)
    assert abs(lhs - rhs) < 1e-14 * abs(lhs)
    e = _inner(psi, A_psi)
    assert abs(e.imag) < 1e-15 * abs(e)
    Vpos = 1.0 + 0.5 * np.cos(2 * np.pi * np.arange(n[0]) / n[0])[:, None, None] * np.ones(n)
    e = _inner(psi, O.apply(n, g, psi, Vpos)[0])
    assert e.real > 0.5 * np.vdot(psi, psi).real


def test_library_fft_cross_check():
    # Check only (not part of either path): numpy's FFT conventions.
    n = (12, 20, 18)
    g = synth.sphere_glist(*n, 4.5, order="shuffled", seed=18)
    c = synth.coefficients(g, 2, seed=19)
    V, _ = synth.potential(*n, "smooth", seed=20)
    N = np.prod(n)
    idx = O.np_index_map(n, g)
    Z = np.zeros((2, N), dtype=np.complex128)
    Z[:, idx] = c
    psi = N * np.fft.ifftn(Z.reshape(2, *n), axes=(1, 2, 3))
    assert _rel(O.to_real(n, g, c), psi) < 1e-13
    out = np.fft.fftn(V[None] * psi, axes=(1, 2, 3)).reshape(2, -1)[:, idx] / N
    assert _rel(O.apply(n, g, c, V), out) < 1e-13


def test_sign_reading_of_eq2():
    # Eq. 2 as printed (e^{-iG.r}) equals our e^{+iG.r} operator on the
    # negated G-list (the reading of the sign).
    n = (12, 10, 14)
    g = synth.sphere_glist(*n, 3.5, order="shuffled", seed=21)
    # keep only G whose negation is also a valid index, so both lists are legal
    ok = np.all([(g[:, a] > -(n[a] // 2)) for a in range(3)], axis=0)
    g = g[ok]
    c = synth.coefficients(g, 2, seed=22)
    V, _ = synth.potential(*n, "smooth", seed=23)
    paper = O.np_apply(n, g, c, V, sign=-1)
    ours = O.apply(n, -g, c, V)
    assert _rel(ours, paper) < 1e-13
    assert _rel(O.apply(n, g, c, V), paper) > 1e-3  # the sign does matter


def test_c_oracle_matches_numpy_mirror():
    n, R = (24, 24, 24), 6
    g = synth.sphere_glist(*n, R)
    c = synth.coefficients(g, 2, seed=0)
    V, _ = synth.potential(*n, "few", seed=1000)
    assert _rel(O.apply(n, g, c, V), O.np_apply(n, g, c, V)) < 1e-14


def test_compact_fft_supports():
    # Sec. 4.3 / Fig. 5: after the first pass only the columns that meet the
    # sphere (the cylinder of sticks) are nonzero; after the second pass only
    # the planes that meet the cylinder (the cuboid).
    n, R = (16, 16, 16), 5
    g = synth.sphere_glist(*n, R)
    c = synth.coefficients(g, 1, seed=24)
    Z = np.zeros(np.prod(n), dtype=np.complex128)
    Z[O.index_map(n, g)] = c[0]
    Z = Z.reshape(n)
    ids, _ = O.sticks(n, g)
    stick_mask = np.zeros((n[0], n[1]), dtype=bool)
    stick_mask[ids // n[1], ids % n[1]] = True
    z1 = O.axis_dft(n, Z, axis=2, sign=+1)[0]
    assert np.all(np.abs(z1[~stick_mask]) == 0) and np.all(np.abs(z1[stick_mask]).sum(-1) > 0)
    z2 = O.axis_dft(n, z1, axis=1, sign=+1)[0]
    planes = np.zeros(n[0], dtype=bool)
    planes[np.unique(ids // n[1])] = True
    assert np.all(np.abs(z2[~planes]) == 0) and np.all(np.abs(z2[planes]).reshape(planes.sum(), -1).sum(-1) > 0)
    assert planes.sum() == 2 * R + 1
    z3 = O.axis_dft(n, z2, axis=0, sign=+1)[0]
    assert _rel(z3, O.to_real(n, g, c)[0]) < 1e-14


# ---------------------------------------------------------------- gradients
def test_gradients_by_finite_differences():
    n, R = (12, 12, 12), 3
    g = synth.sphere_glist(*n, R, order="shuffled", seed=25)
    c = synth.coefficients(g, 2, seed=26)
    V, _ = synth.potential(*n, "smooth", seed=27)
    rng = np.random.default_rng(28)
    t = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
    w = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)

    def loss(cc, VV):
        out = O.apply(n, g, cc, VV)
        return float(np.real(np.vdot(w, out)) + np.sum(np.abs(out - t) ** 2))

    out = O.apply(n, g, c, V)
    gout = w + 2.0 * (out - t)  # dL/dRe(out) + i dL/dIm(out)
    dc, dV = O.grads(n, g, c, V, gout)
    eps = 1e-6
    d = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
    fd = (loss(c + eps * d, V) - loss(c - eps * d, V)) / (2 * eps)
    an = float(np.real(np.vdot(dc, d)))
    assert abs(fd - an) < 1e-7 * abs(an)
    dVdir = rng.standard_normal(n)
    fd = (loss(c, V + eps * dVdir) - loss(c, V - eps * dVdir)) / (2 * eps)
    an = float(np.sum(dV * dVdir))
    assert abs(fd - an) < 1e-7 * abs(an)


# ---------------------------------------------------------------- partitions
def test_greedy_partition_rules():
    # Sec. 3.2 / Fig. 2: sorted round robin.
    n, R = (96, 96, 96), 24
    g = synth.sphere_glist(*n, R)
    ids, w = O.sticks(n, g)
    for P in [1, 7, 57, 148, 152, 304, 1793, 2000]:
        part = O.greedy_partition(ids, w, P)
        assert part.min() >= 0 and part.max() < P
        loads = O.part_loads(part, w, P)
        counts = np.bincount(part, minlength=P)
        assert loads.sum() == len(g)
        assert np.all(np.diff(loads) <= 0)              # non-increasing in part index
        assert loads.max() - loads.min() <= w.max()    # within one stick weight
        assert counts.max() - counts.min() <= 1        # sticks dealt evenly
    part = O.greedy_partition(ids, w, 148)
    loads = O.part_loads(part, w, 148)
    assert (w.max(), loads.min(), loads.max()) == (49, 366, 415)


def test_greedy_partition_tiebreak_small():
    # Hand example: weights 3,5,5,1,3 on ids 10..14 -> sorted (5@11, 5@12, 3@10, 3@14, 1@13)
    ids = np.array([10, 11, 12, 13, 14])
    w = np.array([3, 5, 5, 1, 3])
    assert O.greedy_partition(ids, w, 2).tolist() == [0, 0, 1, 0, 1]


def test_process_grid():
    assert O.process_grid(6) == (3, 2)   # Fig. 3's 3 x 2 example
    assert O.process_grid(16) == (4, 4)
    assert O.process_grid(24) == (6, 4)
    assert O.process_grid(7) == (7, 1)


@pytest.mark.parametrize("fn", [O.basic_partition, O.improved_partition])
def test_row_column_group_rules(fn):
    # Sec. 4.1: sticks sharing one first-pass coordinate share a row group,
    # sticks sharing the other share a column group.
    n, R, p = (32, 32, 32), 8, 6
    g = synth.sphere_glist(*n, R)
    ids, w = O.sticks(n, g)
    m, ncol = O.process_grid(p)
    rank = fn(n, g, p)
    a, b = ids // n[1], ids % n[1]
    for val in np.unique(a):
        assert len(np.unique(rank[a == val] // ncol)) == 1
    for val in np.unique(b):
        assert len(np.unique(rank[b == val] % ncol)) == 1


def test_greedy_balances_best():
    # Tab. 2's ordering, where each part holds many sticks: the greedy
    # max/min #PW ratio is the closest to 1 of the three partitions.
    for n, R in [((64, 64, 64), 16), ((96, 96, 96), 24)]:
        g = synth.sphere_glist(*n, R)
        ids, w = O.sticks(n, g)
        for p in [4, 6, 8, 12, 16, 24, 32, 48, 64]:
            if len(ids) / p < 8:
                continue
            r = {}
            for name, part in [("greedy", O.greedy_partition(ids, w, p)),
                               ("basic", O.basic_partition(n, g, p)),
                               ("improved", O.improved_partition(n, g, p))]:
                L = O.part_loads(part, w, p)
                r[name] = L.max() / L.min()
            assert r["greedy"] <= r["basic"] and r["greedy"] <= r["improved"]


# ---- Gamma-point real mode (Sec. 4.3, last paragraph)
def _gamma_case(n, R, nb, seed, order="canonical"):
    g = synth.sphere_glist(*n, R, order=order, seed=seed)
    gh = synth.half_sphere(g)
    c = synth.coefficients(gh, nb, seed=seed)
    V, _ = synth.potential(*n, kind="smooth", seed=seed + 1)
    return gh, c, V


def test_half_sphere_splits_pairs():
    g = synth.sphere_glist(8, 8, 8, 2.5)
    gh = synth.half_sphere(g)
    full = {tuple(x) for x in g}
    half = {tuple(x) for x in gh}
    assert (0, 0, 0) in half
    for G in full - {(0, 0, 0)}:
        mG = tuple(-x for x in G)
        assert (G in half) != (mG in half)
    assert 2 * len(gh) - 1 == len(g)


@pytest.mark.parametrize("n,R", TINY)
def test_gamma_completion_gives_real_bands(n, R):
    gh, c, _ = _gamma_case(n, R, 3, seed=5, order="shuffled")
    gf, cf = O.gamma_complete(gh, c)
    psi = O.np_to_real(n, gf, cf)
    assert np.abs(psi.imag).max() < 1e-13 * np.abs(psi.real).max()
    # an incomplete (half-only) band is not real
    psi_h = O.np_to_real(n, gh, c)
    assert np.abs(psi_h.imag).max() > 1e-3 * np.abs(psi_h.real).max()


@pytest.mark.parametrize("n,R", TINY)
def test_gamma_apply_matches_real_bruteforce(n, R):
    gh, c, V = _gamma_case(n, R, 3, seed=9, order="shuffled")
    got = O.gamma_apply(n, gh, c, V)
    want = O.bf_real_apply(n, gh, c, V)
    assert _rel(got, want) < 1e-12
    # the G = 0 result of a real band is real
    z = np.flatnonzero(~np.any(gh != 0, axis=1))
    assert np.abs(got[:, z].imag).max() < 1e-14


def test_gamma_result_is_hermitian():
    n, R = (8, 8, 8), 2.5
    gh, c, V = _gamma_case(n, R, 2, seed=3)
    gf, cf = O.gamma_complete(gh, c)
    out = O.apply(n, gf, cf, V)
    nh = len(gh)
    nz = np.any(gh != 0, axis=1)
    assert np.allclose(out[:, nh:], np.conj(out[:, :nh][:, nz]), rtol=0, atol=1e-14)


# ---- the r -> G half on its own and the charge density (Sec. 2, Sec. 3.1)
@pytest.mark.parametrize("n,R", TINY)
def test_to_recip_bruteforce_and_round_trip(n, R):
    g = synth.sphere_glist(*n, R, order="shuffled", seed=2)
    rng = np.random.default_rng(4)
    u = rng.standard_normal((2, *n)) + 1j * rng.standard_normal((2, *n))
    assert _rel(O.to_recip(n, g, u), O.bf_to_recip(n, g, u)) < 1e-12
    # F- F+ = N I on the grid, so the r -> G half undoes the G -> r half
    c = synth.coefficients(g, 3, seed=6)
    assert _rel(O.to_recip(n, g, O.to_real(n, g, c)), c) < 1e-13


def test_to_recip_library_cross_check():
    n = (12, 10, 9)
    g = synth.sphere_glist(*n, 3.3)
    u = np.random.default_rng(1).standard_normal((2, *n)) + 0j
    lib = np.fft.fftn(u, axes=(1, 2, 3)).reshape(2, -1)[:, O.np_index_map(n, g)] / np.prod(n)
    assert _rel(O.to_recip(n, g, u), lib) < 1e-13


@pytest.mark.parametrize("n,R", TINY)
def test_density_bruteforce_and_parseval(n, R):
    g = synth.sphere_glist(*n, R, order="shuffled", seed=3)
    c = synth.coefficients(g, 4, seed=8)
    f = np.array([2.0, 1.5, 0.25, 0.0])
    rho = O.density(n, g, c, f)
    psi = O.bf_to_real(n, g, c).reshape(4, -1)
    assert _rel(rho.ravel(), (f[:, None] * np.abs(psi) ** 2).sum(0)) < 1e-12
    assert rho.min() >= 0.0
    # Parseval for the unnormalised G -> r transform
    N = np.prod(n)
    assert abs(rho.sum() - N * (f * (np.abs(c) ** 2).sum(1)).sum()) < 1e-12 * rho.sum()


def test_density_of_single_plane_wave_is_flat():
    n = (6, 5, 4)
    g = np.array([[1, -2, 1]], dtype=np.int32)
    rho = O.density(n, g, np.array([[0.6 - 0.8j]]), [3.0])
    assert np.allclose(rho, 3.0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("n,R", TINY)
def test_gamma_density_matches_real_bruteforce(n, R):
    gh, c, _ = _gamma_case(n, R, 3, seed=12, order="shuffled")
    f = np.array([1.0, 0.5, 2.0])
    want = (f[:, None] * O.bf_real_psi(n, gh, c) ** 2).sum(0)
    assert _rel(O.gamma_density(n, gh, c, f).ravel(), want) < 1e-12


# ---- the Hamiltonian H = |G|^2/2 + V_loc (Eq. 1 at the Gamma point)
def test_dense_h_free_electrons_and_hermiticity():
    n = (12, 12, 12)
    g = synth.sphere_glist(*n, 3.1, order="shuffled", seed=2)
    T = O.kinetic(g, (10.0, 11.0, 12.0))
    # constant V = v0: eigenvalues are |G|^2 / 2 + v0 exactly
    H0 = O.dense_h(n, g, np.full(n, 0.7), T)
    assert np.allclose(np.linalg.eigvalsh(H0), np.sort(T) + 0.7, rtol=0, atol=1e-12)
    V, _ = synth.potential(*n, "smooth", seed=4)
    H = O.dense_h(n, g, V, T)
    assert np.abs(H - H.conj().T).max() < 1e-14
    # H applied to a vector = kinetic diagonal + the oracle's action
    x = synth.coefficients(g, 1, seed=5)[0]
    assert np.allclose(H @ x, T * x + O.apply(n, g, x, V)[0], rtol=0, atol=1e-13)
    # first-order perturbation: for a weak potential the lowest level is v(0)
    eps = 1e-4
    e = O.lowest_eigs(n, g, 1.0 + eps * (V - V.mean()), T, 1)
    assert abs(e[0] - 1.0) < 1e-6


def test_kinetic_units():
    g = np.array([[1, 0, 0], [0, 2, 0], [1, 1, 1]])
    T = O.kinetic(g, (2 * np.pi, 2 * np.pi, 2 * np.pi))
    assert np.allclose(T, [0.5, 2.0, 1.5])
