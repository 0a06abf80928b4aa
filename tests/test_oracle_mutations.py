"""Planted mistakes in the C oracle must fail its pins (CPU only).

Each case rewrites one line of ``oracle/vloc_oracle.c`` in a temporary copy
(a dropped term, a wrong sign, a wrong index, a transposed operand, a lost
normalisation), builds it, and checks that at least one independent pin --
brute-force plane-wave sums (Eq. 2), the hand-worked 1x1x4 case, the
few-mode closed form or the finite-difference gradient -- rejects it.
"""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_07378_gb300 import synth

SRC = os.path.join(os.path.dirname(O.__file__), "vloc_oracle.c")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

MUTATIONS = {
    "forward_sign": ("dft_axis(w, n, 1, -1);", "dft_axis(w, n, 1, +1);"),
    "no_normalisation": ("o[2 * p] = w[2 * idx[p]] / (double)N;", "o[2 * p] = w[2 * idx[p]];"),
    "transposed_index": ("int64_t j = (pmod(h, n1) * n2 + pmod(k, n2)) * n3 + pmod(l, n3);",
                         "int64_t j = (pmod(k, n2) * n1 + pmod(h, n1)) * n3 + pmod(l, n3);"),
    "dropped_plane_wave": ("for (int64_t p = 0; p < npw; ++p) {\n        psi[2 * idx[p]]",
                           "for (int64_t p = 1; p < npw; ++p) {\n        psi[2 * idx[p]]"),
    "wrong_twiddle_index": ("int t = (int)(((int64_t)m * k) % len);", "int t = (int)(((int64_t)m + k) % len);"),
    "imag_part_of_V_product": ("w[2 * j + 1] *= V[j];", "w[2 * j + 1] *= 1.0;"),
    "conjugated_input": ("psi[2 * idx[p] + 1] = c[2 * p + 1];", "psi[2 * idx[p] + 1] = -c[2 * p + 1];"),
    "grad_dropped_term": ("(gr[2 * j] * psi[2 * j] + gr[2 * j + 1] * psi[2 * j + 1])",
                          "(gr[2 * j] * psi[2 * j])"),
}


def _build_mutant(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so), str(path), "-lm"])
    return ctypes.CDLL(str(so))


def _pins_fail(lib):
    """True when at least one pin rejects the oracle loaded from ``lib``."""
    saved = O._lib
    O._lib = None
    try:
        # reuse the wrapper's argtypes by loading through it, then swap the handle
        real = O._load()
        for fn in ("oracle_index_map", "oracle_to_real", "oracle_apply", "oracle_grad_V", "oracle_axis_dft"):
            getattr(lib, fn).argtypes = getattr(real, fn).argtypes
        O._lib = lib
        failures = 0
        # brute force, shuffled list on a non-square grid
        n = (4, 6, 5)
        g = synth.sphere_glist(*n, 2.2, order="shuffled", seed=1)
        c = synth.coefficients(g, 2, seed=5)
        V, modes = synth.potential(*n, "smooth", seed=7)
        try:
            failures += np.linalg.norm(O.apply(n, g, c, V) - O.bf_apply(n, g, c, V)) > 1e-10
        except O.OracleError:
            failures += 1
        # hand-worked case
        d = json.load(open(os.path.join(GOLDEN, "hand_1x1x4.json")))
        try:
            out = O.apply(tuple(d["grid"]), np.array(d["glist"], dtype=np.int32),
                          np.array(d["coeffs_re"]) + 1j * np.array(d["coeffs_im"]), np.array(d["V"]))
            failures += np.abs(out.ravel() - (np.array(d["out_re"]) + 1j * np.array(d["out_im"]))).max() > 1e-12
        except O.OracleError:
            failures += 1
        # FD gradient in V
        n = (6, 6, 6)
        g = synth.sphere_glist(*n, 2)
        c = synth.coefficients(g, 1, seed=2)
        V, _ = synth.potential(*n, "smooth", seed=3)
        gout = synth.coefficients(g, 1, seed=4)
        try:
            dV = O.grad_V(n, g, c, gout)
            dirn = np.random.default_rng(0).standard_normal(n)
            L = lambda VV: float(np.real(np.vdot(gout, O.np_apply(n, g, c, VV))))
            fd = (L(V + 1e-6 * dirn) - L(V - 1e-6 * dirn)) / 2e-6
            failures += abs(fd - float((dV * dirn).sum())) > 1e-6 * max(1.0, abs(fd))
        except O.OracleError:
            failures += 1
        return failures > 0
    finally:
        O._lib = saved


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert _pins_fail(_build_mutant(tmp_path, name)), f"mutation {name} survived every pin"


def test_unmutated_oracle_passes(tmp_path):
    src = open(SRC).read()
    path = tmp_path / "clean.c"
    path.write_text(src)
    so = tmp_path / "libclean.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so), str(path), "-lm"])
    assert not _pins_fail(ctypes.CDLL(str(so)))


# ---- planted mistakes in the Gamma-point completion (Python side of the oracle)
def _complete_no_conj(g_half, c_half):
    g_half = np.asarray(g_half, dtype=np.int64).reshape(-1, 3)
    c_half = np.asarray(c_half, dtype=np.complex128).reshape(-1, len(g_half))
    nz = np.any(g_half != 0, axis=1)
    return np.concatenate([g_half, -g_half[nz]]).astype(np.int32), np.concatenate([c_half, c_half[:, nz]], axis=1)


def _complete_g0_complex(g_half, c_half):
    g_half = np.asarray(g_half, dtype=np.int64).reshape(-1, 3)
    c_half = np.asarray(c_half, dtype=np.complex128).reshape(-1, len(g_half))
    nz = np.any(g_half != 0, axis=1)
    return (np.concatenate([g_half, -g_half[nz]]).astype(np.int32),
            np.concatenate([c_half, np.conj(c_half[:, nz])], axis=1))


def _complete_same_G(g_half, c_half):
    g_half = np.asarray(g_half, dtype=np.int64).reshape(-1, 3)
    c_half = np.asarray(c_half, dtype=np.complex128).reshape(-1, len(g_half))
    nz = np.any(g_half != 0, axis=1)
    mirrored = g_half[nz] * np.array([-1, -1, 1])          # l not negated
    return (np.concatenate([g_half, mirrored]).astype(np.int32),
            np.concatenate([c_half.real * (~nz) + c_half * nz, np.conj(c_half[:, nz])], axis=1))


@pytest.mark.parametrize("bad", [_complete_no_conj, _complete_g0_complex, _complete_same_G])
def test_planted_gamma_mistake_is_caught(monkeypatch, bad):
    n = (4, 6, 5)
    g = synth.sphere_glist(*n, 2.2, order="shuffled", seed=1)
    gh = synth.half_sphere(g)
    c = synth.coefficients(gh, 2, seed=5)
    V, _ = synth.potential(*n, "smooth", seed=7)
    want = O.bf_real_apply(n, gh, c, V)
    assert np.linalg.norm(O.gamma_apply(n, gh, c, V) - want) < 1e-12 * np.linalg.norm(want)
    monkeypatch.setattr(O, "gamma_complete", bad)
    try:
        got = O.gamma_apply(n, gh, c, V)
        caught = np.linalg.norm(got - want) > 1e-10 * np.linalg.norm(want)
    except O.OracleError:
        caught = True
    assert caught


# ---- planted mistakes in the r -> G transform and the density (Python side)
def _recip_no_norm(n, g, u, nthreads=0):
    return O.to_recip(n, g, u, nthreads) * (n[0] * n[1] * n[2])


def _recip_wrong_sign(n, g, u, nthreads=0):
    N = n[0] * n[1] * n[2]
    a = np.asarray(u, dtype=np.complex128).reshape(-1, *n)
    for axis in range(3):
        a = O.axis_dft(n, a, axis, +1, nthreads)
    return a.reshape(a.shape[0], N)[:, O.index_map(n, g)] / N


def _recip_gather_at_minus_G(n, g, u, nthreads=0):
    N = n[0] * n[1] * n[2]
    a = np.asarray(u, dtype=np.complex128).reshape(-1, *n)
    for axis in range(3):
        a = O.axis_dft(n, a, axis, -1, nthreads)
    h, k, l = (-np.asarray(g, dtype=np.int64)).T
    idx = ((h % n[0]) * n[1] + (k % n[1])) * n[2] + (l % n[2])
    return a.reshape(a.shape[0], N)[:, idx] / N


def _density_no_occ(n, g, c, occ=None, nthreads=0):
    return O.density(n, g, c, None, nthreads)


def _density_abs_not_squared(n, g, c, occ=None, nthreads=0):
    psi = O.to_real(n, g, c, nthreads)
    f = np.ones(psi.shape[0]) if occ is None else np.asarray(occ, dtype=np.float64)
    return np.tensordot(f, np.abs(psi), axes=1)


def _density_real_part_only(n, g, c, occ=None, nthreads=0):
    psi = O.to_real(n, g, c, nthreads)
    f = np.ones(psi.shape[0]) if occ is None else np.asarray(occ, dtype=np.float64)
    return np.tensordot(f, psi.real ** 2, axes=1)


def _half_pins_fail(to_recip, density):
    """True when a pin of the r -> G transform or of the density (point-by-point
    sums of Eqs. 2-3, the G -> r -> G round trip, Parseval) rejects them."""
    n = (4, 6, 5)
    g = synth.sphere_glist(*n, 2.2, order="shuffled", seed=1)
    c = synth.coefficients(g, 3, seed=5)
    rng = np.random.default_rng(9)
    u = rng.standard_normal((2, *n)) + 1j * rng.standard_normal((2, *n))
    fails = 0
    fails += np.linalg.norm(to_recip(n, g, u) - O.bf_to_recip(n, g, u)) > 1e-10 * np.linalg.norm(O.bf_to_recip(n, g, u))
    fails += np.linalg.norm(to_recip(n, g, O.bf_to_real(n, g, c)) - c) > 1e-10 * np.linalg.norm(c)
    occ = np.array([2.0, 1.0, 0.5])
    rho = density(n, g, c, occ)
    want = np.tensordot(occ, np.abs(O.bf_to_real(n, g, c)) ** 2, axes=1)
    fails += np.abs(rho - want).max() > 1e-10 * np.abs(want).max()
    N = n[0] * n[1] * n[2]
    fails += abs(rho.sum() - N * float((occ[:, None] * np.abs(c) ** 2).sum())) > 1e-10 * rho.sum()
    return fails > 0


def test_unmutated_half_transforms_pass():
    assert not _half_pins_fail(O.to_recip, O.density)


@pytest.mark.parametrize("bad", [_recip_no_norm, _recip_wrong_sign, _recip_gather_at_minus_G])
def test_planted_to_recip_mistake_is_caught(bad):
    assert _half_pins_fail(bad, O.density), bad.__name__


@pytest.mark.parametrize("bad", [_density_no_occ, _density_abs_not_squared, _density_real_part_only])
def test_planted_density_mistake_is_caught(bad):
    assert _half_pins_fail(O.to_recip, bad), bad.__name__
