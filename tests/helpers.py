"""Shared helpers for the GPU parity tests (inputs from synth, references from
the oracle, tolerances from the arithmetic)."""
import numpy as np

from oracle import oracle as O
from paper_1601_07378_gb300 import synth

# Relative L2 error per band, max over bands, against the FP64 oracle.
TOL = {"f32": 2e-6, "f64": 1e-12}


def rel_l2_per_band(x, ref):
    x = np.asarray(x).reshape(ref.shape[0], -1)
    ref = np.asarray(ref).reshape(ref.shape[0], -1)
    return np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)


def make_case(n, R, nb, seed, vkind="smooth", order="canonical", prec="f32"):
    """Seeded inputs; returns (g, c, V) with c/V already rounded to the
    precision under test (the oracle then sees exactly the same values)."""
    g = synth.sphere_glist(*n, R, order=order, seed=seed)
    c = synth.coefficients(g, nb, seed=seed)
    V, _ = synth.potential(*n, vkind, seed=seed + 1000)
    if prec == "f32":
        c = c.astype(np.complex64)
        V = V.astype(np.float32)
    return g, c, V


def oracle_apply(n, g, c, V, bands=None):
    cc = np.asarray(c, dtype=np.complex128)
    if bands is not None:
        cc = cc[bands]
    return O.apply(n, g, cc, np.asarray(V, dtype=np.float64))
