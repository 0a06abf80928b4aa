"""C-ABI library: loads, exports every declared symbol, and its host-side
plan logic (validation, index map, stick partition) is bit-exact against the
oracle's independent Python restatement.  No GPU and no compute calls."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_07378_gb300 import synth, vloc
from paper_1601_07378_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return vloc.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "vloc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vloc_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(vloc.EXPORTS) == names


def test_strerror_and_version(lib):
    assert lib.vloc_version() >= 100
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -99):
        assert isinstance(vloc.strerror(code), str) and vloc.strerror(code)


def _create(lib, n, g, flags=vloc.VLOC_F32 | vloc.VLOC_HOST_ONLY):
    h = ctypes.c_void_p()
    g = np.ascontiguousarray(np.asarray(g, dtype=np.int32).reshape(-1, 3))
    rc = lib.vloc_plan_create(ctypes.byref(h), n[0], n[1], n[2], g.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              len(g), flags, 0, None)
    return rc, h


@pytest.mark.parametrize("n,code", [((1, 8, 8), vloc.VLOC_ERR_SIZE), ((7, 8, 8), vloc.VLOC_ERR_SIZE),
                                    ((8, 257, 8), vloc.VLOC_ERR_SIZE), ((8, 8, 14), vloc.VLOC_ERR_SIZE),
                                    ((8, 8, 512), vloc.VLOC_ERR_SIZE)])
def test_rejects_bad_grids(lib, n, code):
    rc, _ = _create(lib, n, [[0, 0, 0]])
    assert rc == code


@pytest.mark.parametrize("g", [[[0, 0, 0], [0, 0, 0]], [[4, 0, 0]], [[0, -5, 0]], [[0, 0, 3]]])
def test_rejects_bad_glists(lib, g):
    rc, _ = _create(lib, (8, 9, 6), g)  # h in [-4, 3], k in [-4, 4], l in [-3, 2]
    assert rc == vloc.VLOC_ERR_GLIST


def test_rejects_bad_arguments(lib):
    g = np.zeros((1, 3), dtype=np.int32)
    gp = g.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    h = ctypes.c_void_p()
    assert lib.vloc_plan_create(None, 8, 8, 8, gp, 1, vloc.VLOC_F32, 0, None) == vloc.VLOC_ERR_ARG
    assert lib.vloc_plan_create(ctypes.byref(h), 8, 8, 8, None, 1, vloc.VLOC_F32, 0, None) == vloc.VLOC_ERR_ARG
    assert lib.vloc_plan_create(ctypes.byref(h), 8, 8, 8, gp, 0, vloc.VLOC_F32, 0, None) == vloc.VLOC_ERR_GLIST
    assert lib.vloc_plan_create(ctypes.byref(h), 8, 8, 8, gp, 1, 0, 0, None) == vloc.VLOC_ERR_ARG
    assert lib.vloc_plan_create(ctypes.byref(h), 8, 8, 8, gp, 1, vloc.VLOC_F32 | vloc.VLOC_F64, 0, None) == vloc.VLOC_ERR_ARG
    assert lib.vloc_plan_create(ctypes.byref(h), 8, 8, 8, gp, 1, vloc.VLOC_F32 | 0x8000, 0, None) == vloc.VLOC_ERR_ARG


def test_host_only_plan_refuses_device_calls(lib):
    rc, h = _create(lib, (8, 8, 8), synth.sphere_glist(8, 8, 8, 2))
    assert rc == 0
    assert lib.vloc_apply(h, ctypes.c_void_p(16), ctypes.c_void_p(16), 1, ctypes.c_void_p(16), None) == vloc.VLOC_ERR_STATE
    assert lib.vloc_backward(h, None, None, None, 1, ctypes.c_void_p(16), None, None) == vloc.VLOC_ERR_STATE
    assert lib.vloc_plan_destroy(h) == 0


def test_host_buffer_entry_checks_sizes_before_the_call(lib):
    # the binding rejects host buffers that the copies would overrun; valid
    # buffers reach the C side, which refuses a host-only plan
    torch = pytest.importorskip("torch")
    n = (8, 8, 8)
    g = synth.sphere_glist(*n, 2)
    plan = vloc.VlocPlan(n, g, torch.complex64, host_only=True)
    c = torch.zeros(3, len(g), dtype=torch.complex64)
    V = torch.zeros(n, dtype=torch.float32)
    with pytest.raises(ValueError):
        plan.apply_host(c, V, torch.zeros(2, len(g), dtype=torch.complex64))       # one band short
    with pytest.raises(ValueError):
        plan.apply_host(c, V, torch.zeros(3, len(g), dtype=torch.complex128))      # wrong precision
    with pytest.raises(ValueError):
        plan.apply_host(c, torch.zeros(8 * 8 * 7, dtype=torch.float32))            # V too small
    import types
    with pytest.raises(vloc.VlocError) as ei:       # a null stream: no CUDA context is needed here
        plan.apply_host(c, V, torch.zeros_like(c), stream=types.SimpleNamespace(cuda_stream=0))
    assert ei.value.code == vloc.VLOC_ERR_STATE


@pytest.mark.parametrize("n,R,order", [((24, 24, 24), 6, "canonical"), ((64, 64, 64), 16, "shuffled"),
                                       ((96, 96, 120), 24, "canonical"), ((6, 5, 4), 2.0, "shuffled"),
                                       ((96, 96, 96), 24, "shuffled")])
def test_index_map_and_partition_bit_exact(lib, n, R, order):
    import torch  # noqa: F401  (VlocPlan imports torch lazily)
    g = synth.sphere_glist(*n, R, order=order, seed=7)
    plan = vloc.VlocPlan(n, g, host_only=True)
    assert np.array_equal(plan.index_map(), O.index_map(n, g))
    ids, w = O.sticks(n, g)
    info = plan.info()
    assert info["nsticks"] == len(ids)
    assert info["nplanes"] == len(np.unique(ids // n[1]))
    part, P = plan.partition()
    assert P == (len(ids) + 31) // 32
    assert np.array_equal(part, O.greedy_partition(ids, w, P))
    for kind, fn in (("basic", O.basic_partition), ("improved", O.improved_partition)):
        p2 = vloc.VlocPlan(n, g, partition=kind, host_only=True)
        part2, P2 = p2.partition()
        assert P2 == P
        assert np.array_equal(part2, fn(n, g, P))


def test_radix_schedules(lib):
    import torch  # noqa: F401
    for n, rad in [(24, [6, 4]), (64, [8, 8]), (96, [12, 8]), (120, [12, 10]), (144, [12, 12]),
                   (125, [5, 5, 5]), (16, [16]), (2, [2]), (256, [16, 16]), (243, [9, 9, 3])]:
        plan = vloc.VlocPlan((n, 8, 8), [[0, 0, 0]], host_only=True)
        assert plan.info()["radix"][0] == rad
        assert int(np.prod(rad)) == n


def test_gamma_host_plan_index_map_and_rejects():
    # Gamma-point real mode (Sec. 4.3): the plan reports the caller's half
    # list; a list holding both G and -G, or whose -G leaves the grid's
    # index range, is rejected
    import torch
    n = (16, 18, 20)
    g = synth.sphere_glist(*n, 4.5, order="shuffled", seed=3)
    gh = synth.half_sphere(g)
    p = vloc.VlocPlan(n, gh, torch.complex64, host_only=True, gamma=True)
    inf = p.info()
    assert inf["gamma"] and inf["npw"] == len(gh)
    assert np.array_equal(p.index_map(), O.index_map(n, gh))
    full = vloc.VlocPlan(n, g, torch.complex64, host_only=True)
    assert p.info()["nsticks"] == full.info()["nsticks"]
    with pytest.raises(vloc.VlocError) as e:
        vloc.VlocPlan(n, g, torch.complex64, host_only=True, gamma=True)
    assert e.value.code == -3
    with pytest.raises(vloc.VlocError) as e:
        vloc.VlocPlan(n, np.array([[-8, 0, 0]], dtype=np.int32), torch.complex64, host_only=True, gamma=True)
    assert e.value.code == -3


def test_noalloc_refuses_gamma_plans_before_any_device_call(lib):
    # A Gamma-point plan's caller arrays hold the half list, while its index
    # tables address the full G / -G list: the allocation-free apply must
    # refuse it before touching any pointer or making a CUDA call (this runs
    # without a GPU; the pointers are never dereferenced).
    import torch  # noqa: F401
    n = (16, 18, 20)
    gh = synth.half_sphere(synth.sphere_glist(*n, 4.5, seed=3))
    for dt in (torch.complex64, torch.complex128):
        p = vloc.VlocPlan(n, gh, dt, host_only=True, gamma=True)
        bogus = ctypes.c_void_p(256)
        for nb in (0, 1, 5):
            rc = lib.vloc_apply_noalloc(p.handle, bogus, bogus, nb, bogus, None)
            assert rc == vloc.VLOC_ERR_STATE, (dt, nb, rc)


def test_fault_injection_fails_plan_creation_cleanly(lib, monkeypatch):
    # VLOC_FAULT=alloc makes the first allocation of vloc_plan_create (the
    # host plan object) fail: the call returns VLOC_ERR_ALLOC and hands back
    # no plan.  A host-only plan makes no CUDA call, so this runs without a GPU.
    g = np.ascontiguousarray(synth.sphere_glist(8, 8, 8, 2), dtype=np.int32)
    monkeypatch.setenv("VLOC_FAULT", "alloc")
    rc, h = _create(lib, (8, 8, 8), g)
    assert rc == vloc.VLOC_ERR_ALLOC and not h.value
    monkeypatch.setenv("VLOC_FAULT", "alloc:0")
    rc, h = _create(lib, (8, 8, 8), g)
    assert rc == vloc.VLOC_ERR_ALLOC and not h.value
    monkeypatch.delenv("VLOC_FAULT")
    rc, h = _create(lib, (8, 8, 8), g)
    assert rc == vloc.VLOC_OK and h.value
    assert lib.vloc_plan_destroy(h) == 0


def test_poison_flag_is_accepted_on_host_plans(lib):
    g = synth.sphere_glist(8, 8, 8, 2)
    rc, h = _create(lib, (8, 8, 8), g, flags=vloc.VLOC_F32 | vloc.VLOC_HOST_ONLY | vloc.VLOC_POISON_WORKSPACE)
    assert rc == 0
    assert lib.vloc_plan_destroy(h) == 0


def test_quarter_sphere_plane_set_is_detected(lib):
    # the x-pass kernels specialise for the plane set of a sphere of radius
    # n1/4 (x = 0..n1/4 and n1 - n1/4 .. n1 - 1, Sec. 4.3 / Fig. 5)
    import torch
    n = (48, 30, 30)
    g = synth.sphere_glist(*n, 12)
    assert vloc.VlocPlan(n, g, torch.complex64, host_only=True).info()["x_quarter"]
    assert vloc.VlocPlan(n, g[::-1], torch.complex64, host_only=True).info()["x_quarter"]
    strict = g[(g.astype(np.int64) ** 2).sum(axis=1) < 144]
    shifted = g + np.array([1, 0, 0], dtype=g.dtype)
    for other in (synth.sphere_glist(*n, 11.5), strict, shifted):
        assert not vloc.VlocPlan(n, other, torch.complex64, host_only=True).info()["x_quarter"]


def test_warp_z_pass_selection(lib):
    # VLOC_Z_WARP plans in FP32 with n3 = 32 C (C = 1..4) run the z-passes as
    # warp-register transforms (info bit 8); without the flag, for Gamma-point
    # and FP64 plans and for other lengths the tile z-passes run
    import torch
    for n3 in (32, 64, 96, 128):
        n = (20, 18, n3)
        g = synth.sphere_glist(*n, 7, order="shuffled", seed=3)
        assert vloc.VlocPlan(n, g, torch.complex64, host_only=True, z_warp=True).info()["z_warp"]
        assert not vloc.VlocPlan(n, g, torch.complex64, host_only=True).info()["z_warp"]
        assert not vloc.VlocPlan(n, g, torch.complex128, host_only=True, z_warp=True).info()["z_warp"]
        gh = synth.half_sphere(synth.sphere_glist(*n, 7))
        assert not vloc.VlocPlan(n, gh, torch.complex64, host_only=True, gamma=True, z_warp=True).info()["z_warp"]
    for n3 in (24, 48, 100, 120, 144):
        n = (20, 18, n3)
        g = synth.sphere_glist(*n, 7)
        assert not vloc.VlocPlan(n, g, torch.complex64, host_only=True, z_warp=True).info()["z_warp"]


def test_bulk_staged_z_pass_selection(lib):
    # VLOC_Z_BULK: the inverse z-pass stages each stick's coefficients by one
    # bulk copy (info bit 9) when every |l| <= n3/4 and each stick's plane
    # waves are consecutive in the caller's list with l ascending (the
    # canonical order); otherwise, and without the flag, the direct loads run
    import torch
    n = (48, 40, 96)
    g = synth.sphere_glist(*n, 24)
    plan = lambda gl, dt=torch.complex64, **kw: vloc.VlocPlan(n, gl, dt, host_only=True, **kw).info()["z_bulk"]
    assert plan(g, z_bulk=True)
    assert not plan(g)
    assert not plan(g, torch.complex128, z_bulk=True)
    assert not plan(synth.sphere_glist(*n, 24, order="shuffled", seed=2), z_bulk=True)
    # l descending within a stick, or a gap in l, breaks the runs
    desc = g[np.lexsort((-g[:, 2], g[:, 1] % n[1], g[:, 0] % n[0]))]
    assert not plan(desc, z_bulk=True)
    gap = g[~((g[:, 0] == 0) & (g[:, 1] == 0) & (g[:, 2] == 3))]
    assert not plan(gap, z_bulk=True)
    # beyond the quarter band the tile scatter runs
    assert not plan(synth.sphere_glist(*n, 25), z_bulk=True)


@pytest.mark.parametrize("n,R", [((16, 18, 20), 4.5), ((96, 96, 96), 24), ((30, 45, 27), 7)])
def test_gamma_partition_deals_mirror_pairs(lib, n, R):
    # Gamma-point plans deal a stick (h, k) and its mirror (-h, -k) to the
    # same part: the greedy rule (Sec. 3.2) applied to pairs, weight
    # descending, ties by the smaller stick id, the k-th pair to part k mod P
    import torch
    g = synth.sphere_glist(*n, R, order="shuffled", seed=5)
    gh = synth.half_sphere(g)
    plan = vloc.VlocPlan(n, gh, torch.complex64, host_only=True, gamma=True)
    part, P = plan.partition()
    ids, w = O.sticks(n, g)            # the full G / -G list's sticks, ascending id
    assert len(part) == len(ids)
    sid = {int(s): i for i, s in enumerate(ids)}
    mirror = np.array([sid[((n[0] - s // n[1]) % n[0]) * n[1] + (n[1] - s % n[1]) % n[1]] for s in ids])
    assert np.array_equal(part, part[mirror])
    assert np.bincount(part, minlength=P).max() <= 32
    # restatement of the rule
    order = sorted(range(len(ids)), key=lambda i: (-int(w[i]), int(ids[i])))
    pairs = [i for i in order if i <= mirror[i]]
    P2 = max((len(ids) + 31) // 32, (len(pairs) + 15) // 16)
    assert P == P2
    want = np.empty(len(ids), dtype=np.int32)
    for r, i in enumerate(pairs):
        want[i] = want[mirror[i]] = r % P2
    assert np.array_equal(part, want)
