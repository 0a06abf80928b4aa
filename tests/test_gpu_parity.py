"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative L2 per band, max over bands): 2e-6 for the FP32 path
and 1e-12 for the FP64 path; the FP32 comparison feeds the oracle the same
FP32-rounded inputs, upcast.  Integer work (index map, partition) is checked
bit-exactly in test_abi_host.py.
"""
import numpy as np
import pytest

from helpers import TOL, make_case, oracle_apply, rel_l2_per_band
from oracle import oracle as O
from paper_1601_07378_gb300 import synth, vloc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f32": (torch.complex64, torch.float32), "f64": (torch.complex128, torch.float64)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1601_07378_gb300.build import build
    build()


def run(n, g, c, V, prec, **kw):
    cd, rd = DT[prec]
    plan = vloc.VlocPlan(n, g, cd, **kw)
    ct = torch.from_numpy(np.ascontiguousarray(c)).to("cuda", cd)
    Vt = torch.from_numpy(np.ascontiguousarray(V)).to("cuda", rd)
    out = plan.apply(ct, Vt)
    torch.cuda.synchronize()
    return plan, ct, Vt, out


@pytest.mark.parametrize("generic", [False, True])
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,R,nb,order", [
    ((24, 24, 24), 6, 1, "canonical"),        # config 0 (ragged: 24 < one 32-line tile)
    ((24, 24, 24), 6, 5, "shuffled"),
    ((4, 6, 5), 2.2, 3, "shuffled"),          # tiny, odd radices
    ((6, 5, 4), 2.0, 2, "canonical"),
    ((8, 8, 8), 2.5, 2, "shuffled"),
    ((20, 18, 25), 4, 3, "shuffled"),
    ((40, 36, 50), 8, 3, "canonical"),        # several z tiles with a ragged tail
    ((30, 45, 27), 7, 2, "shuffled"),         # radices 3, 5, 9, 15
    ((64, 64, 64), 16, 4, "canonical"),
    ((48, 48, 25), 6, 3, "shuffled"),         # compile-time x/y lengths, odd z length
    ((64, 60, 45), 10, 2, "canonical"),
])
def test_apply_matches_oracle(prec, n, R, nb, order, generic):
    # generic=True forces the runtime-radix kernels on every axis; otherwise
    # the compile-time-length kernels run wherever one exists (24, 32, 48, 64)
    g, c, V = make_case(n, R, nb, seed=11, order=order, prec=prec)
    _, _, _, out = run(n, g, c, V, prec, generic=generic)
    err = rel_l2_per_band(out.cpu().numpy(), oracle_apply(n, g, c, V))
    assert err.max() < TOL[prec], err.max()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_config1_64cubed_256_bands_sampled(prec):
    n, R, nb = (64, 64, 64), 16, 256
    g, c, V = make_case(n, R, nb, seed=1, prec=prec)
    _, _, _, out = run(n, g, c, V, prec)
    bands = [0, 1, 77, 128, 200, 255]
    err = rel_l2_per_band(out.cpu().numpy()[bands], oracle_apply(n, g, c, V, bands))
    assert err.max() < TOL[prec], err.max()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,chunk", [((96, 96, 120), 0), ((96, 96, 96), 0), ((96, 96, 96), 430),
                                     ((128, 128, 128), 0), ((144, 144, 144), 0)])
def test_full_size_1024_bands_sampled(prec, n, chunk):
    # The bench's launch configuration (default plan, 1024 bands; and 430-band
    # chunks, three chunks per step), sampled bands from the first, middle and
    # last workspace chunks.
    R, nb = n[0] // 4, (1024 if n[0] == 96 else 64)
    g, c, V = make_case(n, R, nb, seed=2, prec=prec)
    plan, _, _, out = run(n, g, c, V, prec, chunk=chunk)
    chunk = plan.info()["chunk_bands"]
    bands = sorted({b for b in (0, chunk - 1, chunk, nb // 2, nb - 1) if b < nb})
    err = rel_l2_per_band(out.cpu().numpy()[bands], oracle_apply(n, g, c, V, bands))
    assert err.max() < TOL[prec], err.max()


def test_chunk_boundaries_and_alias():
    n, R, nb = (24, 20, 30), 5, 7
    g, c, V = make_case(n, R, nb, seed=3, order="shuffled", prec="f64")
    ref = oracle_apply(n, g, c, V)
    for chunk in (1, 2, 3, 7, 100):
        plan, ct, Vt, out = run(n, g, c, V, "f64", chunk=chunk)
        assert plan.info()["chunk_bands"] == chunk
        assert rel_l2_per_band(out.cpu().numpy(), ref).max() < TOL["f64"]
        # exact alias out == coeffs
        plan.apply(ct, Vt, out=ct)
        torch.cuda.synchronize()
        assert torch.equal(ct, out)


def test_empty_batch_and_bad_arguments():
    n = (16, 16, 16)
    g, c, V = make_case(n, 4, 4, seed=4, prec="f32")
    plan, ct, Vt, out = run(n, g, c, V, "f32")
    e = torch.empty((0, len(g)), dtype=torch.complex64, device="cuda")
    assert plan.apply(e, Vt).shape == (0, len(g))
    with pytest.raises(vloc.VlocError) as ei:   # partial overlap of input and output
        plan.apply(ct[:3], Vt, out=ct[1:])
    assert ei.value.code == vloc.VLOC_ERR_ARG
    lib = vloc.load()
    assert lib.vloc_apply(plan.handle, vloc._ptr(ct), vloc._ptr(Vt), -1, vloc._ptr(out), None) == vloc.VLOC_ERR_ARG
    assert lib.vloc_apply(plan.handle, None, vloc._ptr(Vt), 1, vloc._ptr(out), None) == vloc.VLOC_ERR_ARG
    mis = torch.empty(2 * len(g) + 1, dtype=torch.float32, device="cuda")
    assert lib.vloc_apply(plan.handle, mis.data_ptr() + 4, vloc._ptr(Vt), 1, vloc._ptr(out), None) == vloc.VLOC_ERR_ARG


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_non_sphere_lists(prec):
    # Any G-list is accepted: a random subset of the cube (sticks with gaps),
    # the strict-inequality sphere of Eq. 3, and every grid point.
    rng = np.random.default_rng(5)
    n = (8, 6, 10)
    cube = np.array(np.meshgrid(np.arange(-4, 4), np.arange(-3, 3), np.arange(-5, 5), indexing="ij")).reshape(3, -1).T
    for g in (cube[rng.random(len(cube)) < 0.3], cube[rng.permutation(len(cube))],
              synth.sphere_glist(*n, 3, strict=True)):
        g = np.ascontiguousarray(g.astype(np.int32))
        c = synth.coefficients(g, 2, seed=6)
        V, _ = synth.potential(*n, "smooth", seed=7)
        if prec == "f32":
            c, V = c.astype(np.complex64), V.astype(np.float32)
        _, _, _, out = run(n, g, c, V, prec)
        err = rel_l2_per_band(out.cpu().numpy(), oracle_apply(n, g, c, V))
        assert err.max() < TOL[prec], err.max()


@pytest.mark.parametrize("generic", [False, True])
def test_partitions_do_not_change_results(generic):
    n, R = (32, 32, 32), 8
    g, c, V = make_case(n, R, 3, seed=8, prec="f32")
    outs = [run(n, g, c, V, "f32", partition=k, generic=generic)[3] for k in ("greedy", "basic", "improved")]
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_every_fast_length_matches_oracle():
    # each compile-time length on every axis, against the oracle and against
    # the runtime-radix kernels
    for m in (24, 32, 48, 60, 64, 72, 80, 96, 100, 120, 128, 144):
        n = (m, 24 if m != 24 else 32, 48 if m != 48 else 60)
        for nn in (n, n[::-1], (n[1], m, n[2])):
            R = min(nn) / 4
            g, c, V = make_case(nn, R, 2, seed=m, order="shuffled", prec="f32")
            _, _, _, fast = run(nn, g, c, V, "f32")
            _, _, _, gen = run(nn, g, c, V, "f32", generic=True)
            ref = oracle_apply(nn, g, c, V)
            assert rel_l2_per_band(fast.cpu().numpy(), ref).max() < TOL["f32"], (nn, "fast")
            assert rel_l2_per_band(gen.cpu().numpy(), ref).max() < TOL["f32"], (nn, "generic")


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_adjoint_and_hermiticity(prec):
    n, R = (24, 30, 20), 6
    g, c, V = make_case(n, R, 2, seed=9, order="shuffled", prec=prec)
    plan, ct, Vt, out = run(n, g, c, V, prec)
    adj = plan.apply(ct, Vt, adjoint=True)
    torch.cuda.synchronize()
    assert torch.equal(adj, out)
    a = out.cpu().numpy().astype(np.complex128)
    x = c.astype(np.complex128)
    lhs = np.vdot(x[0], a[1])
    rhs = np.vdot(a[0], x[1])
    assert abs(lhs - rhs) < (1e-5 if prec == "f32" else 1e-13) * abs(lhs)


def test_deterministic():
    n, R = (48, 48, 48), 12
    g, c, V = make_case(n, R, 6, seed=10, prec="f32")
    plan, ct, Vt, out = run(n, g, c, V, "f32")
    again = plan.apply(ct, Vt)
    torch.cuda.synchronize()
    assert torch.equal(out, again)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_host_buffer_entry_matches_device_entry(prec):
    n, R, nb = (32, 36, 40), 8, 13
    g, c, V = make_case(n, R, nb, seed=12, prec=prec)
    plan, ct, Vt, out = run(n, g, c, V, prec, chunk=4)
    ch = ct.cpu().pin_memory()
    Vh = Vt.cpu().pin_memory()
    oh = plan.apply_host(ch, Vh)
    assert torch.equal(oh, out.cpu())


@pytest.mark.parametrize("n,R,nb,chunk", [((32, 36, 40), 8, 13, 4), ((96, 96, 96), 24, 600, 0)])
def test_async_host_buffer_calls_overlap_and_match(n, R, nb, chunk):
    # consecutive asynchronous host-buffer calls on one plan (the staging
    # slots' state carries from call to call): three calls into three
    # outputs, one synchronisation, each equal to the device entry's result
    g, c, V = make_case(n, R, nb, seed=13, prec="f32")
    plan, ct, Vt, out = run(n, g, c, V, "f32", chunk=chunk)
    Vh = Vt.cpu().pin_memory()
    chs = [(ct * s).cpu().pin_memory() for s in (1.0, 2.0, 0.5)]
    ohs = [torch.empty_like(h).pin_memory() for h in chs]
    for h, o in zip(chs, ohs):
        plan.apply_host(h, Vh, o, blocking=False)
    torch.cuda.current_stream().synchronize()
    for s, o in zip((1.0, 2.0, 0.5), ohs):
        want = plan.apply(ct * s, Vt).cpu()
        assert torch.equal(o, want)
    # a blocking call after asynchronous ones
    assert torch.equal(plan.apply_host(chs[0], Vh), out.cpu())


def test_batched_matches_individual():
    cases = []
    for i, m in enumerate([16, 24, 30]):
        n = (m, m, m)
        g, c, V = make_case(n, m / 4, 3 + i, seed=20 + i, prec="f32")
        cases.append(run(n, g, c, V, "f32"))
    outs = vloc.apply_batched([p for p, *_ in cases], [c for _, c, _, _ in cases], [V for _, _, V, _ in cases])
    torch.cuda.synchronize()
    for o, (_, _, _, ref) in zip(outs, cases):
        assert torch.equal(o, ref)


def test_uneven_batch_full_size_sampled():
    # The uneven multi-instance workload at full size, as the bench launches
    # it: 8 cubic grids 48..144, R = n/4, 64 (i + 1) bands each, FP32, one
    # graph-captured batched launch (captured, then replayed); the first and
    # last band of every instance against the oracle.
    cases = []
    for i, m in enumerate(synth.BATCH_GRIDS):
        n = (m, m, m)
        g, c, V = make_case(n, m / 4, 64 * (i + 1), seed=3 + i, prec="f32")
        plan = vloc.VlocPlan(n, g, torch.complex64, graph=True, chunk=64 * (i + 1))
        cases.append((n, g, c, V, plan, torch.from_numpy(c).cuda(), torch.from_numpy(V).cuda()))
    outs = [torch.empty_like(ct) for *_, ct, _ in cases]
    for _ in range(2):
        for o in outs:
            o.zero_()
        vloc.apply_batched([p for *_, p, _, _ in cases], [ct for *_, ct, _ in cases], [Vt for *_, Vt in cases], outs)
        torch.cuda.synchronize()
    for (n, g, c, V, *_), o in zip(cases, outs):
        bands = [0, c.shape[0] - 1]
        err = rel_l2_per_band(o.cpu().numpy()[bands], oracle_apply(n, g, c, V, bands))
        assert err.max() < TOL["f32"], (n, err.max())


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,R", [((32, 32, 32), 8), ((48, 48, 25), 6)])
def test_backward_matches_oracle(prec, n, R):
    # (48, 48, 25): compile-time x/y lengths with an odd z length
    nb = 3
    g, c, V = make_case(n, R, nb, seed=4, prec=prec)
    rng = np.random.default_rng(13)
    gout = (rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).astype(c.dtype)
    plan, ct, Vt, _ = run(n, g, c, V, prec)
    gt = torch.from_numpy(gout).to("cuda")
    gc, gV = plan.backward(ct, gt, Vt)
    torch.cuda.synchronize()
    dc_ref, dV_ref = O.grads(n, g, c.astype(np.complex128), V.astype(np.float64), gout.astype(np.complex128))
    assert rel_l2_per_band(gc.cpu().numpy(), dc_ref).max() < TOL[prec]
    dV = gV.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(dV - dV_ref) / np.linalg.norm(dV_ref) < TOL[prec]


_FULL_GRAD_CACHE = {}


def _full_size_grad_case(prec):
    # 96^3, R = 24 (57777 PWs), 48 bands: three 16-band groups of the dL/dV
    # x-pass.  The oracle's dL/dV over all bands and its dL/dc on sampled
    # bands are computed once per precision (same rounded inputs for every
    # chunk setting).
    if prec not in _FULL_GRAD_CACHE:
        n, R, nb = (96, 96, 96), 24, 48
        g, c, V = make_case(n, R, nb, seed=44, prec=prec)
        rng = np.random.default_rng(45)
        gout = (rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).astype(c.dtype) * 0.01
        sample = [0, 15, 16, 31, 47]
        dc_ref = oracle_apply(n, g, gout, V, bands=sample)
        dV_ref = O.grad_V(n, g, c.astype(np.complex128), gout.astype(np.complex128))
        _FULL_GRAD_CACHE[prec] = (n, g, c, V, gout, sample, dc_ref, dV_ref)
    return _FULL_GRAD_CACHE[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("chunk", [0, 40])
def test_backward_full_size_matches_oracle(prec, chunk):
    # The differentiable workload's grid (96^3, R = 24) with 48 bands.  The
    # default chunk keeps all bands in one workspace chunk, so dL/dV merges
    # three 16-band group sums in FP64; chunk = 40 splits the backward into
    # chunks of 20, 20 and 8 bands (ragged), each with one full and one
    # partial group.  dL/dc is compared per band on sampled bands, dL/dV over
    # the whole grid.
    n, g, c, V, gout, sample, dc_ref, dV_ref = _full_size_grad_case(prec)
    cd, rd = DT[prec]
    plan = vloc.VlocPlan(n, g, cd, chunk=chunk)
    if chunk:
        assert plan.info()["chunk_bands"] == chunk
    ct = torch.from_numpy(c).to("cuda", cd)
    Vt = torch.from_numpy(V).to("cuda", rd)
    gt = torch.from_numpy(gout).to("cuda", cd)
    gc, gV = plan.backward(ct, gt, Vt)
    torch.cuda.synchronize()
    assert rel_l2_per_band(gc.cpu().numpy()[sample], dc_ref).max() < TOL[prec]
    dV = gV.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(dV - dV_ref) / np.linalg.norm(dV_ref) < TOL[prec]


def test_autograd_finite_differences_fp64():
    # loss = sum_n <psi_n|V|psi_n> + ||V psi - t||^2 at 32^3 (R = 8), FP64.
    n, R, nb = (32, 32, 32), 8, 2
    g, c, V = make_case(n, R, nb, seed=14, prec="f64")
    plan = vloc.VlocPlan(n, g, torch.complex128)
    rng = np.random.default_rng(15)
    t = torch.from_numpy(rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).cuda() * 0.01
    ct = torch.from_numpy(c).cuda().requires_grad_(True)
    Vt = torch.from_numpy(V).cuda().requires_grad_(True)

    def loss(cc, VV):
        out = vloc.vloc_apply(cc, VV, plan)
        return (torch.conj(cc) * out).real.sum() + ((out - t).abs() ** 2).sum()

    L = loss(ct, Vt)
    L.backward()
    d = torch.from_numpy(rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).cuda()
    dv = torch.from_numpy(rng.standard_normal(V.shape)).cuda()
    eps = 1e-6
    with torch.no_grad():
        fd_c = (loss(ct + eps * d, Vt) - loss(ct - eps * d, Vt)) / (2 * eps)
        fd_v = (loss(ct, Vt + eps * dv) - loss(ct, Vt - eps * dv)) / (2 * eps)
    an_c = (torch.conj(ct.grad) * d).real.sum()
    an_v = (Vt.grad * dv).sum()
    assert abs(fd_c - an_c) < 1e-7 * abs(an_c)
    assert abs(fd_v - an_v) < 1e-7 * abs(an_v)


def test_graph_replay_matches_direct_launches():
    n, R, nb = (48, 48, 48), 12, 9
    g, c, V = make_case(n, R, nb, seed=50, prec="f32")
    plan, ct, Vt, ref = run(n, g, c, V, "f32")
    gplan = vloc.VlocPlan(n, g, torch.complex64, graph=True, chunk=4)
    out = torch.empty_like(ct)
    l0 = gplan.launch_count()
    for _ in range(3):                        # capture once, replay twice
        out.zero_()
        gplan.apply(ct, Vt, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    per_call = (gplan.launch_count() - l0) // 3
    assert per_call == 5 * 3                  # 3 chunks of the five-kernel chain
    c2 = ct.clone() * 2                       # new pointers -> a second graph
    out2 = gplan.apply(c2, Vt)
    torch.cuda.synchronize()
    assert torch.allclose(out2, 2 * ref, rtol=1e-5, atol=1e-6)


def test_graph_batched_matches_individual():
    cases = []
    for i, m in enumerate([16, 24, 30, 48]):
        n = (m, m, m)
        g, c, V = make_case(n, m / 4, 2 + i, seed=60 + i, prec="f32")
        p0, ct, Vt, ref = run(n, g, c, V, "f32")
        cases.append((vloc.VlocPlan(n, g, torch.complex64, graph=True), ct, Vt, ref))
    outs = [torch.empty_like(c) for _, c, _, _ in cases]
    for _ in range(3):                        # capture once, replay twice
        for o in outs:
            o.zero_()
        vloc.apply_batched([p for p, *_ in cases], [c for _, c, _, _ in cases], [V for _, _, V, _ in cases], outs)
        torch.cuda.synchronize()
        for o, (_, _, _, ref) in zip(outs, cases):
            assert torch.equal(o, ref)


@pytest.mark.parametrize("n,R,nb,chunk", [((96, 96, 96), 24, 300, 0), ((64, 64, 64), 16, 37, 5),
                                          ((48, 60, 72), 11, 9, 0), ((32, 48, 96), 8, 20, 7)])
def test_x_tma_option_is_bit_identical(n, R, nb, chunk, monkeypatch):
    # the persistent TMA x-pass (VLOC_X_TMA) runs the same arithmetic as the
    # general x-pass (k3_ct; the quarter-sphere forms are turned off in both
    # plans): forward and backward results equal bit for bit
    g, c, V = make_case(n, R, nb, seed=5, order="shuffled", prec="f32")
    monkeypatch.setenv("VLOC_NO_XQ", "1")   # the same general z-, y- and x-passes in both plans
    ref_plan, ct, Vt, ref = run(n, g, c, V, "f32", chunk=chunk)
    plan = vloc.VlocPlan(n, g, torch.complex64, chunk=chunk, x_tma=True)
    monkeypatch.delenv("VLOC_NO_XQ")
    assert plan.info()["x_tma"]
    out = plan.apply(ct, Vt)
    gt = torch.from_numpy(synth.coefficients(g, nb, seed=6, dtype=np.complex64)).cuda()
    gc0, gV0 = ref_plan.backward(ct, gt, Vt)
    gc1, gV1 = plan.backward(ct, gt, Vt)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    assert torch.equal(out, ref) and torch.equal(gc0, gc1) and torch.equal(gV0, gV1)


def test_x_tma_option_falls_back_for_odd_z():
    n = (48, 48, 25)
    g, c, V = make_case(n, 6, 2, seed=5, prec="f32")
    plan = vloc.VlocPlan(n, g, torch.complex64, x_tma=True)
    assert not plan.info()["x_tma"]
