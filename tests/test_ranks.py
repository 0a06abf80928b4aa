"""Multi-rank layouts of Sec. 3-4 (CPU only): owner tables against the
oracle's partitions (bit-exact), message counts against the paper's
p (p - 1) / p (sqrt(p) - 1) (Eqs. 4-5), the load-balance ordering of Tab. 2,
and a distributed compact-FFT V_loc apply over gloo ranks (world sizes 4
and 6) whose transposes run through ``ranks.transpose`` and whose result
must equal the oracle's.

The per-layout 1-D transforms in the distributed test are numpy FFTs
written here (the module under test only moves data)."""
import math
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_1601_07378_gb300 import ranks, synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def test_proc_grid_matches_oracle():
    for p in range(1, 65):
        m, n = ranks.proc_grid(p)
        assert (m, n) == O.process_grid(p)
        assert m * n == p and m >= n


@pytest.mark.parametrize("alg", ranks.ALGORITHMS)
@pytest.mark.parametrize("n,R,p", [((24, 24, 24), 6, 4), ((40, 36, 50), 8, 6), ((96, 96, 96), 24, 16),
                                   ((96, 96, 96), 24, 12)])
def test_first_pass_owners_match_oracle(alg, n, R, p):
    g = synth.sphere_glist(*n, R, order="shuffled", seed=3)
    L = ranks.RankLayout(n, g, p, alg)
    ids, w = O.sticks(n, g)
    assert np.array_equal(L.sticks, ids) and np.array_equal(L.stick_pw, w)
    want = {"greedy": lambda: O.greedy_partition(ids, w, p),
            "basic": lambda: O.basic_partition(n, g, p),
            "improved": lambda: O.improved_partition(n, g, p)}[alg]()
    assert np.array_equal(L.recip_owner, want)


@pytest.mark.parametrize("alg", ranks.ALGORITHMS)
def test_layouts_cover_each_column_once(alg):
    n, p = (20, 18, 25), 6
    L = ranks.RankLayout(n, synth.sphere_glist(*n, 4.5), p, alg)
    st = np.concatenate([L.local_sticks(r) for r in range(p)])
    assert np.array_equal(np.sort(st), np.arange(len(L.sticks)))
    inter = np.concatenate([L.local_inter(r) for r in range(p)])
    assert len(inter) == len(L.planes) * n[2] and len(np.unique(inter[:, 0] * n[2] + inter[:, 1])) == len(inter)
    real = np.concatenate([L.local_real(r) for r in range(p)])
    assert len(np.unique(real[:, 0] * n[2] + real[:, 1])) == n[1] * n[2]
    assert sum(len(L.local_pw(r)[0]) for r in range(p)) == L.npw


@pytest.mark.parametrize("p", [4, 9, 16, 36, 64, 8, 12])
def test_message_counts(p):
    # Sec. 4.1: a global all-to-all makes p (p - 1) messages, the row / column
    # all-to-alls p (n - 1) and p (m - 1) (= p (sqrt(p) - 1) each when m = n);
    # the greedy layout's second transpose moves nothing (Sec. 5)
    n = (96, 96, 96)
    g = synth.sphere_glist(*n, 24)
    m, nc = ranks.proc_grid(p)
    G = ranks.RankLayout(n, g, p, "greedy")
    assert G.message_count(1) == p * (p - 1)
    assert G.message_count(2) == 0
    for alg in ("basic", "improved"):
        L = ranks.RankLayout(n, g, p, alg)
        assert L.message_count(1) == p * (nc - 1)
        assert L.message_count(2) == p * (m - 1)
        if m == nc:
            assert L.message_count(1) == L.message_count(2) == p * (math.isqrt(p) - 1)
        # messages stay inside the transpose's groups
        for which in (1, 2):
            M = L.message_matrix(which)
            same = np.zeros((p, p), dtype=bool)
            for gr in L.groups(which):
                same[np.ix_(gr, gr)] = True
            assert not np.any(M[~same])
        # larger messages: about mu N / (p sqrt p) against mu N / p^2
        if m == nc and p >= 16:
            M1, MG = L.message_matrix(1), G.message_matrix(1)
            off = ~np.eye(p, dtype=bool)
            ratio = M1[off][M1[off] > 0].mean() / MG[off][MG[off] > 0].mean()
            assert abs(ratio / math.sqrt(p) - 1) < 0.25, ratio


@pytest.mark.parametrize("p", [4, 8, 16, 32, 64])
def test_greedy_balances_plane_waves_best(p):
    # Tab. 2 compares the max / min plane waves per process: greedy is best
    n = (80, 80, 80)
    g = synth.sphere_glist(*n, 20.3)
    spread = {}
    for alg in ranks.ALGORITHMS:
        w = ranks.RankLayout(n, g, p, alg).pw_per_rank()
        assert w.sum() == len(g)
        spread[alg] = w.max() / w.min()
    assert spread["greedy"] <= min(spread["basic"], spread["improved"])
    assert spread["greedy"] < 1.1


def test_comm_cost_latency_ratio():
    for p in (4, 16, 64, 256):
        tg = ranks.comm_cost(p, 80 ** 3, alpha=1.0, beta=math.inf, kind="global")
        tl = ranks.comm_cost(p, 80 ** 3, alpha=1.0, beta=math.inf, kind="local")
        assert tg / tl == pytest.approx((p - 1) / (math.sqrt(p) - 1))


# ---------------------------------------------------------------- gloo ranks
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_apply(rank, world, port, alg, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = (12, 10, 9)
        n1, n2, n3 = n
        g = synth.sphere_glist(*n, 3.2, order="shuffled", seed=4)
        c = synth.coefficients(g, 2, seed=5)
        V, _ = synth.potential(*n, "smooth", seed=6)
        L = ranks.RankLayout(n, g, world, alg)
        groups = ranks.make_groups(L)
        sent = [0, 0]
        psis, outs = [], []
        for band in c:
            # G -> r: z-pass on sticks, transpose, y-pass, transpose, x-pass
            cyl = n3 * np.fft.ifft(L.scatter(rank, band), axis=1)
            inter, k = ranks.transpose(L, 1, rank, cyl, groups)
            sent[0] += k
            inter = n2 * np.fft.ifft(inter, axis=1)
            real, k = ranks.transpose(L, 2, rank, inter, groups)
            sent[1] += k
            psi = n1 * np.fft.ifft(real, axis=1)                  # [cols (b, c)][a]
            cols = L.local_real(rank)
            psis.append(psi)
            # x V(r), then back: x-pass, transposes reversed, y-pass, z-pass, gather
            u = psi * V[:, cols[:, 0], cols[:, 1]].T
            inter2, _ = ranks.transpose(L, 2, rank, np.fft.fft(u, axis=1), groups, reverse=True)
            cyl2, _ = ranks.transpose(L, 1, rank, np.fft.fft(inter2, axis=1), groups, reverse=True)
            qi, val = L.gather(rank, np.fft.fft(cyl2, axis=1) / (n1 * n2 * n3))
            outs.append((qi, val))
        q.put((rank, L.local_real(rank), psis, outs, sent))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("alg,world", [("greedy", 4), ("basic", 4), ("improved", 6), ("basic", 6)])
def test_distributed_apply_over_gloo_ranks(alg, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_apply, args=(r, world, port, alg, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = (12, 10, 9)
    g = synth.sphere_glist(*n, 3.2, order="shuffled", seed=4)
    c = synth.coefficients(g, 2, seed=5)
    V, _ = synth.potential(*n, "smooth", seed=6)
    psi_ref = O.to_real(n, g, c)
    out_ref = O.apply(n, g, c, V)
    out = np.zeros_like(out_ref)
    L = ranks.RankLayout(n, g, world, alg)
    sent = np.zeros(2, dtype=np.int64)
    for rank, cols, psis, outs, s in res:
        sent += s
        for b in range(2):
            want = psi_ref[b][:, cols[:, 0], cols[:, 1]].T
            assert np.abs(psis[b] - want).max() < 1e-12 * np.abs(psi_ref[b]).max()
            qi, val = outs[b]
            out[b, qi] = val
    assert np.abs(out - out_ref).max() < 1e-12 * np.abs(out_ref).max()
    # every message the model counts was sent (twice: one per band)
    assert sent[0] == 2 * L.message_count(1) and sent[1] == 2 * L.message_count(2)
