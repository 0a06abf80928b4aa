"""Multi-rank layouts of the compact 3-D FFT and their transposes (Sec. 3-4).

The paper distributes one band's FFT grid over p processes in three layouts,
one per set of 1-D FFTs, and transposes the data between them:

* greedy (Sec. 3.2, Fig. 2): first-pass columns sorted by plane-wave count
  (descending) and dealt round robin to the p ranks; the second- and
  third-pass columns dealt cyclically by complete planes, so the second
  transpose moves nothing (Sec. 5) and the first is one global all-to-all
  (p (p - 1) messages, Eq. 4);
* basic (Sec. 4.1, Figs. 3-4): ranks form an m x n grid (p = m n, |m - n|
  minimal, m >= n); columns are dealt cyclically so the first transpose is m
  independent all-to-alls inside row groups and the second n inside column
  groups (p (sqrt(p) - 1) messages each when m = n, Eq. 5);
* improved (Sec. 4.2): the basic algorithm with the first-pass layout's
  planes sorted by plane-wave count and dealt round robin to row and column
  groups.

Axis naming follows the GPU path: the first pass runs along axis 2 (the
paper's x), on "sticks" (a, b) = (h mod n1, k mod n2); the second along axis
1 on columns (a, c), a an occupied plane; the third along axis 0 on columns
(b, c).  The paper's x, y, z are our axes 2, 1, 0.

This module is host logic: it builds the owner tables, counts the messages
and moves data between ranks with ``torch.distributed`` all-to-alls inside
the row/column process groups.  The 1-D transforms themselves are not here:
the caller runs them on each layout's local columns.
"""
from __future__ import annotations

import math

import numpy as np

ALGORITHMS = ("greedy", "basic", "improved")


def proc_grid(p: int) -> tuple[int, int]:
    """p = m x n with |m - n| minimal and m >= n (m rows, n columns), Sec. 4.1."""
    if p < 1:
        raise ValueError("p must be positive")
    m = p
    for d in range(1, int(math.isqrt(p)) + 1):
        if p % d == 0:
            m = p // d
    return m, p // m


def _round_robin(order, k):
    out = np.empty(len(order), dtype=np.int64)
    out[np.asarray(order, dtype=np.int64)] = np.arange(len(order)) % k
    return out


class RankLayout:
    """Owner tables of the three layouts for one grid, G-list, p and algorithm.

    recip_owner[s]  rank of first-pass stick s (sticks in ascending id
                    a * n2 + b order, ``sticks``);
    inter_owner[a, c]  rank of second-pass column (a, c);
    real_owner[b, c]   rank of third-pass column (b, c).
    """

    def __init__(self, n, g, p: int, algorithm: str = "greedy"):
        if algorithm not in ALGORITHMS:
            raise ValueError(f"algorithm must be one of {ALGORITHMS}")
        self.n = tuple(int(x) for x in n)
        n1, n2, n3 = self.n
        self.p, self.algorithm = int(p), algorithm
        self.m, self.ncol = proc_grid(self.p)
        g = np.asarray(g, dtype=np.int64).reshape(-1, 3)
        self.npw = len(g)
        self.pw_a, self.pw_b, self.pw_c = g[:, 0] % n1, g[:, 1] % n2, g[:, 2] % n3
        sid = self.pw_a * n2 + self.pw_b
        self.sticks, self.pw_stick, self.stick_pw = np.unique(sid, return_inverse=True, return_counts=True)
        self.stick_a, self.stick_b = self.sticks // n2, self.sticks % n2
        self.planes = np.unique(self.stick_a)
        m, nc, P = self.m, self.ncol, self.p
        if algorithm == "greedy":
            # Sec. 3.2: sticks by #PW descending (ties: ascending id), round robin
            order = np.lexsort((self.sticks, -self.stick_pw))
            self.recip_owner = _round_robin(order, P)
            # complete planes of constant c (the paper's yz-planes) per rank
            self.inter_owner = np.broadcast_to(np.arange(n3) % P, (n1, n3)).copy()
            self.real_owner = np.broadcast_to(np.arange(n3) % P, (n2, n3)).copy()
        else:
            if algorithm == "basic":
                row_of_a = np.arange(n1) % m
                col_of_b = np.arange(n2) % nc
            else:
                # Sec. 4.2: plane weights = #PW; sorted descending (ties by
                # index), dealt round robin to row / column groups
                wa = np.bincount(self.stick_a, weights=self.stick_pw, minlength=n1)
                wb = np.bincount(self.stick_b, weights=self.stick_pw, minlength=n2)
                row_of_a = _round_robin(np.lexsort((np.arange(n1), -wa)), m)
                col_of_b = _round_robin(np.lexsort((np.arange(n2), -wb)), nc)
            self.recip_owner = row_of_a[self.stick_a] * nc + col_of_b[self.stick_b]
            # second pass shares the first's rows (by a) and the third's columns (by c)
            self.inter_owner = row_of_a[:, None] * nc + (np.arange(n3) % nc)[None, :]
            self.real_owner = (np.arange(n2) % m)[:, None] * nc + (np.arange(n3) % nc)[None, :]
        self._plans = {}

    # ------------------------------------------------------------ loads
    def pw_per_rank(self) -> np.ndarray:
        """Plane waves held by each rank in the first-pass layout (Tab. 2)."""
        return np.bincount(self.recip_owner, weights=self.stick_pw, minlength=self.p).astype(np.int64)

    def columns_per_rank(self):
        """1-D transforms per rank in each layout (compact FFT: sticks, the
        occupied planes' (a, c) columns, every (b, c) column)."""
        r = np.bincount(self.recip_owner, minlength=self.p)
        i = np.bincount(self.inter_owner[self.planes].ravel(), minlength=self.p)
        x = np.bincount(self.real_owner.ravel(), minlength=self.p)
        return r, i, x

    # -------------------------------------------------- the two transposes
    def _elements(self, which: int):
        """Global elements moved by transpose `which` (1 or 2): canonical
        linear index, source and destination rank."""
        n1, n2, n3 = self.n
        if which == 1:  # sticks (a, b) x every c
            a = np.repeat(self.stick_a, n3)
            b = np.repeat(self.stick_b, n3)
            c = np.tile(np.arange(n3), len(self.sticks))
            src = np.repeat(self.recip_owner, n3)
            dst = self.inter_owner[a, c]
        else:           # occupied planes a x every (b, c)
            a = np.repeat(self.planes, n2 * n3)
            b = np.tile(np.repeat(np.arange(n2), n3), len(self.planes))
            c = np.tile(np.arange(n3), len(self.planes) * n2)
            src = self.inter_owner[a, c]
            dst = self.real_owner[b, c]
        return (a * n2 + b) * n3 + c, a, b, c, src, dst

    def message_matrix(self, which: int) -> np.ndarray:
        """Elements sent from rank i to rank j by transpose `which` [p][p]."""
        _, _, _, _, src, dst = self._elements(which)
        return np.bincount(src * self.p + dst, minlength=self.p * self.p).reshape(self.p, self.p)

    def message_count(self, which: int) -> int:
        """Messages of transpose `which`: non-empty (i -> j) pairs, i != j."""
        M = self.message_matrix(which)
        return int(np.count_nonzero(M) - np.count_nonzero(np.diag(M)))

    def groups(self, which: int):
        """Process groups transpose `which` exchanges within (sorted rank
        lists): the whole world (greedy, first transpose), none (greedy,
        second), rows of n ranks (first) or columns of m ranks (second)."""
        m, nc = self.m, self.ncol
        if self.algorithm == "greedy":
            return [list(range(self.p))] if which == 1 else []
        if which == 1:
            return [[r * nc + j for j in range(nc)] for r in range(m)]
        return [[r * nc + j for r in range(m)] for j in range(nc)]

    # ------------------------------------------------------ local layouts
    def local_sticks(self, rank: int) -> np.ndarray:
        """Indices (into ``sticks``) of the rank's first-pass sticks, ascending."""
        return np.flatnonzero(self.recip_owner == rank)

    def local_inter(self, rank: int) -> np.ndarray:
        """(a, c) second-pass columns of the rank, a an occupied plane,
        ascending a * n3 + c; int64 [k, 2]."""
        a, c = np.nonzero(self.inter_owner[self.planes] == rank)
        return np.stack([self.planes[a], c], axis=1)

    def local_real(self, rank: int) -> np.ndarray:
        """(b, c) third-pass columns of the rank, ascending b * n3 + c; [k, 2]."""
        b, c = np.nonzero(self.real_owner == rank)
        return np.stack([b, c], axis=1)

    def local_pw(self, rank: int):
        """(plane-wave indices, local stick index, c) of the rank's plane waves."""
        loc = np.full(len(self.sticks), -1, dtype=np.int64)
        ls = self.local_sticks(rank)
        loc[ls] = np.arange(len(ls))
        q = np.flatnonzero(self.recip_owner[self.pw_stick] == rank)
        return q, loc[self.pw_stick[q]], self.pw_c[q]

    def scatter(self, rank: int, c_band) -> np.ndarray:
        """The rank's first-pass stick array [local sticks][n3] from one
        band's coefficients (zeros off the sphere)."""
        q, s, z = self.local_pw(rank)
        out = np.zeros((len(self.local_sticks(rank)), self.n[2]), dtype=np.complex128)
        out[s, z] = np.asarray(c_band)[q]
        return out

    def gather(self, rank: int, cyl) -> tuple[np.ndarray, np.ndarray]:
        """(plane-wave indices, values) of the rank's plane waves from its
        first-pass stick array."""
        q, s, z = self.local_pw(rank)
        return q, np.asarray(cyl)[s, z]

    def _plan(self, which: int, rank: int):
        """Send / receive index lists of one rank for transpose `which`
        (forward direction), ordered by group member, then canonical index."""
        key = (which, rank)
        if key in self._plans:
            return self._plans[key]
        n1, n2, n3 = self.n
        lin, a, b, c, src, dst = self._elements(which)
        if which == 1:
            ls = self.local_sticks(rank)
            sloc = np.full(len(self.sticks), -1, dtype=np.int64)
            sloc[ls] = np.arange(len(ls))
            stick_of = np.searchsorted(self.sticks, a * n2 + b)
            src_pos = sloc[stick_of] * n3 + c                   # in [sticks][n3]
            li = self.local_inter(rank)
            key_in = li[:, 0] * n3 + li[:, 1]
            dst_pos = np.searchsorted(key_in, a * n3 + c) * n2 + b  # in [cols][n2]
        else:
            li = self.local_inter(rank)
            key_in = li[:, 0] * n3 + li[:, 1]
            src_pos = np.searchsorted(key_in, a * n3 + c) * n2 + b
            lr = self.local_real(rank)
            key_r = lr[:, 0] * n3 + lr[:, 1]
            dst_pos = np.searchsorted(key_r, b * n3 + c) * n1 + a   # in [cols][n1]
        group = next((gr for gr in self.groups(which) if rank in gr), [rank])
        send, recv = [], []
        for peer in group:
            s = np.flatnonzero((src == rank) & (dst == peer))
            r = np.flatnonzero((src == peer) & (dst == rank))
            send.append(src_pos[s[np.argsort(lin[s], kind="stable")]])
            recv.append(dst_pos[r[np.argsort(lin[r], kind="stable")]])
        plan = (group, send, recv)
        self._plans[key] = plan
        return plan

    def local_shape(self, rank: int, layout: int) -> tuple[int, int]:
        """Shape of a rank's local array in layout 1 (sticks x n3), 2 (second-
        pass columns x n2) or 3 (third-pass columns x n1)."""
        if layout == 1:
            return len(self.local_sticks(rank)), self.n[2]
        if layout == 2:
            return len(self.local_inter(rank)), self.n[1]
        return len(self.local_real(rank)), self.n[0]


def transpose(layout: RankLayout, which: int, rank: int, data, pgroups=None, *, reverse: bool = False):
    """Run transpose `which` (1: layout 1 -> 2, 2: layout 2 -> 3; ``reverse``
    for 2 -> 1 / 3 -> 2) for this rank with torch.distributed all-to-alls in
    the transpose's process group.  ``pgroups`` maps a sorted rank tuple to
    its ``dist.new_group`` handle (None: the default group).  Entries of the
    target layout that no element reaches are zero.  Returns (array, number
    of non-empty messages this rank sent)."""
    import torch
    import torch.distributed as dist
    group, send, recv = layout._plan(which, rank)
    if reverse:
        send, recv = recv, send
    src_layout, dst_layout = (which, which + 1) if not reverse else (which + 1, which)
    out = np.zeros(layout.local_shape(rank, dst_layout), dtype=np.complex128)
    flat_in = np.ascontiguousarray(data, dtype=np.complex128).reshape(-1)
    flat_out = out.reshape(-1)
    buf = np.concatenate([flat_in[s] for s in send]) if send else np.zeros(0, np.complex128)
    sizes_in = [len(s) for s in send]
    sizes_out = [len(r) for r in recv]
    sent = sum(1 for peer, k in zip(group, sizes_in) if peer != rank and k > 0)
    if len(group) == 1:
        rbuf = buf
    else:
        tin = torch.from_numpy(buf.view(np.float64).copy())
        tout = torch.empty(2 * sum(sizes_out), dtype=torch.float64)
        pg = None if pgroups is None else pgroups.get(tuple(group))
        dist.all_to_all_single(tout, tin, [2 * k for k in sizes_out], [2 * k for k in sizes_in], group=pg)
        rbuf = tout.numpy().view(np.complex128)
    off = 0
    for r in recv:
        flat_out[r] = rbuf[off:off + len(r)]
        off += len(r)
    return out, sent


def make_groups(layout: RankLayout):
    """Create every process group the layout's transposes use (call on all
    ranks, in the same order); returns {sorted rank tuple: group}."""
    import torch.distributed as dist
    out = {}
    for which in (1, 2):
        for gr in layout.groups(which):
            t = tuple(gr)
            if len(t) > 1 and t not in out:
                out[t] = dist.new_group(list(t)) if len(t) < dist.get_world_size() else None
    return out


def comm_cost(p: int, n_fft: int, alpha: float, beta: float, mu: float = 16.0, *, kind: str = "global") -> float:
    """Qualitative cost of one transpose: Eq. 4 (global all-to-all,
    (p - 1)(alpha + mu N / (beta p^2))) or Eq. 5 (local all-to-alls,
    (sqrt(p) - 1)(alpha + mu N / (beta p sqrt(p))))."""
    if kind == "global":
        return (p - 1) * (alpha + mu * n_fft / (beta * p * p))
    if kind == "local":
        s = math.sqrt(p)
        return (s - 1) * (alpha + mu * n_fft / (beta * p * s))
    raise ValueError(kind)
