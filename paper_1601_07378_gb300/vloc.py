"""Python binding of libvloc (argument marshalling only).

Every step of the V_loc action runs in the CUDA kernels behind the C ABI of
``include/vloc.h``; this module only passes device pointers, sizes and the
current CUDA stream.  PyTorch supplies device memory and streams.  There is
no CPU or library fallback: if the extension is missing, the first call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvloc.so")

VLOC_OK = 0
VLOC_ERR_ARG = -1
VLOC_ERR_SIZE = -2
VLOC_ERR_GLIST = -3
VLOC_ERR_ALLOC = -4
VLOC_ERR_CUDA = -5
VLOC_ERR_TIMEOUT = -6
VLOC_ERR_STATE = -7

VLOC_F32 = 0x001
VLOC_F64 = 0x002
VLOC_PARTITION_GREEDY = 0x000
VLOC_PARTITION_BASIC = 0x010
VLOC_PARTITION_IMPROVED = 0x020
VLOC_GRAPH = 0x100
VLOC_HOST_ONLY = 0x200
VLOC_GENERIC_KERNELS = 0x400
VLOC_GAMMA = 0x1000
VLOC_DOUBLE_FLOAT = 0x2000
VLOC_X_TMA = 0x4000
VLOC_Z_WARP = 0x20000
VLOC_Z_BULK = 0x40000
VLOC_POISON_WORKSPACE = 0x10000

# every exported symbol declared in include/vloc.h
EXPORTS = [
    "vloc_plan_create", "vloc_plan_destroy", "vloc_apply", "vloc_apply_adjoint", "vloc_backward",
    "vloc_apply_batched", "vloc_apply_host", "vloc_get_index_map", "vloc_get_partition",
    "vloc_get_info", "vloc_strerror", "vloc_version", "vloc_last_cuda_error",
    "vloc_profile", "vloc_get_profile", "vloc_get_launch_count", "vloc_apply_noalloc",
    "vloc_plan_set_schedule", "vloc_to_real", "vloc_to_recip", "vloc_density",
    "vloc_apply_h", "vloc_device_status", "vloc_alu_peak", "vloc_apply_host_async",
]

KERNEL_NAMES = ["k1_scatter_zpass", "k2_ypass_inv", "k3_xpass_v", "k2_ypass_fwd", "k4_zpass_gather",
                "k3b_grad_v", "aux", "gamma_pack_unpack", "k3_to_grid", "k3_from_grid", "k3d_density",
                "unused"]


class VlocKernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class VlocInfo(ctypes.Structure):
    _fields_ = [
        ("n1", ctypes.c_int32), ("n2", ctypes.c_int32), ("n3", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("npw", ctypes.c_int64),
        ("nsticks", ctypes.c_int32), ("nplanes", ctypes.c_int32), ("nparts", ctypes.c_int32),
        ("lines_per_tile", ctypes.c_int32), ("chunk_bands", ctypes.c_int64),
        ("workspace_bytes", ctypes.c_int64), ("radix", (ctypes.c_int32 * 4) * 3),
        ("nstages", ctypes.c_int32 * 3), ("path", ctypes.c_int32),
    ]


class VlocError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = f"{what}: {strerror(code)} ({code})"
        extra = last_cuda_error()
        if extra and code in (VLOC_ERR_CUDA, VLOC_ERR_ALLOC):
            msg += f" [{extra}]"
        super().__init__(msg)


_lib = None
_lock = threading.Lock()


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libvloc.so (built by ``paper_1601_07378_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libvloc.so is not built ({p}); run paper_1601_07378_gb300.build.build()")
        lib = ctypes.CDLL(p)
        vp, i64, i32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        lib.vloc_plan_create.argtypes = [ctypes.POINTER(vp), c_int, c_int, c_int, ctypes.POINTER(i32), i64, c_int, i64, vp]
        lib.vloc_plan_destroy.argtypes = [vp]
        for f in (lib.vloc_apply, lib.vloc_apply_adjoint, lib.vloc_apply_host, lib.vloc_apply_noalloc,
                  lib.vloc_apply_host_async):
            f.argtypes = [vp, vp, vp, i64, vp, vp]
        lib.vloc_backward.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
        lib.vloc_apply_batched.argtypes = [c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                           ctypes.POINTER(i64), ctypes.POINTER(vp), vp]
        lib.vloc_get_index_map.argtypes = [vp, ctypes.POINTER(i64)]
        lib.vloc_get_partition.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.vloc_get_info.argtypes = [vp, ctypes.POINTER(VlocInfo)]
        lib.vloc_strerror.argtypes = [c_int]
        lib.vloc_strerror.restype = ctypes.c_char_p
        lib.vloc_last_cuda_error.argtypes = []
        lib.vloc_last_cuda_error.restype = ctypes.c_char_p
        lib.vloc_version.argtypes = []
        lib.vloc_profile.argtypes = [vp, c_int]
        lib.vloc_plan_set_schedule.argtypes = [vp, c_int, c_int, ctypes.POINTER(i32)]
        lib.vloc_get_profile.argtypes = [vp, ctypes.POINTER(VlocKernelStat)]
        lib.vloc_get_launch_count.argtypes = [vp, ctypes.POINTER(i64)]
        lib.vloc_apply_h.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        lib.vloc_device_status.argtypes = [vp]
        lib.vloc_to_real.argtypes = [vp, vp, i64, vp, vp]
        lib.vloc_to_recip.argtypes = [vp, vp, i64, vp, vp]
        lib.vloc_density.argtypes = [vp, vp, vp, i64, vp, vp]
        lib.vloc_alu_peak.argtypes = [c_int, i64, vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), vp]
        for name in EXPORTS:
            getattr(lib, name)
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().vloc_strerror(code).decode()
    except RuntimeError:
        return str(code)


def last_cuda_error() -> str:
    try:
        return load().vloc_last_cuda_error().decode()
    except RuntimeError:
        return ""


def _check(code: int, what: str):
    if code != VLOC_OK:
        raise VlocError(code, what)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


PEAK_KINDS = {"dfma": 0, "dadd": 1, "ffma": 2, "ffma2": 3, "fadd2": 4}


def alu_peak(kind: str, iters: int, *, stream=None) -> dict:
    """Run one arithmetic-rate probe (vloc_alu_peak) on the current device;
    returns the FLOPs of the launch, its event time and the GFLOP/s."""
    import torch
    lib = load()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    flops, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib.vloc_alu_peak(PEAK_KINDS[kind], int(iters), _ptr(sink), ctypes.byref(flops), ctypes.byref(ms),
                             _stream_ptr(stream)), "vloc_alu_peak")
    return {"flops": flops.value, "ms": ms.value, "gflops": flops.value / (ms.value * 1e6)}


class VlocPlan:
    """Plan of the V_loc action for one grid (n1, n2, n3) and one G-list.

    ``glist`` is an int array [npw, 3] of Miller indices; ``dtype`` is
    ``torch.complex64`` (FP32 path) or ``torch.complex128`` (FP64 path).
    ``double_float=True`` (with complex128) runs the apply in double-float
    arithmetic on the FP32 pipes, FP64 data in and out.
    ``poison=True`` (a test aid) fills the workspace with NaN before every
    chunk, so a pass that reads a cell its chunk never wrote shows up as a
    non-finite result.
    ``gamma=True`` selects the Gamma-point real mode (Sec. 4.3): ``glist`` is
    half of a G -> -G symmetric sphere, the bands are real in r-space
    (c(-G) = conj c(G) implied, c(0) taken real) and two of them share one
    complex transform.
    """

    def __init__(self, grid, glist, dtype=None, *, partition: str = "greedy", chunk: int = 0,
                 graph: bool = False, host_only: bool = False, generic: bool = False, gamma: bool = False,
                 double_float: bool = False, x_tma: bool = False, z_warp: bool = False, z_bulk: bool = False,
                 poison: bool = False, stream=None):
        import torch
        dtype = dtype or torch.complex64
        if dtype not in (torch.complex64, torch.complex128):
            raise TypeError("dtype must be torch.complex64 or torch.complex128")
        self.lib = load()
        self.grid = tuple(int(x) for x in grid)
        self.dtype = dtype
        self.real_dtype = torch.float32 if dtype == torch.complex64 else torch.float64
        g = np.ascontiguousarray(np.asarray(glist, dtype=np.int32).reshape(-1, 3))
        self.glist = g
        self.npw = len(g)
        flags = VLOC_F32 if dtype == torch.complex64 else VLOC_F64
        flags |= {"greedy": VLOC_PARTITION_GREEDY, "basic": VLOC_PARTITION_BASIC,
                  "improved": VLOC_PARTITION_IMPROVED}[partition]
        if graph:
            flags |= VLOC_GRAPH
        if host_only:
            flags |= VLOC_HOST_ONLY
        if generic:
            flags |= VLOC_GENERIC_KERNELS
        self.gamma = bool(gamma)
        if gamma:
            flags |= VLOC_GAMMA
        if double_float:
            flags |= VLOC_DOUBLE_FLOAT
        if x_tma:
            flags |= VLOC_X_TMA
        if z_warp:
            flags |= VLOC_Z_WARP
        if z_bulk:
            flags |= VLOC_Z_BULK
        if poison:
            flags |= VLOC_POISON_WORKSPACE
        h = ctypes.c_void_p()
        sp = ctypes.c_void_p(None) if host_only else _stream_ptr(stream)
        _check(self.lib.vloc_plan_create(ctypes.byref(h), *self.grid,
                                         g.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self.npw,
                                         flags, int(chunk), sp), "vloc_plan_create")
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.lib.vloc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- info
    def info(self) -> dict:
        inf = VlocInfo()
        _check(self.lib.vloc_get_info(self.handle, ctypes.byref(inf)), "vloc_get_info")
        return {
            "grid": (inf.n1, inf.n2, inf.n3), "precision": inf.precision, "npw": inf.npw,
            "nsticks": inf.nsticks, "nplanes": inf.nplanes, "nparts": inf.nparts,
            "lines_per_tile": inf.lines_per_tile, "chunk_bands": inf.chunk_bands,
            "workspace_bytes": inf.workspace_bytes,
            "radix": [[inf.radix[a][i] for i in range(inf.nstages[a])] for a in range(3)],
            "compile_time_kernels": bool(inf.path & 1),
            "gamma": bool(inf.path & 4),
            "double_float": bool(inf.path & 8),
            "x_tma": bool(inf.path & 16),
            "x_quarter": bool(inf.path & 32),
            "z_quarter": bool(inf.path & 64),
            "gamma_fused": bool(inf.path & 128),
            "z_warp": bool(inf.path & 256),
            "z_bulk": bool(inf.path & 512),
        }

    def set_schedule(self, axis: int, radices):
        """Replace one axis's radix schedule (switches the plan to the
        runtime-radix kernels)."""
        arr = (ctypes.c_int32 * len(radices))(*[int(r) for r in radices])
        _check(self.lib.vloc_plan_set_schedule(self.handle, int(axis), len(radices), arr), "vloc_plan_set_schedule")

    def profile(self, enable: bool = True):
        _check(self.lib.vloc_profile(self.handle, int(enable)), "vloc_profile")

    def get_profile(self) -> dict:
        arr = (VlocKernelStat * len(KERNEL_NAMES))()
        _check(self.lib.vloc_get_profile(self.handle, arr), "vloc_get_profile")
        return {KERNEL_NAMES[i]: (int(arr[i].launches), float(arr[i].total_ms)) for i in range(len(KERNEL_NAMES)) if arr[i].launches}

    def device_status(self) -> int:
        """Synchronise; VLOC_ERR_TIMEOUT if a bounded in-kernel wait gave up since the last call."""
        return int(self.lib.vloc_device_status(self.handle))

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        _check(self.lib.vloc_get_launch_count(self.handle, ctypes.byref(n)), "vloc_get_launch_count")
        return int(n.value)

    def index_map(self) -> np.ndarray:
        out = np.empty(self.npw, dtype=np.int64)
        _check(self.lib.vloc_get_index_map(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "vloc_get_index_map")
        return out

    def partition(self) -> tuple[np.ndarray, int]:
        n = ctypes.c_int32()
        _check(self.lib.vloc_get_partition(self.handle, None, ctypes.byref(n)), "vloc_get_partition")
        S = self.info()["nsticks"]
        out = np.empty(S, dtype=np.int32)
        _check(self.lib.vloc_get_partition(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           ctypes.byref(n)), "vloc_get_partition")
        return out, int(n.value)

    # ------------------------------------------------------------- checks
    def _check_c(self, c, name="coeffs"):
        if not c.is_cuda or c.dtype != self.dtype or not c.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {self.dtype} tensor")
        if c.shape[-1] != self.npw:
            raise ValueError(f"{name} last dim must be npw={self.npw}")

    def _check_V(self, V):
        if not V.is_cuda or V.dtype != self.real_dtype or not V.is_contiguous() or V.numel() != np.prod(self.grid):
            raise ValueError(f"V must be a contiguous CUDA {self.real_dtype} tensor with {np.prod(self.grid)} elements")

    def _check_out(self, out, c, name="out"):
        # the kernels write as many bands as they read: a smaller buffer would be overrun
        self._check_c(out, name)
        if out.numel() != c.numel():
            raise ValueError(f"{name} must hold as many bands as the input ({c.numel() // self.npw})")

    # ---------------------------------------------------------------- calls
    def apply(self, c, V, out=None, *, adjoint: bool = False, stream=None):
        """out = A c (or A^H c) for c of shape [..., npw]."""
        import torch
        self._check_c(c)
        self._check_V(V)
        if out is None:
            out = torch.empty_like(c)
        else:
            self._check_out(out, c)
        nb = c.numel() // self.npw
        fn = self.lib.vloc_apply_adjoint if adjoint else self.lib.vloc_apply
        _check(fn(self.handle, _ptr(c), _ptr(V), nb, _ptr(out), _stream_ptr(stream)),
               "vloc_apply_adjoint" if adjoint else "vloc_apply")
        return out

    def apply_h(self, c, V, diag, out=None, *, stream=None):
        """out = (diag(d) + A) c: V_loc plus a term diagonal in G (e.g. kinetic |k+G|^2/2)."""
        import torch
        self._check_c(c)
        self._check_V(V)
        if not diag.is_cuda or diag.dtype != self.real_dtype or not diag.is_contiguous() or diag.numel() != self.npw:
            raise ValueError(f"diag must be a contiguous CUDA {self.real_dtype} tensor of npw={self.npw} entries")
        if out is None:
            out = torch.empty_like(c)
        else:
            self._check_out(out, c)
        nb = c.numel() // self.npw
        _check(self.lib.vloc_apply_h(self.handle, _ptr(c), _ptr(V), _ptr(diag), nb, _ptr(out), _stream_ptr(stream)),
               "vloc_apply_h")
        return out

    def backward(self, c, grad_out, V, *, need_c: bool = True, need_V: bool = True, stream=None):
        """(dL/dc, dL/dV) through out = A c (PyTorch complex-gradient convention)."""
        import torch
        self._check_c(c)
        self._check_c(grad_out, "grad_out")
        self._check_V(V)
        gc = torch.empty_like(c) if need_c else None
        gV = torch.empty(self.grid, dtype=self.real_dtype, device=c.device) if need_V else None
        nb = c.numel() // self.npw
        _check(self.lib.vloc_backward(self.handle, _ptr(c), _ptr(grad_out), _ptr(V), nb,
                                      _ptr(gc) if gc is not None else None,
                                      _ptr(gV) if gV is not None else None, _stream_ptr(stream)), "vloc_backward")
        return gc, gV

    def to_real(self, c, psi=None, *, stream=None):
        """psi_n = F+ S c_n on the full grid: [nb, n1, n2, n3] complex."""
        import torch
        self._check_c(c)
        nb = c.numel() // self.npw
        if psi is None:
            psi = torch.empty((nb, *self.grid), dtype=self.dtype, device=c.device)
        elif not psi.is_cuda or psi.dtype != self.dtype or not psi.is_contiguous() or \
                psi.numel() != nb * int(np.prod(self.grid)):
            raise ValueError("psi must be a contiguous CUDA tensor of nb full grids")
        _check(self.lib.vloc_to_real(self.handle, _ptr(c), nb, _ptr(psi), _stream_ptr(stream)), "vloc_to_real")
        return psi

    def to_recip(self, u, out=None, *, stream=None):
        """out_n(G) = (1/N) sum_r u_n(r) exp(-2 pi i G.r/n) for full grids u [nb, n1, n2, n3]."""
        import torch
        N = int(np.prod(self.grid))
        if not u.is_cuda or u.dtype != self.dtype or not u.is_contiguous() or u.numel() % N:
            raise ValueError("u must be a contiguous CUDA tensor of full grids")
        nb = u.numel() // N
        if out is None:
            out = torch.empty((nb, self.npw), dtype=self.dtype, device=u.device)
        else:
            self._check_c(out, "out")
            if out.numel() != nb * self.npw:
                raise ValueError(f"out must hold nb = {nb} bands of npw = {self.npw}")
        _check(self.lib.vloc_to_recip(self.handle, _ptr(u), nb, _ptr(out), _stream_ptr(stream)), "vloc_to_recip")
        return out

    def density(self, c, occ=None, rho=None, *, stream=None):
        """rho(r) = sum_n f_n |psi_n(r)|^2 (f_n = occ[n], 1 when None): real [n1, n2, n3]."""
        import torch
        self._check_c(c)
        nb = c.numel() // self.npw
        if occ is not None and (not occ.is_cuda or occ.dtype != self.real_dtype or not occ.is_contiguous()
                                or occ.numel() != nb):
            raise ValueError(f"occ must be a contiguous CUDA {self.real_dtype} tensor of nb weights")
        if rho is None:
            rho = torch.empty(self.grid, dtype=self.real_dtype, device=c.device)
        elif not rho.is_cuda or rho.dtype != self.real_dtype or not rho.is_contiguous() or \
                rho.numel() != int(np.prod(self.grid)):
            raise ValueError(f"rho must be a contiguous CUDA {self.real_dtype} tensor with {np.prod(self.grid)} elements")
        _check(self.lib.vloc_density(self.handle, _ptr(c), _ptr(occ) if occ is not None else None, nb, _ptr(rho),
                                     _stream_ptr(stream)), "vloc_density")
        return rho

    def apply_host(self, c_host, V_host, out_host=None, *, stream=None, blocking: bool = True):
        """A c with host (CPU, preferably pinned) tensors; copies inside the call.
        ``blocking=False`` enqueues the copies and applies and returns at
        once: ``out_host`` holds the result after ``stream`` is synchronised,
        and the host tensors must stay untouched until then."""
        import torch
        if c_host.is_cuda or V_host.is_cuda:
            raise ValueError("apply_host takes CPU tensors")
        if c_host.dtype != self.dtype or not c_host.is_contiguous() or c_host.shape[-1] != self.npw:
            raise ValueError("bad host coefficients")
        if V_host.dtype != self.real_dtype or not V_host.is_contiguous() or V_host.numel() != np.prod(self.grid):
            raise ValueError("bad host V")
        if out_host is None:
            out_host = torch.empty_like(c_host, pin_memory=c_host.is_pinned())
        elif out_host.is_cuda or out_host.dtype != self.dtype or not out_host.is_contiguous() or \
                out_host.numel() != c_host.numel():
            raise ValueError("out_host must be a contiguous host tensor shaped like the coefficients")
        nb = c_host.numel() // self.npw
        fn = self.lib.vloc_apply_host if blocking else self.lib.vloc_apply_host_async
        _check(fn(self.handle, _ptr(c_host), _ptr(V_host), nb, _ptr(out_host), _stream_ptr(stream)),
               "vloc_apply_host")
        return out_host


def apply_batched(plans, cs, Vs, outs=None, *, stream=None):
    """Several plans (different grids / spheres) applied back to back in one call."""
    import torch
    n = len(plans)
    if outs is None:
        outs = [torch.empty_like(c) for c in cs]
    if not (len(cs) == len(Vs) == len(outs) == n):
        raise ValueError("plans, coefficients, potentials and outputs must have one entry per instance")
    for p, c, V, o in zip(plans, cs, Vs, outs):
        p._check_c(c)
        p._check_V(V)
        p._check_out(o, c)
    arr = lambda xs: (ctypes.c_void_p * n)(*[ctypes.c_void_p(x) for x in xs])
    nbs = (ctypes.c_int64 * n)(*[c.numel() // p.npw for p, c in zip(plans, cs)])
    lib = load()
    _check(lib.vloc_apply_batched(n, arr([p.handle.value for p in plans]), arr([c.data_ptr() for c in cs]),
                                  arr([V.data_ptr() for V in Vs]), nbs, arr([o.data_ptr() for o in outs]),
                                  _stream_ptr(stream)), "vloc_apply_batched")
    return outs


def _autograd_function():
    import torch

    class VlocApply(torch.autograd.Function):
        """out = A(V) c with the hand-written backward kernels.

        backward: dL/dc = A grad_out (A is Hermitian for real V),
        dL/dV(r) = (1/N) sum_n Re(conj(g_n(r)) psi_n(r)), psi_n recomputed.
        """

        @staticmethod
        def forward(ctx, c, V, plan):
            ctx.plan = plan
            ctx.save_for_backward(c, V)
            return plan.apply(c.contiguous(), V.contiguous())

        @staticmethod
        def backward(ctx, grad_out):
            c, V = ctx.saved_tensors
            plan = ctx.plan
            gc, gV = plan.backward(c.contiguous(), grad_out.contiguous(), V.contiguous(),
                                   need_c=ctx.needs_input_grad[0], need_V=ctx.needs_input_grad[1])
            if gV is not None:
                gV = gV.reshape(V.shape)
            return gc, gV, None

    return VlocApply


_VlocApply = None


def vloc_apply(c, V, plan):
    """Differentiable out = A(V) c (torch.autograd)."""
    global _VlocApply
    if _VlocApply is None:
        _VlocApply = _autograd_function()
    return _VlocApply.apply(c, V, plan)
