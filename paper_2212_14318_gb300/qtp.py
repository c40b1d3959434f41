"""Thin ctypes binding of libqtp (include/qtp.h).

Argument marshalling only: every step of the T-product runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors of shape (2, rows, cols, p, 2),
dtype float32, contiguous ("tube-contiguous complex-pair planes": plane 0 is
a + b i, plane 1 is c + d i of the quaternion a + b i + c j + d k).

There is no CPU fallback: if the library is not built, or no GPU is present,
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libqtp.so")

QTP_OK = 0
STATUS_NAMES = {0: "QTP_OK", 1: "QTP_ERR_INVALID_ARG", 2: "QTP_ERR_UNSUPPORTED", 3: "QTP_ERR_WORKSPACE",
                4: "QTP_ERR_CUDA", 5: "QTP_ERR_TIMEOUT", 6: "QTP_ERR_INTERNAL", 7: "QTP_ERR_NOT_CONVERGED"}
PRECISIONS = {"fp32": 0, "bf16x3": 1, "bf16": 2}
PLAN_AUTOTUNE = 1

# Every function the C header declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_i = ctypes.c_int
_sz = ctypes.c_size_t
SIGNATURES = {
    "qtp_plan_create": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _i, ctypes.c_uint]),
    "qtp_plan_destroy": (_i, [_vp]),
    "qtp_plan_get_tiles": (_i, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "qtp_plan_launch_count": (_i, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "qtp_workspace_size": (_i, [_vp, ctypes.POINTER(_sz)]),
    "qtp_backward_workspace_size": (_i, [_vp, ctypes.POINTER(_sz)]),
    "qtp_forward": (_i, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "qtp_host_buffer_size": (_i, [_vp, ctypes.POINTER(_sz)]),
    "qtp_forward_host": (_i, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "qtp_host_many_buffer_size": (_i, [_vp, ctypes.POINTER(_sz)]),
    "qtp_tsvd_workspace_size": (_i, [_i, _i, _i, ctypes.POINTER(_sz)]),
    "qtp_forward_saving": (_i, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "qtp_backward_saved": (_i, [_vp, _vp, _vp, _sz, _vp, _vp, _vp, _sz, _vp]),
    "qtp_tsvd": (_i, [_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "qtp_tsvd_sync": (_i, [_i, _i, _i, _vp, _vp]),
    "qtp_forward_host_many": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _sz,
                                   _vp]),
    "qtp_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "qtp_plan_sync": (_i, [_vp, _vp]),
    "qtp_plan_set_tracing": (_i, [_vp, _i]),
    "qtp_plan_stage_times": (_i, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "qtp_forward_noalloc": (_i, [_i, _i, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "qtp_batch_plan_create": (_i, [ctypes.POINTER(_vp), _vp, _i, _i, ctypes.c_uint]),
    "qtp_batch_plan_destroy": (_i, [_vp]),
    "qtp_batch_workspace_size": (_i, [_vp, ctypes.POINTER(_sz)]),
    "qtp_forward_batched": (_i, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "qtp_batch_plan_set_tracing": (_i, [_vp, _i]),
    "qtp_batch_stage_times": (_i, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "qtp_batch_plan_sync": (_i, [_vp, _vp]),
    "qtp_batch_plan_route": (_i, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(ctypes.c_int)]),
    "qtp_last_error": (ctypes.c_char_p, []),
    "qtp_version": (_i, []),
}

_lib = None
_lock = threading.Lock()


class QtpError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def lib() -> ctypes.CDLL:
    """Load libqtp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libqtp is not built ({LIB_PATH} missing); run "
                                   "`python -m paper_2212_14318_gb300.build` or __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != QTP_OK:
        msg = lib().qtp_last_error()
        raise QtpError(status, where, msg.decode() if msg else "")


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check_tensor(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float32")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _check_host_tensor(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float32")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def tsvd(A, workspace=None, stream=None, check=False):
    """T-SVD A = U * S * V^H of a CUDA tensor A (2, m, n, p, 2) (qtp_tsvd):
    returns U (2, m, k, p, 2), S (2, k, k, p, 2), V (2, n, k, p, 2) and sigma
    (p, k), k = min(m, n).  check: synchronise and raise QtpError
    (QTP_ERR_NOT_CONVERGED) if a frequency pair's sweeps did not converge
    (qtp_tsvd_sync)."""
    import torch
    if not isinstance(A, torch.Tensor) or A.dim() != 5 or A.shape[0] != 2 or A.shape[4] != 2:
        raise ValueError("A must have shape (2, m, n, p, 2)")
    _, m, n, p, _ = A.shape
    _check_tensor(A, (2, m, n, p, 2), "A")
    k = min(m, n)
    dev = A.device
    U = torch.empty((2, m, k, p, 2), dtype=torch.float32, device=dev)
    S = torch.empty((2, k, k, p, 2), dtype=torch.float32, device=dev)
    V = torch.empty((2, n, k, p, 2), dtype=torch.float32, device=dev)
    sigma = torch.empty((p, k), dtype=torch.float32, device=dev)
    need = ctypes.c_size_t()
    _check(lib().qtp_tsvd_workspace_size(m, n, p, ctypes.byref(need)), "qtp_tsvd_workspace_size")
    ws = workspace if workspace is not None else torch.empty(max(int(need.value), 256), dtype=torch.uint8, device=dev)
    _check(lib().qtp_tsvd(m, n, p, _ptr(A), _ptr(U), _ptr(S), _ptr(V), _ptr(sigma), _ptr(ws),
                          ws.numel() * ws.element_size(), _stream(stream)), "qtp_tsvd")
    if check:
        _check(lib().qtp_tsvd_sync(m, n, p, _ptr(ws), _stream(stream)), "qtp_tsvd_sync")
    return U, S, V, sigma


class Plan:
    """A qtp_plan for C = A * B with A in Q^{m x n x p}, B in Q^{n x s x p}."""

    def __init__(self, m: int, n: int, s: int, p: int, precision: str = "bf16x3", autotune: bool = False):
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {list(PRECISIONS)}")
        self.m, self.n, self.s, self.p = m, n, s, p
        self.precision = precision
        h = ctypes.c_void_p()
        _check(lib().qtp_plan_create(ctypes.byref(h), m, n, s, p, PRECISIONS[precision],
                                     PLAN_AUTOTUNE if autotune else 0), "qtp_plan_create")
        self._h = h
        self._ws = None
        self._bws = None

    # ------------------------------------------------------------------ sizes
    def _size(self, fn) -> int:
        v = ctypes.c_size_t()
        _check(getattr(lib(), fn)(self._h, ctypes.byref(v)), fn)
        return int(v.value)

    def workspace_size(self) -> int:
        return self._size("qtp_workspace_size")

    def backward_workspace_size(self) -> int:
        return self._size("qtp_backward_workspace_size")

    def host_buffer_size(self) -> int:
        return self._size("qtp_host_buffer_size")

    def _workspace(self, which: str, nbytes: int, device):
        import torch
        cur = getattr(self, which)
        if cur is None or cur.numel() < nbytes or cur.device != device:
            cur = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
            setattr(self, which, cur)
        return cur

    # ------------------------------------------------------------------ calls
    def forward(self, A, B, C=None, workspace=None, stream=None):
        import torch
        _check_tensor(A, (2, self.m, self.n, self.p, 2), "A")
        _check_tensor(B, (2, self.n, self.s, self.p, 2), "B")
        if C is None:
            C = torch.empty((2, self.m, self.s, self.p, 2), dtype=torch.float32, device=A.device)
        _check_tensor(C, (2, self.m, self.s, self.p, 2), "C")
        need = self.workspace_size()
        ws = workspace if workspace is not None else self._workspace("_ws", need, A.device)
        _check(lib().qtp_forward(self._h, _ptr(A), _ptr(B), _ptr(C), _ptr(ws), ws.numel() * ws.element_size(),
                                 _stream(stream)), "qtp_forward")
        return C

    def forward_host(self, A_host, B_host, C_host, dev_buffer, stream=None):
        """A, B, C are pinned CPU tensors; dev_buffer a CUDA byte tensor."""
        _check_host_tensor(A_host, (2, self.m, self.n, self.p, 2), "A_host")
        _check_host_tensor(B_host, (2, self.n, self.s, self.p, 2), "B_host")
        _check_host_tensor(C_host, (2, self.m, self.s, self.p, 2), "C_host")
        _check(lib().qtp_forward_host(self._h, _ptr(A_host), _ptr(B_host), _ptr(C_host), _ptr(dev_buffer),
                                      dev_buffer.numel() * dev_buffer.element_size(), _stream(stream)),
               "qtp_forward_host")
        return C_host

    def host_many_buffer_size(self) -> int:
        return self._size("qtp_host_many_buffer_size")

    def forward_host_many(self, A_hosts, B_hosts, C_hosts, dev_buffer, stream=None):
        """Independent products C_hosts[i] = A_hosts[i] * B_hosts[i] from pinned
        CPU tensors, copies overlapped with compute (qtp_forward_host_many);
        dev_buffer is a CUDA byte tensor of host_many_buffer_size() bytes."""
        count = len(A_hosts)
        if len(B_hosts) != count or len(C_hosts) != count:
            raise ValueError("A_hosts, B_hosts and C_hosts must have the same length")
        for i in range(count):
            _check_host_tensor(A_hosts[i], (2, self.m, self.n, self.p, 2), f"A_hosts[{i}]")
            _check_host_tensor(B_hosts[i], (2, self.n, self.s, self.p, 2), f"B_hosts[{i}]")
            _check_host_tensor(C_hosts[i], (2, self.m, self.s, self.p, 2), f"C_hosts[{i}]")
        arr = ctypes.c_void_p * max(count, 1)
        a = arr(*[_ptr(t) for t in A_hosts])
        b = arr(*[_ptr(t) for t in B_hosts])
        c = arr(*[_ptr(t) for t in C_hosts])
        _check(lib().qtp_forward_host_many(self._h, count, a, b, c, _ptr(dev_buffer),
                                           dev_buffer.numel() * dev_buffer.element_size(), _stream(stream)),
               "qtp_forward_host_many")
        return C_hosts

    def forward_saving(self, A, B, C=None, saved=None, stream=None):
        """C = A * B (qtp_forward_saving) with the spectra of A and B kept in
        `saved` (a CUDA byte tensor of workspace_size() bytes, allocated when
        None) for backward_saved.  Returns (C, saved)."""
        import torch
        _check_tensor(A, (2, self.m, self.n, self.p, 2), "A")
        _check_tensor(B, (2, self.n, self.s, self.p, 2), "B")
        if C is None:
            C = torch.empty((2, self.m, self.s, self.p, 2), dtype=torch.float32, device=A.device)
        _check_tensor(C, (2, self.m, self.s, self.p, 2), "C")
        if saved is None:
            saved = torch.empty(max(self.workspace_size(), 256), dtype=torch.uint8, device=A.device)
        _check(lib().qtp_forward_saving(self._h, _ptr(A), _ptr(B), _ptr(C), _ptr(saved),
                                        saved.numel() * saved.element_size(), _stream(stream)), "qtp_forward_saving")
        return C, saved

    def backward_saved(self, dC, saved, need_dA=True, need_dB=True, workspace=None, stream=None):
        """dA = dC * B^H, dB = A^H * dC (qtp_backward_saved) from the spectra a
        forward_saving call left in `saved`."""
        import torch
        _check_tensor(dC, (2, self.m, self.s, self.p, 2), "dC")
        dA = torch.empty((2, self.m, self.n, self.p, 2), dtype=torch.float32, device=dC.device) if need_dA else None
        dB = torch.empty((2, self.n, self.s, self.p, 2), dtype=torch.float32, device=dC.device) if need_dB else None
        need = self.backward_workspace_size()
        ws = workspace if workspace is not None else self._workspace("_bws", need, dC.device)
        _check(lib().qtp_backward_saved(self._h, _ptr(dC), _ptr(saved), saved.numel() * saved.element_size(),
                                        _ptr(dA), _ptr(dB), _ptr(ws), ws.numel() * ws.element_size(),
                                        _stream(stream)), "qtp_backward_saved")
        return dA, dB

    def backward(self, dC, A, B, need_dA=True, need_dB=True, workspace=None, stream=None):
        import torch
        _check_tensor(dC, (2, self.m, self.s, self.p, 2), "dC")
        _check_tensor(A, (2, self.m, self.n, self.p, 2), "A")
        _check_tensor(B, (2, self.n, self.s, self.p, 2), "B")
        dA = torch.empty_like(A) if need_dA else None
        dB = torch.empty_like(B) if need_dB else None
        need = self.backward_workspace_size()
        ws = workspace if workspace is not None else self._workspace("_bws", need, A.device)
        _check(lib().qtp_backward(self._h, _ptr(dC), _ptr(A), _ptr(B), _ptr(dA), _ptr(dB), _ptr(ws),
                                  ws.numel() * ws.element_size(), _stream(stream)), "qtp_backward")
        return dA, dB

    def launch_count(self):
        """(forward, backward) kernel launches per call; see qtp_plan_launch_count."""
        f, b = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().qtp_plan_launch_count(self._h, ctypes.byref(f), ctypes.byref(b)), "qtp_plan_launch_count")
        return f.value, b.value

    def tiles(self):
        """Tensor-core tile choice per product kind (forward, dA, dB); see qtp_plan_get_tiles."""
        buf = (ctypes.c_int * 3)()
        _check(lib().qtp_plan_get_tiles(self._h, buf), "qtp_plan_get_tiles")
        return [int(x) for x in buf]

    def set_tracing(self, enable: bool = True):
        _check(lib().qtp_plan_set_tracing(self._h, 1 if enable else 0), "qtp_plan_set_tracing")

    def stage_times(self):
        """Durations (ms) of Steps 1, 2, 3 of the last traced call."""
        buf = (ctypes.c_float * 3)()
        _check(lib().qtp_plan_stage_times(self._h, buf), "qtp_plan_stage_times")
        return [float(x) for x in buf]

    def sync(self, stream=None):
        _check(lib().qtp_plan_sync(self._h, _stream(stream)), "qtp_plan_sync")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().qtp_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Shape(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("s", ctypes.c_int), ("p", ctypes.c_int)]


BATCH_NO_GRAPH = 1
BATCH_AUTOTUNE = 2


class BatchPlan:
    """A qtp_batch_plan: many independent products C_i = A_i * B_i of uneven shapes."""

    def __init__(self, shapes, precision: str = "bf16x3", graph: bool = True, autotune: bool = False):
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {list(PRECISIONS)}")
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        self.precision = precision
        arr = (Shape * len(self.shapes))(*[Shape(*sh) for sh in self.shapes])
        h = ctypes.c_void_p()
        flags = (0 if graph else BATCH_NO_GRAPH) | (BATCH_AUTOTUNE if autotune else 0)
        _check(lib().qtp_batch_plan_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), len(self.shapes),
                                           PRECISIONS[precision], flags),
               "qtp_batch_plan_create")
        self._h = h
        self._ws = None

    def workspace_size(self) -> int:
        v = ctypes.c_size_t()
        _check(lib().qtp_batch_workspace_size(self._h, ctypes.byref(v)), "qtp_batch_workspace_size")
        return int(v.value)

    def forward(self, As, Bs, Cs=None, workspace=None, stream=None):
        """C_i = A_i * B_i for every product (qtp_forward_batched); returns the Cs.
        Validates and marshals every tensor on each call; for a batch whose
        tensors stay the same across calls, bind() does that once."""
        bound = self.bind(As, Bs, Cs, workspace)
        bound.forward(stream)
        return bound.Cs

    def bind(self, As, Bs, Cs=None, workspace=None):
        """Validate the batch's tensors once and keep their device pointers:
        the returned object's forward() is one qtp_forward_batched call.  It
        holds references to the tensors and the workspace, so their memory
        stays valid; their contents may change between calls."""
        import torch
        n = len(self.shapes)
        if len(As) != n or len(Bs) != n:
            raise ValueError("one A and one B per product")
        if Cs is None:
            Cs = [torch.empty((2, m, s, p, 2), dtype=torch.float32, device=As[0].device)
                  for (m, _, s, p) in self.shapes]
        if len(Cs) != n:
            raise ValueError("one C per product")
        for i, (m, k, s, p) in enumerate(self.shapes):
            _check_tensor(As[i], (2, m, k, p, 2), f"A[{i}]")
            _check_tensor(Bs[i], (2, k, s, p, 2), f"B[{i}]")
            _check_tensor(Cs[i], (2, m, s, p, 2), f"C[{i}]")
        if workspace is None:
            need = self.workspace_size()
            if self._ws is None or self._ws.numel() < need:
                self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=As[0].device)
            workspace = self._ws
        return BoundBatch(self, list(As), list(Bs), list(Cs), workspace)

    def route(self):
        """(route_min, tuned times in ms per candidate threshold) of qtp_batch_plan_route."""
        r = ctypes.c_int()
        n = ctypes.c_int()
        ms = (ctypes.c_float * 8)()
        _check(lib().qtp_batch_plan_route(self._h, ctypes.byref(r), ms, ctypes.byref(n)), "qtp_batch_plan_route")
        return int(r.value), [float(ms[i]) for i in range(n.value)]

    def set_tracing(self, enable: bool = True):
        _check(lib().qtp_batch_plan_set_tracing(self._h, 1 if enable else 0), "qtp_batch_plan_set_tracing")

    def stage_times(self):
        buf = (ctypes.c_float * 3)()
        _check(lib().qtp_batch_stage_times(self._h, buf), "qtp_batch_stage_times")
        return [float(x) for x in buf]

    def sync(self, stream=None):
        _check(lib().qtp_batch_plan_sync(self._h, _stream(stream)), "qtp_batch_plan_sync")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().qtp_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BoundBatch:
    """A batch plan with its tensors validated and their pointers marshalled
    (BatchPlan.bind)."""

    def __init__(self, plan, As, Bs, Cs, workspace):
        n = len(plan.shapes)
        self.plan, self.As, self.Bs, self.Cs, self.workspace = plan, As, Bs, Cs, workspace
        self._pa = (ctypes.c_void_p * n)(*[t.data_ptr() for t in As])
        self._pb = (ctypes.c_void_p * n)(*[t.data_ptr() for t in Bs])
        self._pc = (ctypes.c_void_p * n)(*[t.data_ptr() for t in Cs])
        self._ws_bytes = workspace.numel() * workspace.element_size()

    def forward(self, stream=None):
        _check(lib().qtp_forward_batched(self.plan._h, ctypes.cast(self._pa, ctypes.c_void_p),
                                         ctypes.cast(self._pb, ctypes.c_void_p), ctypes.cast(self._pc, ctypes.c_void_p),
                                         _ptr(self.workspace), self._ws_bytes, _stream(stream)),
               "qtp_forward_batched")
        return self.Cs


_plan_cache = {}


def plan_for(m, n, s, p, precision="bf16x3") -> Plan:
    key = (m, n, s, p, precision)
    pl = _plan_cache.get(key)
    if pl is None:
        pl = Plan(m, n, s, p, precision)
        _plan_cache[key] = pl
    return pl


def forward_noalloc(A, B, C=None, precision: str = "bf16x3", stream=None):
    """C = A * B through qtp_forward_noalloc: no plan and no workspace.

    For callers that may not allocate device memory (another allocator owns
    it, or cudaMalloc's synchronisation is unaffordable); the library keeps a
    32 MiB static device array for the scratch instead.  Only C may be
    allocated here, and only when the caller passes none.  Calls that overlap
    on the GPU share that array and race; order them.
    """
    import torch
    _, m, n, p, _ = A.shape
    s = B.shape[2]
    _check_tensor(A, (2, m, n, p, 2), "A")
    _check_tensor(B, (2, n, s, p, 2), "B")
    if C is None:
        C = torch.empty((2, m, s, p, 2), dtype=torch.float32, device=A.device)
    _check_tensor(C, (2, m, s, p, 2), "C")
    _check(lib().qtp_forward_noalloc(m, n, s, p, PRECISIONS[precision], _ptr(A), _ptr(B), _ptr(C),
                                     _stream(stream)), "qtp_forward_noalloc")
    return C


def tprod(A, B, precision: str = "bf16x3", stream=None):
    """C = A * B for CUDA tensors in plane layout (2, m, n, p, 2) and (2, n, s, p, 2)."""
    _, m, n, p, _ = A.shape
    s = B.shape[2]
    return plan_for(m, n, s, p, precision).forward(A, B, stream=stream)
