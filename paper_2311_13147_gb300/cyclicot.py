"""Thin Python binding of ``libcyclicot.so`` (declared in ``include/cyclicot.h``).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch supplies device memory (outputs, workspaces) and the
current CUDA stream.  The functions carry the C names and follow the C
argument order; outputs that the caller does not pass are allocated here as
torch tensors on the inputs' device.

There is no CPU fallback: if the library is missing or a tensor is not on a
CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcyclicot.so")

OT_OK = 0
OT_ERR_ARG = 1
OT_ERR_NOT_DIVISIBLE = 2
OT_ERR_NOT_CONVERGED = 3
OT_ERR_TIMEOUT = 4
OT_ERR_NONFINITE = 5
OT_ERR_CUDA = 6
OT_ERR_WORKSPACE = 7
OT_ERR_UNSUPPORTED = 8

OT_MIN = 0
OT_SOFTMIN = 1
OT_PLAN_LOT = 0
OT_PLAN_EROT = 1
OT_ADJ_ENVELOPE = 0
OT_ADJ_UNROLLED = 1
OT_FP32_LOG = 0
OT_BF16_KERNEL_POLISH = 1
OT_OP_SINKHORN_REDUCED = 0
OT_OP_SINKHORN_FULL = 1
OT_OP_VALUE_AND_GRAD = 2
OT_OP_UNROLLED = 3
OT_DEBUG_WITHHOLD_ARRIVAL = 1
OT_DEBUG_TRACE = 2
OT_DEBUG_NO_CLUSTER = 4
OT_DEBUG_NO_RING = 8
OT_STOP_L1_FULL = 0
OT_STOP_L2_ROW = 1

EXPORTED = ("ot_version", "ot_status_string", "ot_workspace_bytes", "ot_fold_cost", "ot_sinkhorn_reduced",
            "ot_sinkhorn_reduced_static", "ot_sinkhorn_full", "ot_unfold_plan", "ot_value_and_grad")


class OTError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (code {code})")


class ot_options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("tol_l1", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("check_every", ctypes.c_int), ("precision", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("timeout_ns", ctypes.c_ulonglong), ("tile_override", ctypes.c_int),
                ("debug_flags", ctypes.c_int), ("stop_norm", ctypes.c_int)]


class ot_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("marg_l1", ctypes.c_double),
                ("marg_l2_col", ctypes.c_double), ("value", ctypes.c_double),
                ("transport_cost", ctypes.c_double), ("marg_l1_col", ctypes.c_double),
                ("reserved", ctypes.c_double * 2)]


assert ctypes.sizeof(ot_result) == 64

_lib = None
_vp = ctypes.c_void_p


def lib():
    """Load the library once (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with paper_2311_13147_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    L.ot_version.restype = ctypes.c_char_p
    L.ot_status_string.restype = ctypes.c_char_p
    L.ot_status_string.argtypes = [ctypes.c_int]
    L.ot_workspace_bytes.restype = ctypes.c_size_t
    L.ot_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ot_options)]
    L.ot_fold_cost.restype = ctypes.c_int
    L.ot_fold_cost.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_float, _vp, _vp,
                               _vp]
    L.ot_sinkhorn_reduced.restype = ctypes.c_int
    L.ot_sinkhorn_reduced.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(ot_options), _vp,
                                      _vp, _vp, _vp, ctypes.c_size_t, _vp]
    L.ot_sinkhorn_reduced_static.restype = ctypes.c_int
    L.ot_sinkhorn_reduced_static.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(ot_options),
                                             _vp, _vp, _vp, _vp]
    L.ot_sinkhorn_full.restype = ctypes.c_int
    L.ot_sinkhorn_full.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ot_options), _vp, _vp,
                                   _vp, _vp, ctypes.c_size_t, _vp]
    L.ot_unfold_plan.restype = ctypes.c_int
    L.ot_unfold_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                                 ctypes.c_float, ctypes.c_int, _vp, _vp]
    L.ot_value_and_grad.restype = ctypes.c_int
    L.ot_value_and_grad.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                    ctypes.c_float, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                    ctypes.c_size_t, _vp]
    _lib = L
    return L


def status_string(code: int) -> str:
    try:
        return lib().ot_status_string(int(code)).decode()
    except Exception:  # library missing: still give a readable message
        return f"status {code}"


def version() -> str:
    return lib().ot_version().decode()


# ------------------------------------------------------------------ marshalling helpers

def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("cyclicot takes CUDA tensors only (no CPU path)")
    if not t.is_contiguous():
        raise ValueError("cyclicot takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(code: int, where: str):
    if code != OT_OK:
        raise OTError(code, where)


def options(eps: float, tol: float = 1e-6, max_iter: int = 10000, check_every: int = 1,
            warm_start: bool = False, timeout_ns: int = 0, precision: int = OT_FP32_LOG,
            tile_override: int = 0, debug_flags: int = 0, stop_norm: int = 0) -> ot_options:
    return ot_options(float(eps), float(tol), int(max_iter), int(check_every), int(precision),
                      int(bool(warm_start)), int(timeout_ns), int(tile_override), int(debug_flags),
                      int(stop_norm))


def new_result(device) -> torch.Tensor:
    """A device-side ot_result record (64 bytes)."""
    return torch.zeros(64, dtype=torch.uint8, device=device)


def read_result(res: torch.Tensor) -> dict:
    """Copy an ot_result record to the host (synchronises its stream)."""
    raw = bytes(res.cpu().numpy().tobytes())
    r = ot_result.from_buffer_copy(raw)
    return {"iters": r.iters, "status": r.status, "marg_l1": r.marg_l1, "marg_l2_col": r.marg_l2_col,
            "value": r.value, "transport_cost": r.transport_cost, "marg_l1_col": r.marg_l1_col,
            "mass": r.reserved[0],
            "variant": {1.0: "bulk", 2.0: "fused", 3.0: "twopass", 4.0: "stream", 5.0: "srot", 6.0: "lot",
                        7.0: "ring"}.get(r.reserved[1], "other")}


def ot_workspace_bytes(op: int, m_or_n: int, N: int, opt: Optional[ot_options] = None) -> int:
    return int(lib().ot_workspace_bytes(int(op), int(m_or_n), int(N),
                                        ctypes.byref(opt) if opt is not None else None))


def workspace(op: int, m_or_n: int, N: int, device, opt: Optional[ot_options] = None) -> torch.Tensor:
    nbytes = ot_workspace_bytes(op, m_or_n, N, opt)
    if nbytes <= 0:
        raise OTError(OT_ERR_ARG, "ot_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


# ------------------------------------------------------------------ entry points

def ot_fold_cost(mode: int, m: int, N: int, C_base=None, x=None, y=None, eps: float = 0.0,
                 G=None, kstar=None, stream=None):
    dev = (C_base if C_base is not None else x).device
    if G is None:
        G = torch.empty((m, m), dtype=torch.float32, device=dev)
    if mode == OT_MIN and kstar is None:
        kstar = torch.empty((m, m), dtype=torch.uint8, device=dev)
    code = lib().ot_fold_cost(int(mode), int(m), int(N), _ptr(C_base), _ptr(x), _ptr(y), float(eps), _ptr(G),
                              _ptr(kstar), _stream(stream))
    _check(code, "ot_fold_cost")
    return G, kstar


def ot_sinkhorn_reduced(m: int, N: int, a_base, b_base, G, opt: ot_options, w=None, z=None, out=None,
                        ws=None, stream=None):
    dev = G.device
    w = torch.empty(m, dtype=torch.float64, device=dev) if w is None else w
    z = torch.zeros(m, dtype=torch.float64, device=dev) if z is None else z
    out = new_result(dev) if out is None else out
    ws = workspace(OT_OP_SINKHORN_REDUCED, m, N, dev, opt) if ws is None else ws
    code = lib().ot_sinkhorn_reduced(int(m), int(N), _ptr(a_base), _ptr(b_base), _ptr(G), ctypes.byref(opt),
                                     _ptr(w), _ptr(z), _ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "ot_sinkhorn_reduced")
    return w, z, out


def ot_sinkhorn_reduced_static(m: int, N: int, a_base, b_base, G, opt: ot_options, w=None, z=None, out=None,
                               stream=None):
    """ot_sinkhorn_reduced with the library's own scratch array instead of a workspace.

    For callers that cannot allocate device memory at the call site (the
    outputs here are allocated only when not passed).  The scratch is shared
    by all calls on a device: calls that overlap on the GPU race.
    """
    dev = G.device
    w = torch.empty(m, dtype=torch.float64, device=dev) if w is None else w
    z = torch.zeros(m, dtype=torch.float64, device=dev) if z is None else z
    out = new_result(dev) if out is None else out
    code = lib().ot_sinkhorn_reduced_static(int(m), int(N), _ptr(a_base), _ptr(b_base), _ptr(G), ctypes.byref(opt),
                                            _ptr(w), _ptr(z), _ptr(out), _stream(stream))
    _check(code, "ot_sinkhorn_reduced_static")
    return w, z, out


def ot_sinkhorn_full(n: int, a, b, C=None, X=None, Y=None, opt: ot_options = None, f=None, g=None, out=None,
                     ws=None, stream=None):
    dev = a.device
    f = torch.empty(n, dtype=torch.float64, device=dev) if f is None else f
    g = torch.zeros(n, dtype=torch.float64, device=dev) if g is None else g
    out = new_result(dev) if out is None else out
    ws = workspace(OT_OP_SINKHORN_FULL, n, 1, dev, opt) if ws is None else ws
    code = lib().ot_sinkhorn_full(int(n), _ptr(a), _ptr(b), _ptr(C), _ptr(X), _ptr(Y), ctypes.byref(opt), _ptr(f),
                                  _ptr(g), _ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "ot_sinkhorn_full")
    return f, g, out


def ot_unfold_plan(mode: int, m: int, N: int, S_or_w, z=None, C_base=None, x=None, y=None, kstar=None,
                   eps: float = 0.0, dense: bool = False, T=None, stream=None):
    dev = S_or_w.device
    if T is None:
        shape = (N * m, N * m) if dense else (N, m, m)
        T = torch.empty(shape, dtype=torch.float32, device=dev)
    code = lib().ot_unfold_plan(int(mode), int(m), int(N), _ptr(S_or_w), _ptr(z), _ptr(C_base), _ptr(x), _ptr(y),
                                _ptr(kstar), float(eps), int(bool(dense)), _ptr(T), _stream(stream))
    _check(code, "ot_unfold_plan")
    return T


def ot_value_and_grad(m: int, N: int, a_base, b_base, C_base=None, x=None, y=None, G=None, w=None, z=None,
                      eps: float = 0.0, adjoint: int = OT_ADJ_ENVELOPE, unroll_iters: int = 0, out=None,
                      d_a=None, d_b=None, d_C=None, d_x=None, d_y=None, ws=None, stream=None):
    dev = a_base.device
    out = new_result(dev) if out is None else out
    if ws is None:
        if adjoint == OT_ADJ_UNROLLED:
            ws = workspace(OT_OP_UNROLLED, m, N, dev, options(eps, max_iter=unroll_iters))
        else:
            ws = workspace(OT_OP_VALUE_AND_GRAD, m, N, dev)
    code = lib().ot_value_and_grad(int(m), int(N), _ptr(a_base), _ptr(b_base), _ptr(C_base), _ptr(x), _ptr(y),
                                   _ptr(G), _ptr(w), _ptr(z), float(eps), int(adjoint), int(unroll_iters),
                                   _ptr(out), _ptr(d_a), _ptr(d_b), _ptr(d_C), _ptr(d_x), _ptr(d_y), _ptr(ws),
                                   ws.numel(), _stream(stream))
    _check(code, "ot_value_and_grad")
    return out


# ------------------------------------------------------------------ convenience pipeline

@dataclass
class ReducedSolution:
    w: torch.Tensor          # [m] float64, potentials for marginals of mass 1/N
    z: torch.Tensor
    G: torch.Tensor          # [m, m] folded cost
    result: dict


def cyclic_erot(a_base, b_base, eps: float, C_base=None, x=None, y=None, tol: float = 1e-6,
                max_iter: int = 10000, check: bool = True) -> ReducedSolution:
    """Fold (Eq. def_Kij) + cyclic Sinkhorn (Algorithm 2) through the C ABI."""
    src = C_base if C_base is not None else x
    N = C_base.shape[0] if C_base is not None else None
    m = a_base.shape[0]
    if N is None:
        raise ValueError("pass N through C_base or use ot_fold_cost directly for points")
    G, _ = ot_fold_cost(OT_SOFTMIN, m, N, C_base=C_base, x=x, y=y, eps=eps)
    opt = options(eps, tol=tol, max_iter=max_iter)
    w, z, out = ot_sinkhorn_reduced(m, N, a_base, b_base, G, opt)
    res = read_result(out)
    if check and res["status"] not in (OT_OK,):
        raise OTError(res["status"], "ot_sinkhorn_reduced")
    del src
    return ReducedSolution(w=w, z=z, G=G, result=res)


def read_trace(ws: torch.Tensor) -> "np.ndarray":
    """Per-sweep phase timestamps (ns) written with debug_flags & OT_DEBUG_TRACE.

    The trace occupies the last 16 KB of a solver workspace: 256 sweeps x 8
    uint64 slots ([0] sweep start, [1] row phase done, [2] after the first
    grid barrier, [3] column phase done).  Rows never written are zero.
    """
    import numpy as np
    torch.cuda.synchronize()
    raw = ws[-256 * 8 * 8:].cpu().numpy().tobytes()
    return np.frombuffer(raw, dtype=np.uint64).reshape(256, 8).astype(np.int64)


# ------------------------------------------------------------------ batches

class ot_problem_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("N", ctypes.c_int), ("eps", ctypes.c_float), ("ld", ctypes.c_int),
                ("g_off", ctypes.c_longlong), ("v_off", ctypes.c_longlong), ("x_off", ctypes.c_longlong),
                ("y_off", ctypes.c_longlong)]


assert ctypes.sizeof(ot_problem_desc) == 48


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        L.ot_batch_workspace_bytes.restype = ctypes.c_size_t
        L.ot_batch_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_longlong]
        L.ot_batch_prepare.restype = ctypes.c_int
        L.ot_batch_prepare.argtypes = [ctypes.POINTER(ot_problem_desc), ctypes.c_int, _vp, ctypes.c_size_t, _vp]
        L.ot_batch_fold.restype = ctypes.c_int
        L.ot_batch_fold.argtypes = [ctypes.c_int, _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L.ot_batch_solve.restype = ctypes.c_int
        L.ot_batch_solve.argtypes = [ctypes.c_int, ctypes.c_longlong, _vp, _vp, _vp, ctypes.POINTER(ot_options),
                                     _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L.ot_batch_autotune.restype = ctypes.c_int
        L.ot_batch_autotune.argtypes = [ctypes.c_int, ctypes.c_longlong, _vp, _vp, _vp, ctypes.POINTER(ot_options),
                                        _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_float)]
        L._batch_ready = True
    return L


def ot_batch_workspace_bytes(count: int, total_m: int) -> int:
    return int(_batch_lib().ot_batch_workspace_bytes(int(count), int(total_m)))


def ot_batch_prepare(descs, workspace_t, stream=None):
    arr = (ot_problem_desc * len(descs))(*descs)
    code = _batch_lib().ot_batch_prepare(arr, len(descs), _ptr(workspace_t), workspace_t.numel(), _stream(stream))
    _check(code, "ot_batch_prepare")


def ot_batch_fold(count: int, points, G_all, workspace_t, stream=None):
    code = _batch_lib().ot_batch_fold(int(count), _ptr(points), _ptr(G_all), _ptr(workspace_t), workspace_t.numel(),
                                      _stream(stream))
    _check(code, "ot_batch_fold")


def ot_batch_solve(count: int, total_m: int, G_all, a_all, b_all, opt: ot_options, w_all, z_all, results,
                   workspace_t, stream=None):
    code = _batch_lib().ot_batch_solve(int(count), int(total_m), _ptr(G_all), _ptr(a_all), _ptr(b_all),
                                       ctypes.byref(opt), _ptr(w_all), _ptr(z_all), _ptr(results),
                                       _ptr(workspace_t), workspace_t.numel(), _stream(stream))
    _check(code, "ot_batch_solve")


def read_results(res: torch.Tensor, count: int):
    raw = bytes(res.cpu().numpy().tobytes())
    out = []
    for p in range(count):
        r = ot_result.from_buffer_copy(raw[64 * p:64 * (p + 1)])
        out.append({"iters": r.iters, "status": r.status, "marg_l1": r.marg_l1})
    return out


def ot_batch_autotune(count: int, total_m: int, G_all, a_all, b_all, opt: ot_options, w_all, z_all, results,
                      workspace_t, stream=None):
    """Returns (configuration code, measured candidate times in ms)."""
    code = ctypes.c_int(0)
    ms = (ctypes.c_float * 5)()
    rc = _batch_lib().ot_batch_autotune(int(count), int(total_m), _ptr(G_all), _ptr(a_all), _ptr(b_all),
                                        ctypes.byref(opt), _ptr(w_all), _ptr(z_all), _ptr(results),
                                        _ptr(workspace_t), workspace_t.numel(), _stream(stream), ctypes.byref(code), ms)
    _check(rc, "ot_batch_autotune")
    return code.value, list(ms)


# ------------------------------------------------------------------ kernel domain (BF16, tensor cores)

def _kd_lib():
    L = lib()
    if not getattr(L, "_kd_ready", False):
        L.ot_kdomain_workspace_bytes.restype = ctypes.c_size_t
        L.ot_kdomain_workspace_bytes.argtypes = [ctypes.c_int]
        L.ot_kdomain_solve.restype = ctypes.c_int
        L.ot_kdomain_solve.argtypes = [ctypes.c_int, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_int, _vp, _vp,
                                       ctypes.c_int, _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L.ot_kdomain_status.restype = ctypes.c_int
        L.ot_kdomain_status.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp]
        L.ot_kdomain_product.restype = ctypes.c_int
        L.ot_kdomain_product.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L._kd_ready = True
    return L


def ot_kdomain_workspace_bytes(m: int) -> int:
    return int(_kd_lib().ot_kdomain_workspace_bytes(int(m)))


def ot_kdomain_solve(m: int, G, ld: int, eps: float, a_hist, b_hist, iters: int, z_out=None, row_err=None,
                     workspace_t=None, stream=None):
    nrhs = a_hist.shape[0]
    dev = G.device
    if z_out is None:
        z_out = torch.empty((nrhs, m), dtype=torch.float64, device=dev)
    if workspace_t is None:
        workspace_t = torch.empty(ot_kdomain_workspace_bytes(m), dtype=torch.uint8, device=dev)
    rc = _kd_lib().ot_kdomain_solve(int(m), _ptr(G), int(ld), float(eps), int(nrhs), _ptr(a_hist), _ptr(b_hist),
                                    int(iters), _ptr(z_out), _ptr(row_err) if row_err is not None else None,
                                    _ptr(workspace_t), workspace_t.numel(), _stream(stream))
    _check(rc, "ot_kdomain_solve")
    return z_out, workspace_t


def ot_kdomain_status(workspace_t, m: int, stream=None) -> int:
    st = ctypes.c_int(0)
    _check(_kd_lib().ot_kdomain_status(_ptr(workspace_t), int(m), ctypes.byref(st), _stream(stream)),
           "ot_kdomain_status")
    return st.value


def ot_kdomain_product(mp: int, A, X, Dt, workspace_t=None, stream=None):
    if workspace_t is None:
        workspace_t = torch.empty(max(ot_kdomain_workspace_bytes(mp), 256), dtype=torch.uint8, device=Dt.device)
    _check(_kd_lib().ot_kdomain_product(int(mp), _ptr(A), _ptr(X), _ptr(Dt), _ptr(workspace_t), workspace_t.numel(),
                                        _stream(stream)), "ot_kdomain_product")


# ------------------------------------------------------------------ Algorithm 3 helpers

def _ts_lib():
    L = lib()
    if not getattr(L, "_ts_ready", False):
        L.ot_first_block_row.restype = ctypes.c_int
        L.ot_first_block_row.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
        L.ot_block_average.restype = ctypes.c_int
        L.ot_block_average.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
        L.ot_tile_potentials.restype = ctypes.c_int
        L.ot_tile_potentials.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
        L._ts_ready = True
    return L


def ot_first_block_row(m: int, N: int, C, C_base=None, stream=None):
    if C_base is None:
        C_base = torch.empty((N, m, m), dtype=torch.float32, device=C.device)
    _check(_ts_lib().ot_first_block_row(int(m), int(N), _ptr(C), _ptr(C_base), _stream(stream)), "ot_first_block_row")
    return C_base


def ot_block_average(m: int, N: int, v, out=None, stream=None):
    if out is None:
        out = torch.empty(m, dtype=torch.float32, device=v.device)
    _check(_ts_lib().ot_block_average(int(m), int(N), _ptr(v), _ptr(out), _stream(stream)), "ot_block_average")
    return out


def ot_tile_potentials(m: int, N: int, z, g=None, stream=None):
    if g is None:
        g = torch.empty(m * N, dtype=torch.float64, device=z.device)
    _check(_ts_lib().ot_tile_potentials(int(m), int(N), _ptr(z), _ptr(g), _stream(stream)), "ot_tile_potentials")
    return g


def two_stage(n: int, N: int, a, b, C, eps: float, stage1_l2: float = 1e-3, tol: float = 1e-6,
              max_iter: int = 100000, stream=None):
    """Algorithm 3 through the C ABI (every step in the library's kernels).

    Returns (f, g, stage-1 result, stage-2 result); f, g are the full problem's
    potentials (unit-mass convention of ot_sinkhorn_full).
    """
    m = n // N
    C_base = ot_first_block_row(m, N, C, stream=stream)
    alpha = ot_block_average(m, N, a, stream=stream)
    beta = ot_block_average(m, N, b, stream=stream)
    G, _ = ot_fold_cost(OT_SOFTMIN, m, N, C_base=C_base, eps=eps, stream=stream)
    o1 = options(eps, tol=stage1_l2, max_iter=max_iter, stop_norm=OT_STOP_L2_ROW)
    w1, z1, r1 = ot_sinkhorn_reduced(m, N, alpha, beta, G, o1, stream=stream)
    g0 = ot_tile_potentials(m, N, z1, stream=stream)
    o2 = options(eps, tol=tol, max_iter=max_iter, warm_start=True)
    f, g, r2 = ot_sinkhorn_full(n, a, b, C=C, opt=o2, g=g0, stream=stream)
    return f, g, read_result(r1), read_result(r2)


# ------------------------------------------------------------------ C-SROT (squared-L2 regulariser)

def _srot_lib():
    L = lib()
    if not getattr(L, "_srot_ready", False):
        L.ot_srot_workspace_bytes.restype = ctypes.c_size_t
        L.ot_srot_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
        L.ot_srot_reduced.restype = ctypes.c_int
        L.ot_srot_reduced.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(ot_options), _vp,
                                      _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L._srot_ready = True
    return L


def srot_workspace(m: int, N: int, device) -> torch.Tensor:
    nbytes = _srot_lib().ot_srot_workspace_bytes(int(m), int(N))
    if nbytes == 0:
        raise OTError(OT_ERR_UNSUPPORTED, "ot_srot_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def ot_srot_reduced(m: int, N: int, a_base, b_base, C_base, lam: float, tol: float = 1e-6, max_iter: int = 100000,
                    w=None, z=None, out=None, ws=None, warm_start: bool = False, stream=None):
    """C-SROT with phi(x) = (lam/2) x^2 (Sec. 5.3): alternating minimisation of the reduced dual.

    Returns (w, z, out): FP64 dual potentials of the mass-1/N problem and the result record
    (value and transport cost at full scale).  N = 1 solves the plain full problem.
    """
    dev = C_base.device
    w = torch.empty(m, dtype=torch.float64, device=dev) if w is None else w
    z = torch.zeros(m, dtype=torch.float64, device=dev) if z is None else z
    out = new_result(dev) if out is None else out
    ws = srot_workspace(m, N, dev) if ws is None else ws
    opt = options(lam, tol=tol, max_iter=max_iter, warm_start=warm_start)
    code = _srot_lib().ot_srot_reduced(int(m), int(N), _ptr(a_base), _ptr(b_base), _ptr(C_base), ctypes.byref(opt),
                                       _ptr(w), _ptr(z), _ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "ot_srot_reduced")
    return w, z, out


def _lot_lib():
    L = lib()
    if not getattr(L, "_lot_ready", False):
        L.ot_lot_workspace_bytes.restype = ctypes.c_size_t
        L.ot_lot_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
        L.ot_lot_reduced.restype = ctypes.c_int
        L.ot_lot_reduced.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp,
                                     ctypes.POINTER(ot_options), _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
        L._lot_ready = True
    return L


def lot_workspace(count: int, m: int, device) -> torch.Tensor:
    nbytes = _lot_lib().ot_lot_workspace_bytes(int(count), int(m))
    if nbytes == 0:
        raise OTError(OT_ERR_UNSUPPORTED, "ot_lot_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def ot_lot_reduced(m: int, N: int, a_base, b_base, G, count: int = 1, max_pivots: Optional[int] = None,
                   S=None, u=None, v=None, out=None, ws=None, stream=None, single_cta: bool = False,
                   debug_flags: int = 0, timeout_ns: int = 0):
    """Small LOT of Theorem 1 by the network simplex: S [count][m][m] FP32, duals u, v [count][m] FP64.

    a_base, b_base: [count][m] (or [m] when count = 1); G: [count][m][m] (or [m][m]), the min-fold.
    single_cta: one thread block per instance even where a cluster of them would fit.
    debug_flags, timeout_ns: as in ot_options (failure-detection tests).
    Returns (S, u, v, out) with out a [count] result buffer (value = <G, S>, reserved[0] = dual value).
    """
    dev = G.device
    S = torch.empty((count, m, m), dtype=torch.float32, device=dev) if S is None else S
    u = torch.empty((count, m), dtype=torch.float64, device=dev) if u is None else u
    v = torch.empty((count, m), dtype=torch.float64, device=dev) if v is None else v
    if out is None:
        out = torch.zeros((count, ctypes.sizeof(ot_result)), dtype=torch.uint8, device=dev)
    ws = lot_workspace(count, m, dev) if ws is None else ws
    opt = options(1.0, max_iter=int(max_pivots if max_pivots is not None else 100 * m + 10000),
                  debug_flags=(OT_DEBUG_NO_CLUSTER if single_cta else 0) | int(debug_flags), timeout_ns=int(timeout_ns))
    code = _lot_lib().ot_lot_reduced(int(count), int(m), int(N), _ptr(a_base), _ptr(b_base), _ptr(G),
                                     ctypes.byref(opt), _ptr(S), _ptr(u), _ptr(v), _ptr(out), _ptr(ws), ws.numel(),
                                     _stream(stream))
    _check(code, "ot_lot_reduced")
    return S, u, v, out


def read_lot_results(res: torch.Tensor, count: int):
    """Host copies of the [count] records written by ot_lot_reduced."""
    raw = bytes(res.cpu().numpy().tobytes())
    out = []
    for p in range(count):
        r = ot_result.from_buffer_copy(raw[64 * p:64 * (p + 1)])
        out.append({"pivots": r.iters, "status": r.status, "value": r.value, "dual": r.reserved[0],
                    "marg_l1": r.marg_l1, "marg_l1_col": r.marg_l1_col, "marg_l2_col": r.marg_l2_col,
                    "variant": "lot" if r.reserved[1] == 6.0 else "other"})
    return out
