"""ctypes binding of libkmeans_aa (include/kmeans_aa.h): argument marshalling only.

Every function has the name of the C entry point it calls and takes torch tensors (device
tensors, or host tensors / numpy arrays for ``kmeans_solve_host``).  Every step of the path runs
in the CUDA library; there is no CPU fallback: if the library cannot be loaded, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

KM_OK, KM_EINVAL, KM_ENOMEM, KM_ECUDA, KM_ETIMEOUT, KM_ENONFINITE, KM_EBUSY = range(7)
KM_F64, KM_F32, KM_BF16_F32 = 0, 1, 2

_STATUS = {0: "KM_OK", 1: "KM_EINVAL", 2: "KM_ENOMEM", 3: "KM_ECUDA", 4: "KM_ETIMEOUT",
           5: "KM_ENONFINITE", 6: "KM_EBUSY"}


class KmeansError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class kmeans_data(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("X_bf16", ctypes.c_void_p), ("N", ctypes.c_int64),
                ("d", ctypes.c_int32), ("prec", ctypes.c_int32), ("X_bf16_lo", ctypes.c_void_p)]


class kmeans_params(ctypes.Structure):
    _fields_ = [("m_max", ctypes.c_int32), ("m_init", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("lloyd_only", ctypes.c_int32), ("eps1", ctypes.c_double), ("eps2", ctypes.c_double),
                ("tol", ctypes.c_double), ("rank_tol", ctypes.c_double), ("fixed_m", ctypes.c_int32)]


class kmeans_problem(ctypes.Structure):
    _fields_ = [("X", kmeans_data), ("K", ctypes.c_int32), ("C0", ctypes.c_void_p), ("C_out", ctypes.c_void_p),
                ("rho_out", ctypes.c_void_p)]


class kmeans_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("accepted", ctypes.c_int32), ("rejected", ctypes.c_int32),
                ("assign_passes", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("m_final", ctypes.c_int32), ("E", ctypes.c_double), ("rescored_rows", ctypes.c_int64),
                ("device_ms", ctypes.c_double), ("status", ctypes.c_int32), ("ls_qr_solves", ctypes.c_int32),
                ("scanned_rows", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class kmeans_state(ctypes.Structure):
    _fields_ = [("C", ctypes.c_void_p), ("C_AU", ctypes.c_void_p), ("F", ctypes.c_void_p), ("dF", ctypes.c_void_p),
                ("dG", ctypes.c_void_p), ("rho", ctypes.c_void_p),
                ("t", ctypes.c_int32), ("m", ctypes.c_int32), ("m_t", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("from_lloyd", ctypes.c_int32), ("ring_count", ctypes.c_int32), ("done", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("accepted", ctypes.c_int32), ("rejected", ctypes.c_int32),
                ("passes", ctypes.c_int32), ("ls_qr_solves", ctypes.c_int32), ("E_prev", ctypes.c_double),
                ("E_prev2", ctypes.c_double), ("E_trial", ctypes.c_double), ("theta", ctypes.c_double * 32)]


class kmeans_server_stats(ctypes.Structure):
    _fields_ = [("waiting", ctypes.c_int32), ("active_small", ctypes.c_int32), ("active_large", ctypes.c_int32),
                ("completed", ctypes.c_int32), ("steps", ctypes.c_int64), ("pool_bytes", ctypes.c_size_t),
                ("pool_used", ctypes.c_size_t), ("pool_peak", ctypes.c_size_t)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libkmeans_aa.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libkmeans_aa.so not found at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    L.kmeans_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t, vp]
    L.kmeans_destroy.argtypes = [vp]
    L.kmeans_set_stream.argtypes = [vp, vp]
    L.kmeans_workspace_bytes.argtypes = [vp]
    L.kmeans_workspace_bytes.restype = ctypes.c_size_t
    L.kmeans_status_string.argtypes = [ctypes.c_int]
    L.kmeans_status_string.restype = ctypes.c_char_p
    L.kmeans_last_error.argtypes = [vp]
    L.kmeans_last_error.restype = ctypes.c_char_p
    L.kmeans_default_params.argtypes = [ctypes.POINTER(kmeans_params)]
    L.kmeans_default_params.restype = None
    pd = ctypes.POINTER(kmeans_data)
    L.kmeans_assign.argtypes = [vp, pd, vp, i32, vp, vp, vp, vp]
    L.kmeans_update.argtypes = [vp, pd, vp, i32, vp, vp, vp]
    L.kmeans_energy.argtypes = [vp, pd, vp, i32, vp, dp]
    L.kmeans_seed_pp.argtypes = [vp, pd, i32, ctypes.POINTER(ctypes.c_double), vp, vp]
    L.kmeans_solve.argtypes = [vp, pd, i32, vp, ctypes.POINTER(kmeans_params), vp, vp,
                               ctypes.POINTER(kmeans_info)]
    L.kmeans_solve_host.argtypes = [vp, pd, i32, vp, ctypes.POINTER(kmeans_params), vp, vp,
                                    ctypes.POINTER(kmeans_info)]
    L.kmeans_update_static.argtypes = [pd, vp, i32, vp, vp, vp, vp]
    L.kmeans_lsq.argtypes = [vp, vp, i64, i32, vp, ctypes.c_double, i32, vp, vp, vp]
    L.kmeans_measure_fp32_fma.argtypes = [ctypes.c_int, i32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
    L.kmeans_solve_passes.argtypes = [vp, pd, i32, vp, ctypes.POINTER(kmeans_params), i32,
                                      ctypes.POINTER(kmeans_state)]
    L.kmeans_solve_batched.argtypes = [vp, ctypes.POINTER(kmeans_problem), i32, ctypes.POINTER(kmeans_params),
                                       ctypes.POINTER(kmeans_info)]
    L.kmeans_batch_describe.argtypes = [vp]
    L.kmeans_batch_describe.restype = ctypes.c_char_p
    L.kmeans_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t, i32, i32]
    L.kmeans_server_destroy.argtypes = [vp]
    L.kmeans_server_submit.argtypes = [vp, pd, i32, vp, ctypes.POINTER(kmeans_params), vp, vp,
                                       ctypes.POINTER(i64)]
    L.kmeans_server_step.argtypes = [vp, ctypes.POINTER(i32)]
    L.kmeans_server_poll.argtypes = [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(kmeans_info)]
    L.kmeans_server_get_stats.argtypes = [vp, ctypes.POINTER(kmeans_server_stats)]
    L.kmeans_server_last_error.argtypes = [vp]
    L.kmeans_server_last_error.restype = ctypes.c_char_p
    for name in ("kmeans_create", "kmeans_destroy", "kmeans_set_stream", "kmeans_assign",
                 "kmeans_update", "kmeans_energy", "kmeans_solve", "kmeans_solve_host",
                 "kmeans_update_static", "kmeans_lsq", "kmeans_solve_passes", "kmeans_measure_fp32_fma",
                 "kmeans_solve_batched", "kmeans_server_create",
                 "kmeans_server_destroy", "kmeans_server_submit", "kmeans_server_step",
                 "kmeans_server_poll", "kmeans_server_get_stats"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(ctx, status: int):
    if status != KM_OK:
        msg = load().kmeans_last_error(ctx.handle if ctx is not None else None)
        raise KmeansError(status, msg.decode() if msg else "")


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _prec_of(X, X_bf16=None) -> int:
    dt = X.dtype
    if dt in (torch.float64, np.float64):
        return KM_F64
    if dt in (torch.float32, np.float32):
        return KM_BF16_F32 if X_bf16 is not None else KM_F32
    raise TypeError(f"X must be float64 or float32, got {dt}")


def make_data(X, X_bf16=None, X_lo=None) -> kmeans_data:
    """X_bf16: the BF16 rounding of X (tensor-core path); X_lo: optional BF16 rounding of X - X_bf16."""
    assert X.ndim == 2 and (X.is_contiguous() if torch.is_tensor(X) else X.flags.c_contiguous)
    return kmeans_data(_ptr(X), _ptr(X_bf16), X.shape[0], X.shape[1], _prec_of(X, X_bf16), _ptr(X_lo))


def default_params(**kw) -> kmeans_params:
    p = kmeans_params()
    load().kmeans_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Context:
    """A kmeans_ctx bound to a device and a CUDA stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, stream=None):
        L = load()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        st = L.kmeans_create(ctypes.byref(h), device, hbm_budget, ctypes.c_void_p(stream))
        if st != KM_OK:
            raise KmeansError(st, "kmeans_create failed")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            load().kmeans_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self) -> int:
        return int(load().kmeans_workspace_bytes(self.handle))


def kmeans_assign(ctx: Context, X, C, rho=None, rho_prev=None, n_changed=None, dmin=None, X_bf16=None, X_lo=None):
    """Eq. 3 on the device; returns rho (int32 [N])."""
    N = X.shape[0]
    if rho is None:
        rho = torch.empty(N, dtype=torch.int32, device=X.device)
    data = make_data(X, X_bf16, X_lo)
    _check(ctx, load().kmeans_assign(ctx.handle, ctypes.byref(data), _ptr(C), C.shape[0], _ptr(rho),
                                     _ptr(rho_prev), _ptr(n_changed), _ptr(dmin)))
    return rho


def kmeans_update(ctx: Context, X, rho, K: int, C_prev, C_out=None, counts=None):
    """Eq. 4 on the device; returns (C_out, counts)."""
    if C_out is None:
        C_out = torch.empty_like(C_prev)
    if counts is None:
        counts = torch.empty(K, dtype=torch.int64, device=X.device)
    data = make_data(X)
    _check(ctx, load().kmeans_update(ctx.handle, ctypes.byref(data), _ptr(rho), K, _ptr(C_prev), _ptr(C_out),
                                     _ptr(counts)))
    return C_out, counts


def kmeans_update_static(X, rho, K: int, C_prev, C_out=None, counts=None, stream=None):
    """kmeans_update without allocation (no context; scratch in a fixed device array).

    For callers that must not allocate device memory: pass C_out and counts, otherwise this
    wrapper allocates them with torch before the call.  Runs on X's device (made current for the
    call) and on `stream` (default: torch's current stream of that device); returns (C_out, counts).
    """
    dev = X.device
    for name, t in (("rho", rho), ("C_prev", C_prev), ("C_out", C_out), ("counts", counts)):
        if t is not None and t.device != dev:
            raise ValueError(f"{name} is on {t.device}, X on {dev}")
    with torch.cuda.device(dev):
        if C_out is None:
            C_out = torch.empty_like(C_prev)
        if counts is None:
            counts = torch.empty(K, dtype=torch.int64, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        data = make_data(X)
        st = load().kmeans_update_static(ctypes.byref(data), _ptr(rho), K, _ptr(C_prev), _ptr(C_out), _ptr(counts),
                                         ctypes.c_void_p(stream))
    if st != KM_OK:
        raise KmeansError(st, "kmeans_update_static failed")
    return C_out, counts


def kmeans_energy(ctx: Context, X, C, rho, E=None):
    """Eq. 1 with a given assignment; returns a device float64 scalar tensor."""
    if E is None:
        E = torch.empty((), dtype=torch.float64, device=X.device)
    data = make_data(X)
    _check(ctx, load().kmeans_energy(ctx.handle, ctypes.byref(data), _ptr(C), C.shape[0], _ptr(rho), _ptr(E)))
    return E


def kmeans_seed_pp(ctx: Context, X, K: int, u, C_out=None, idx_out=None):
    """K-Means++ seeding on the device with the uniforms u[0..K-1]; returns (C [K, d], idx [K])."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    if u.shape != (K,):
        raise ValueError("u must hold K uniforms")
    if C_out is None:
        C_out = torch.empty((K, X.shape[1]), dtype=X.dtype, device=X.device)
    if idx_out is None:
        idx_out = torch.empty(K, dtype=torch.int32, device=X.device)
    data = make_data(X)
    _check(ctx, load().kmeans_seed_pp(ctx.handle, ctypes.byref(data), K,
                                      u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(C_out),
                                      _ptr(idx_out)))
    return C_out, idx_out


def kmeans_solve(ctx: Context, X, C0, C_out=None, rho_out=None, X_bf16=None, X_lo=None, **params):
    """Lloyd (lloyd_only=1) or Algorithm 1 on the device; returns (C, rho, info dict)."""
    if C_out is None:
        C_out = torch.empty_like(C0)
    if rho_out is None:
        rho_out = torch.empty(X.shape[0], dtype=torch.int32, device=X.device)
    data = make_data(X, X_bf16, X_lo)
    p = default_params(**params)
    info = kmeans_info()
    _check(ctx, load().kmeans_solve(ctx.handle, ctypes.byref(data), C0.shape[0], _ptr(C0), ctypes.byref(p),
                                    _ptr(C_out), _ptr(rho_out), ctypes.byref(info)))
    return C_out, rho_out, info.as_dict()


def kmeans_solve_host(ctx: Context, X, C0, C_out=None, rho_out=None, X_bf16=None, **params):
    """kmeans_solve with host buffers (torch CPU tensors, ideally pinned, or numpy arrays)."""
    if C_out is None:
        C_out = torch.empty(C0.shape, dtype=C0.dtype).pin_memory() if torch.is_tensor(C0) else np.empty_like(C0)
    if rho_out is None:
        rho_out = (torch.empty(X.shape[0], dtype=torch.int32).pin_memory() if torch.is_tensor(X)
                   else np.empty(X.shape[0], np.int32))
    data = make_data(X, X_bf16)
    p = default_params(**params)
    info = kmeans_info()
    _check(ctx, load().kmeans_solve_host(ctx.handle, ctypes.byref(data), C0.shape[0], _ptr(C0),
                                         ctypes.byref(p), _ptr(C_out), _ptr(rho_out), ctypes.byref(info)))
    return C_out, rho_out, info.as_dict()


def kmeans_lsq(ctx: Context, dF, f, rank_tol: float = 1e-12, method: int = 0, theta=None):
    """Eq. 7 on the device for a caller's history.  dF: float64 device tensor [m, n] (row j = the
    difference dF_{j+1}, row 0 the newest), f: [n].  method 0 = the solver's rule, 1 = Householder
    QR, 2 = Gram matrix + Cholesky.  Returns (theta [m] device tensor, rank, qr_used)."""
    m, n = dF.shape
    if theta is None:
        theta = torch.empty(m, dtype=torch.float64, device=dF.device)
    out = torch.zeros(2, dtype=torch.int32, device=dF.device)
    _check(ctx, load().kmeans_lsq(ctx.handle, _ptr(dF), n, m, _ptr(f), float(rank_tol), int(method), _ptr(theta),
                                  out.data_ptr(), out.data_ptr() + 4))
    r = out.cpu().tolist()
    return theta, r[0], r[1]


def kmeans_solve_passes(ctx: Context, X, C0, passes: int, X_bf16=None, **params):
    """The solver stopped after `passes` loop passes; returns its state as a dict of numpy arrays
    (C, C_AU, F, dF and dG newest first, rho) and scalars (see kmeans_state in the header)."""
    K, d = C0.shape
    N = X.shape[0]
    p = default_params(**params)
    m_max = 0 if p.lloyd_only else p.m_max
    n = K * d
    bufs = dict(C=np.empty((K, d)), C_AU=np.empty((K, d)), F=np.empty((K, d)),
                dF=np.empty((max(m_max, 1), n)), dG=np.empty((max(m_max, 1), n)), rho=np.empty(N, np.int32))
    st = kmeans_state()
    for k, v in bufs.items():
        setattr(st, k, v.ctypes.data)
    data = make_data(X, X_bf16)
    _check(ctx, load().kmeans_solve_passes(ctx.handle, ctypes.byref(data), K, _ptr(C0), ctypes.byref(p), int(passes),
                                           ctypes.byref(st)))
    out = {f: getattr(st, f) for f, _ in kmeans_state._fields_ if f not in bufs and f != "theta"}
    out["theta"] = np.array(st.theta[:], np.float64)
    out.update(bufs)
    out["dF"] = bufs["dF"][:st.ring_count]
    out["dG"] = bufs["dG"][:st.ring_count]
    return out


def kmeans_solve_batched(ctx: Context, Xs, C0s, C_outs=None, rho_outs=None, params=None, check=True,
                         X_bf16s=None):
    """Solve independent instances together.

    Xs, C0s: lists of device tensors; X_bf16s: list of BF16 copies (None entries for d <= 16);
    params: one dict for all instances or a list of dicts.
    Returns (C_outs, rho_outs, infos, status).  With check=True a non-OK status raises."""
    n = len(Xs)
    if C_outs is None:
        C_outs = [torch.empty_like(c) for c in C0s]
    if rho_outs is None:
        rho_outs = [torch.empty(x.shape[0], dtype=torch.int32, device=x.device) for x in Xs]
    probs = (kmeans_problem * n)()
    for i in range(n):
        xb = X_bf16s[i] if X_bf16s is not None else None
        probs[i] = kmeans_problem(make_data(Xs[i], xb), C0s[i].shape[0], _ptr(C0s[i]), _ptr(C_outs[i]),
                                  _ptr(rho_outs[i]))
    if params is None or isinstance(params, dict):
        params = [params or {}] * n
    ps = (kmeans_params * n)(*[default_params(**q) for q in params])
    infos = (kmeans_info * n)()
    st = load().kmeans_solve_batched(ctx.handle, probs, n, ps, infos)
    if check:
        _check(ctx, st)
    return C_outs, rho_outs, [infos[i].as_dict() for i in range(n)], st


class Server:
    """kmeans_server: requests of different shapes admitted against an HBM budget and solved in a
    continuously stepping batch (low-d) or on a second stream (d > 16, BF16).

    submit() takes host arrays (numpy or CPU torch tensors; pinned memory keeps the copies
    asynchronous) and returns a ticket; step() advances the server; poll(ticket) returns
    None while pending, else (C_out, rho_out, info)."""

    def __init__(self, device: int = 0, hbm_budget: int = 1 << 30, max_slots: int = 512, max_large: int = 1):
        L = load()
        h = ctypes.c_void_p()
        st = L.kmeans_server_create(ctypes.byref(h), device, hbm_budget, max_slots, max_large)
        if st != KM_OK:
            raise KmeansError(st, "kmeans_server_create failed")
        self.handle = h
        self._keep = {}

    def _raise(self, st):
        if st != KM_OK:
            msg = load().kmeans_server_last_error(self.handle)
            raise KmeansError(st, msg.decode() if msg else "")

    def submit(self, X, C0, X_bf16=None, C_out=None, rho_out=None, **params) -> int:
        if C_out is None:
            C_out = (torch.empty(C0.shape, dtype=C0.dtype).pin_memory() if torch.is_tensor(C0)
                     else np.empty_like(C0))
        if rho_out is None:
            rho_out = (torch.empty(X.shape[0], dtype=torch.int32).pin_memory() if torch.is_tensor(X)
                       else np.empty(X.shape[0], np.int32))
        data = make_data(X, X_bf16)
        p = default_params(**params)
        t = ctypes.c_int64()
        self._raise(load().kmeans_server_submit(self.handle, ctypes.byref(data), C0.shape[0], _ptr(C0),
                                                ctypes.byref(p), _ptr(C_out), _ptr(rho_out), ctypes.byref(t)))
        self._keep[t.value] = (X, X_bf16, C0, C_out, rho_out)
        return t.value

    def step(self) -> int:
        n = ctypes.c_int32()
        self._raise(load().kmeans_server_step(self.handle, ctypes.byref(n)))
        return n.value

    def poll(self, ticket: int):
        done = ctypes.c_int32()
        info = kmeans_info()
        self._raise(load().kmeans_server_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(info)))
        if not done.value:
            return None
        _, _, _, C_out, rho_out = self._keep.pop(ticket)
        return C_out, rho_out, info.as_dict()

    def stats(self) -> dict:
        s = kmeans_server_stats()
        self._raise(load().kmeans_server_get_stats(self.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load().kmeans_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fp32_fma(device: int = 0, iters: int = 20000):
    """(FP32 FMAs per second, kernel ms) of kmeans_measure_fp32_fma."""
    r, t = ctypes.c_double(), ctypes.c_double()
    st = load().kmeans_measure_fp32_fma(device, iters, ctypes.byref(r), ctypes.byref(t))
    if st != KM_OK:
        raise KmeansError(st, "kmeans_measure_fp32_fma failed")
    return r.value, t.value


def batch_describe(ctx: Context) -> str:
    return load().kmeans_batch_describe(ctx.handle).decode()


def exported_symbols():
    """Names of the C entry points declared in include/kmeans_aa.h."""
    import re
    hdr = os.path.join(os.path.dirname(_build.PKG), "include", "kmeans_aa.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"\b(kmeans_[a-z_]+)\s*\(", txt)))
