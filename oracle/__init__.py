"""FP64 CPU oracle for Lloyd and Anderson-accelerated K-Means (test infrastructure only).

This package is the slow, obviously-correct reference the CUDA path is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it;
the CUDA library and its Python binding never do.  It wraps ``kmeans_oracle.c`` (plain C, FP64,
sequential sums) through ctypes and builds it with gcc on first use.

Every function cites the passage of "Fast K-Means Clustering with Anderson Acceleration" it
follows:

* ``assign``  - Eq. 3 (direct squared distances, lowest index on ties, top-2 gap)
* ``energy``  - Eq. 1
* ``update``  - Eq. 4 (empty cluster keeps its centroid)
* ``ls_qr``   - Eq. 7 (Householder QR, column truncation on rank loss)
* ``m_rule``  - Section 2.2 / Algorithm 1, dynamic m
* ``aa_affine`` - Eq. 7-8 on an affine map (classical Anderson, used as a textbook pin)
* ``solve``   - Lloyd (Section 1) and Algorithm 1
* ``step``    - one loop pass of Algorithm 1 from an explicit state (the body of ``solve``)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmeans_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libkmeans_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)


class _Params(ctypes.Structure):
    _fields_ = [("m_max", ctypes.c_int), ("m_init", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("lloyd_only", ctypes.c_int), ("eps1", ctypes.c_double), ("eps2", ctypes.c_double),
                ("tol", ctypes.c_double), ("rank_tol", ctypes.c_double), ("fixed_m", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("accepted", ctypes.c_int), ("rejected", ctypes.c_int),
                ("assign_passes", ctypes.c_int), ("converged", ctypes.c_int),
                ("m_final", ctypes.c_int), ("E", ctypes.c_double)]


class _Trace(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int), ("n_changed", ctypes.c_int), ("m", ctypes.c_int),
                ("m_t", ctypes.c_int), ("rank", ctypes.c_int), ("accelerated", ctypes.c_int),
                ("rejected", ctypes.c_int), ("pad", ctypes.c_int), ("E_trial", ctypes.c_double),
                ("E", ctypes.c_double), ("margin_lo", ctypes.c_double),
                ("margin_hi", ctypes.c_double), ("margin_safe", ctypes.c_double)]


class _State(ctypes.Structure):
    _fields_ = [("C", _dp), ("CAU", _dp), ("F", _dp), ("dF", _dp), ("dG", _dp), ("Pprev", _ip),
                ("count", ctypes.c_int), ("t", ctypes.c_int), ("m", ctypes.c_int), ("from_lloyd", ctypes.c_int),
                ("E_prev", ctypes.c_double), ("E_prev2", ctypes.c_double), ("done", ctypes.c_int),
                ("E", ctypes.c_double), ("accepted", ctypes.c_int), ("rejected", ctypes.c_int),
                ("assign_passes", ctypes.c_int), ("theta", ctypes.c_double * 64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP on); returns the .so path."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    lib.orc_assign.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, _dp, ctypes.c_int, _ip, _dp, _dp]
    lib.orc_assign.restype = None
    lib.orc_energy.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, _dp, _ip]
    lib.orc_energy.restype = ctypes.c_double
    lib.orc_update.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, _ip, ctypes.c_int, _dp, _dp, _lp]
    lib.orc_update.restype = None
    lib.orc_ls_qr.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, _dp, ctypes.c_double, _dp]
    lib.orc_ls_qr.restype = ctypes.c_int
    lib.orc_m_rule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.orc_m_rule.restype = ctypes.c_int
    lib.orc_aa_affine.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, _dp, _dp]
    lib.orc_aa_affine.restype = None
    lib.orc_solve.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _dp,
                              ctypes.POINTER(_Params), _dp, _ip, ctypes.POINTER(_Info),
                              ctypes.POINTER(_Trace)]
    lib.orc_solve.restype = ctypes.c_int
    lib.orc_step.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Params),
                             ctypes.POINTER(_State), ctypes.POINTER(_Trace), _ip, _dp, _dp, _dp]
    lib.orc_step.restype = ctypes.c_int
    lib.orc_kmeanspp.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _dp, _ip, _dp]
    lib.orc_kmeanspp.restype = None
    lib.orc_num_threads.argtypes = []
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_num_threads.argtypes = [ctypes.c_int]
    lib.orc_set_num_threads.restype = None
    _lib = lib
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray, typ):
    return a.ctypes.data_as(typ)


def num_threads() -> int:
    """OpenMP threads the oracle's assignment loop uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the assignment loop from now on (results do not depend on it)."""
    _load().orc_set_num_threads(int(n))


def assign(X, C):
    """Eq. 3.  Returns (rho int32[N], dmin f64[N], gap f64[N]) with lowest-index ties."""
    X, C = _f64(X), _f64(C)
    N, d = X.shape
    K = C.shape[0]
    assert C.shape[1] == d
    rho = np.empty(N, np.int32)
    dmin = np.empty(N, np.float64)
    gap = np.empty(N, np.float64)
    _load().orc_assign(_ptr(X, _dp), N, d, _ptr(C, _dp), K, _ptr(rho, _ip), _ptr(dmin, _dp),
                       _ptr(gap, _dp))
    return rho, dmin, gap


def energy(X, C, rho) -> float:
    """Eq. 1 with a given assignment: sum_i ||x_i - c_{rho_i}||^2 (sequential FP64)."""
    X, C = _f64(X), _f64(C)
    rho = np.ascontiguousarray(rho, dtype=np.int32)
    return float(_load().orc_energy(_ptr(X, _dp), X.shape[0], X.shape[1], _ptr(C, _dp),
                                    _ptr(rho, _ip)))


def update(X, rho, K: int, C_prev):
    """Eq. 4.  Returns (C f64[K,d], counts int64[K]); empty clusters keep C_prev."""
    X, C_prev = _f64(X), _f64(C_prev)
    rho = np.ascontiguousarray(rho, dtype=np.int32)
    N, d = X.shape
    C = np.empty((K, d), np.float64)
    counts = np.empty(K, np.int64)
    _load().orc_update(_ptr(X, _dp), N, d, _ptr(rho, _ip), K, _ptr(C_prev, _dp), _ptr(C, _dp),
                       _ptr(counts, _lp))
    return C, counts


def ls_qr(dF, f, rank_tol: float = 1e-12):
    """Eq. 7 by Householder QR.  dF is [n, m] (column 0 = newest difference).

    Returns (theta f64[m], rank); columns from the first with |R_kk| <= rank_tol*|R_00| on are
    dropped (theta = 0).
    """
    dF = np.asarray(dF, dtype=np.float64)
    n, m = dF.shape
    assert m <= 63
    cols = np.ascontiguousarray(dF.T)     # column-major storage: column j contiguous
    f = _f64(f)
    theta = np.zeros(m, np.float64)
    rank = _load().orc_ls_qr(_ptr(cols, _dp), n, m, _ptr(f, _dp), rank_tol, _ptr(theta, _dp))
    return theta, int(rank)


def m_rule(m: int, m_max: int, t: int, E_cur: float, E_prev: float, E_prev2: float,
           eps1: float = 0.02, eps2: float = 0.5) -> int:
    """Dynamic-m adjustment of Algorithm 1 (only for t >= 3, division-free)."""
    return int(_load().orc_m_rule(m, m_max, t, E_cur, E_prev, E_prev2, eps1, eps2))


def aa_affine(A, b, x0, m: int, iters: int, rank_tol: float = 1e-12):
    """Classical Anderson (Eq. 7-8, no safeguard) on g(x) = A x + b; returns [iters+1, n]."""
    A, b = _f64(A), _f64(b)
    n = b.shape[0]
    x = _f64(x0).copy()
    traj = np.empty((iters + 1, n), np.float64)
    _load().orc_aa_affine(_ptr(A, _dp), _ptr(b, _dp), n, m, iters, rank_tol, _ptr(x, _dp),
                          _ptr(traj, _dp))
    return traj


DEFAULT_PARAMS = dict(m_max=10, m_init=2, max_iter=1000, lloyd_only=0, eps1=0.02, eps2=0.5,
                      tol=0.0, rank_tol=1e-12, fixed_m=0)


def kmeanspp(X, K: int, u):
    """K-Means++ seeding with the given uniforms u[0..K-1]; returns (row indices, C)."""
    X = _f64(X)
    u = _f64(u)
    N, d = X.shape
    assert u.shape == (K,) and 1 <= K and N >= 1
    idx = np.empty(K, np.int32)
    C = np.empty((K, d), np.float64)
    _load().orc_kmeanspp(_ptr(X, _dp), N, d, K, _ptr(u, _dp), _ptr(idx, _ip), _ptr(C, _dp))
    return idx, C


def solve(X, C0, lloyd: bool = False, trace: bool = False, **kw):
    """Lloyd (lloyd=True) or Algorithm 1.  Returns (C, rho, info dict[, trace list])."""
    X, C0 = _f64(X), _f64(C0)
    N, d = X.shape
    K = C0.shape[0]
    prm = dict(DEFAULT_PARAMS)
    prm.update(kw)
    if lloyd:
        prm["lloyd_only"] = 1
    assert 0 <= prm["m_max"] <= 63
    p = _Params(**prm)
    C = np.empty((K, d), np.float64)
    rho = np.empty(N, np.int32)
    info = _Info()
    tr = (_Trace * max(1, prm["max_iter"]))() if trace else None
    _load().orc_solve(_ptr(X, _dp), N, d, K, _ptr(C0, _dp), ctypes.byref(p), _ptr(C, _dp),
                      _ptr(rho, _ip), ctypes.byref(info),
                      ctypes.cast(tr, ctypes.POINTER(_Trace)) if tr is not None else None)
    out = {f: getattr(info, f) for f, _ in _Info._fields_}
    if not trace:
        return C, rho, out
    recs = [{f: getattr(tr[i], f) for f, _ in _Trace._fields_ if f != "pad"}
            for i in range(out["iters"])]
    return C, rho, out, recs


def step(X, state: dict, **kw):
    """One loop pass t of Algorithm 1 from an explicit state (the same routine ``solve`` loops over).

    state: C (C^t, the iterate to assign), CAU (G^{t-1}), F (F^{t-1}), dF and dG ([count, K*d]
    differences, newest first), Pprev (P^{t-1}), t, m, from_lloyd (1 if C^t is a plain Lloyd
    iterate), E_prev (E^{t-1}), E_prev2 (E^{t-2}); kw are solver parameters as for ``solve``.
    Returns (new_state, record): new_state holds the same keys after the pass (C = C^{t+1},
    CAU = G^t, F = F^t, Pprev = P^t, t + 1, ...) plus done, E (terminal energy), theta (the last
    least-squares solution, zeros past its rank) and the pass counters; record is the pass's trace
    record (n_changed, m, m_t, rank, rejected, E_trial, E)."""
    X = _f64(X)
    N, d = X.shape
    C = _f64(state["C"]).copy()
    K = C.shape[0]
    n = K * d
    prm = dict(DEFAULT_PARAMS)
    prm.update(kw)
    m_max = 0 if prm["lloyd_only"] else prm["m_max"]
    mm = max(m_max, 1)
    dF = np.zeros((mm, n), np.float64)
    dG = np.zeros((mm, n), np.float64)
    cnt = int(state.get("count", len(state.get("dF", []))))
    if cnt:
        dF[:cnt] = np.asarray(state["dF"], np.float64).reshape(cnt, n)
        dG[:cnt] = np.asarray(state["dG"], np.float64).reshape(cnt, n)
    CAU = _f64(state["CAU"]).reshape(K, d).copy()
    F = _f64(state["F"]).reshape(K, d).copy()
    Pprev = np.ascontiguousarray(state["Pprev"], dtype=np.int32).copy()
    st = _State()
    st.C, st.CAU, st.F = _ptr(C, _dp), _ptr(CAU, _dp), _ptr(F, _dp)
    st.dF, st.dG, st.Pprev = _ptr(dF, _dp), _ptr(dG, _dp), _ptr(Pprev, _ip)
    st.count, st.t, st.m, st.from_lloyd = cnt, int(state["t"]), int(state["m"]), int(state["from_lloyd"])
    st.E_prev, st.E_prev2 = float(state["E_prev"]), float(state["E_prev2"])
    st.accepted = int(state.get("accepted", 0))
    st.rejected = int(state.get("rejected", 0))
    st.assign_passes = int(state.get("assign_passes", 0))
    p = _Params(**prm)
    rec = _Trace()
    P = np.empty(N, np.int32)
    G = np.empty(n, np.float64)
    Fn = np.empty(n, np.float64)
    Cn = np.empty(n, np.float64)
    _load().orc_step(_ptr(X, _dp), N, d, K, ctypes.byref(p), ctypes.byref(st), ctypes.byref(rec),
                     _ptr(P, _ip), _ptr(G, _dp), _ptr(Fn, _dp), _ptr(Cn, _dp))
    out = dict(C=C, CAU=CAU, F=F, dF=dF[:st.count].copy(), dG=dG[:st.count].copy(), Pprev=Pprev,
               count=st.count, t=st.t, m=st.m, from_lloyd=st.from_lloyd, E_prev=st.E_prev,
               E_prev2=st.E_prev2, done=st.done, E=st.E, accepted=st.accepted, rejected=st.rejected,
               assign_passes=st.assign_passes, theta=np.array(st.theta[:], np.float64))
    return out, {f: getattr(rec, f) for f, _ in _Trace._fields_ if f != "pad"}
