"""FP64 CPU oracle for tensorized tree-based GP fitness evaluation.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference that
the CUDA library is checked against; it is imported only by the tests, the
smoke check and the CPU-baseline leg of the benchmark.  The library never
imports it and never falls back to it.  It shares no code with the CUDA path.

The arithmetic lives in ``tgp_oracle.c`` (plain recursive FP64 interpreter,
Sec. II-A node semantics, Sec. III-A encoding, Sec. III-C MSE fitness,
Sec. IV-C Modi nodes, plus reverse mode).  This module only compiles it with
gcc and marshals numpy arrays.

Pinned by ``tests/test_oracle_pins.py`` (closed forms of the paper's sigmoid
and Modi examples, brute force over tiny trees against a separately written
Python restatement, subtree-size invariants, finite differences, guards).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tgp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtgp_oracle.so")
_lock = threading.Lock()
_lib = None

# restated encoding (Sec. III-A and the readings in tgp_oracle.c)
VAR, CONST, UFUNC, BFUNC, TFUNC, MODI = 0, 1, 2, 3, 4, 16
ADD, SUB, MUL, PDIV, MAX, SIN, COS, PLOG, CEXP, TAN, ITE = range(11)

ST_LEN, ST_TYPE, ST_FUNC, ST_VAR, ST_MODI, ST_CONST, ST_SIZE = 1, 2, 4, 8, 16, 32, 64


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (host code only, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            fp, dp, ip = (ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_int))
            L, I, D = ctypes.c_long, ctypes.c_int, ctypes.c_double
            lib.orc_validate.argtypes = [fp, fp, fp, L, L, I, I, I, ip, ip]
            lib.orc_validate.restype = None
            lib.orc_eval.argtypes = [fp, fp, fp, L, L, I, fp, L, I, L, I, dp, dp, ip, I]
            lib.orc_eval.restype = None
            lib.orc_mse.argtypes = [fp, fp, fp, L, L, I, fp, L, I, L, fp, L, I, dp, dp, D, ip, I]
            lib.orc_mse.restype = None
            lib.orc_grad.argtypes = [fp, fp, fp, L, L, I, fp, L, I, L, fp, L, I, dp, dp, dp, dp, ip, I]
            lib.orc_grad.restype = None
            lib.orc_grad_bound.argtypes = [fp, fp, fp, L, L, I, fp, L, I, L, fp, L, I, dp, dp, dp, dp,
                                           dp, dp, D, ip, I]
            lib.orc_grad_bound.restype = None
            lib.orc_apply.argtypes = [I, D, D]
            lib.orc_apply.restype = D
            lib.orc_apply3.argtypes = [I, D, D, D]
            lib.orc_apply3.restype = D
            _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


def _pop(type_, val, size):
    t, v, s = _f32(type_), _f32(val), _f32(size)
    if t.ndim == 1:
        t, v, s = t[None], v[None], s[None]
    assert t.shape == v.shape == s.shape
    return t, v, s


def validate(type_, val, size, n_features, n_outputs=1, max_len=None):
    """Per-tree status bitmask and length (Sec. III-A encoding rules)."""
    t, v, s = _pop(type_, val, size)
    pop, ld = t.shape
    ml = ld if max_len is None else max_len
    st = np.zeros(pop, np.int32)
    ln = np.zeros(pop, np.int32)
    _load().orc_validate(_ptr(t, ctypes.c_float), _ptr(v, ctypes.c_float), _ptr(s, ctypes.c_float),
                         pop, ld, ml, n_features, n_outputs, _ptr(st, ctypes.c_int),
                         _ptr(ln, ctypes.c_int))
    return st, ln


def evaluate(type_, val, size, X, n_outputs=1, with_err=False, threads=None, max_len=None):
    """Outputs [pop, O, D] in FP64 (and the FP32 error bound if asked)."""
    t, v, s = _pop(type_, val, size)
    X = _f32(X)
    pop, ld = t.shape
    D, F = X.shape
    out = np.empty((pop, n_outputs, D), np.float64)
    err = np.empty_like(out) if with_err else None
    st = np.zeros(pop, np.int32)
    _load().orc_eval(_ptr(t, ctypes.c_float), _ptr(v, ctypes.c_float), _ptr(s, ctypes.c_float),
                     pop, ld, ld if max_len is None else max_len, _ptr(X, ctypes.c_float), D, F, F,
                     n_outputs, _ptr(out, ctypes.c_double),
                     _ptr(err, ctypes.c_double) if with_err else None,
                     _ptr(st, ctypes.c_int), _threads(threads))
    return (out, err, st) if with_err else (out, st)


def mse(type_, val, size, X, y, n_outputs=1, rel_tol=None, threads=None, max_len=None):
    """MSE [pop, O] in FP64; with rel_tol also the per-tree MSE allowance."""
    t, v, s = _pop(type_, val, size)
    X = _f32(X)
    y = _f32(y).reshape(X.shape[0], n_outputs)
    pop, ld = t.shape
    D, F = X.shape
    m = np.empty((pop, n_outputs), np.float64)
    allow = np.empty_like(m) if rel_tol is not None else None
    st = np.zeros(pop, np.int32)
    _load().orc_mse(_ptr(t, ctypes.c_float), _ptr(v, ctypes.c_float), _ptr(s, ctypes.c_float),
                    pop, ld, ld if max_len is None else max_len, _ptr(X, ctypes.c_float), D, F, F,
                    _ptr(y, ctypes.c_float), n_outputs, n_outputs, _ptr(m, ctypes.c_double),
                    _ptr(allow, ctypes.c_double) if allow is not None else None,
                    float(rel_tol or 0.0), _ptr(st, ctypes.c_int), _threads(threads))
    return (m, allow, st) if rel_tol is not None else (m, st)


def grad(type_, val, size, X, y, g, n_outputs=1, threads=None, max_len=None, with_err=False,
         acc_terms=1024):
    """Reverse mode of sum(g * MSE): (mse [pop,O], grad_val [pop,ld], grad_X [D,F], status);
    with_err adds (egrad_val [pop,ld], egrad_X [D,F]): per element, a first-order
    bound on how far an FP32 evaluation of the gradient may land (FP32 partial
    sums of at most `acc_terms` contributions per constant before FP64)."""
    t, v, s = _pop(type_, val, size)
    X = _f32(X)
    y = _f32(y).reshape(X.shape[0], n_outputs)
    pop, ld = t.shape
    D, F = X.shape
    g = np.ascontiguousarray(np.broadcast_to(np.asarray(g, np.float64), (pop, n_outputs)))
    m = np.empty((pop, n_outputs), np.float64)
    gv = np.empty((pop, ld), np.float64)
    gx = np.empty((D, F), np.float64)
    st = np.zeros(pop, np.int32)
    egv = np.empty((pop, ld), np.float64) if with_err else None
    egx = np.empty((D, F), np.float64) if with_err else None
    _load().orc_grad_bound(_ptr(t, ctypes.c_float), _ptr(v, ctypes.c_float), _ptr(s, ctypes.c_float),
                           pop, ld, ld if max_len is None else max_len, _ptr(X, ctypes.c_float), D, F, F,
                           _ptr(y, ctypes.c_float), n_outputs, n_outputs, _ptr(g, ctypes.c_double),
                           _ptr(m, ctypes.c_double), _ptr(gv, ctypes.c_double),
                           _ptr(gx, ctypes.c_double),
                           _ptr(egv, ctypes.c_double) if with_err else None,
                           _ptr(egx, ctypes.c_double) if with_err else None,
                           float(acc_terms), _ptr(st, ctypes.c_int), _threads(threads))
    return (m, gv, gx, st, egv, egx) if with_err else (m, gv, gx, st)


def apply(f: int, a: float, b: float = 0.0) -> float:
    """One function of the table in FP64."""
    return _load().orc_apply(int(f), float(a), float(b))
