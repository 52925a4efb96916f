"""Launch-shape autotuner for the evaluation kernels.

Measures candidate launch shapes (points per lane, trees per block, points
per tile, tiles per item) of ``tgp_fitness_mse`` on the problem at hand with
CUDA events, and caches the fastest per GPU and shape bucket in a JSON file
(``$TGP_AUTOTUNE_CACHE``, default ``~/.cache/tgp_gb300/autotune.json``).

The candidates span the two schedules of the paper's adaptive parallelism
(Sec. III-C): many trees per block over small point tiles (population
parallelism, the paper's "hybrid" mode for small D) and few trees per block
over large point tiles (data parallelism, its mode for large D).
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import api

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("TGP_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tgp_gb300", "autotune.json"))


def _bucket(P: int, D: int, F: int, O: int, max_len: int) -> str:
    lg = lambda x: int(round(math.log2(max(int(x), 1))))
    return f"P{lg(P)}_D{lg(D)}_F{F}_O{O}_L{lg(max_len)}"


def _key(device, P, D, F, O, max_len) -> str:
    name = torch.cuda.get_device_name(device).replace(" ", "_")
    return f"{name}|{_bucket(P, D, F, O, max_len)}"


def candidates(P: int, D: int, O: int = 1):
    out = [{}]  # the library's own shape heuristic
    for K in ((4,) if O > 1 else (8, 4)):
        ch = 32 * K
        for tp_mult in (1, 2, 4, 8):
            tp = ch * tp_mult
            if tp > 4096 or (tp > ch and tp // 2 >= D):
                continue
            for bt in (1, 4, 8, 16, 32):
                if bt > P:
                    continue
                out.append({"points_per_lane": K, "points_per_tile": tp, "trees_per_block": bt})
    return out


def _load():
    p = cache_path()
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except (OSError, ValueError):
            return {}
    return {}


def _store(db):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".{os.getpid()}.tmp"
    json.dump(db, open(tmp, "w"), indent=1, sort_keys=True)
    os.replace(tmp, p)


def lookup(device, P, D, F, O, max_len):
    with _lock:
        return _load().get(_key(device, P, D, F, O, max_len))


def tune(type_, val, size, X, y, n_outputs=1, max_len=None, reps=3, cands=None, store=True,
         verbose=False):
    """Times every candidate on this problem; returns (best config, table)."""
    P, L = type_.shape
    D, F = X.shape
    max_len = max_len or L
    cands = cands or candidates(P, D, n_outputs)
    table = []
    for cfg in cands:
        try:
            api.tgp_fitness_mse(type_, val, size, X, y, n_outputs, max_len=max_len, config=cfg or None)
        except Exception:  # shape not supported (shared memory): skip
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c = dict(cfg, eval_begin_event=e0, eval_end_event=e1)
        best = float("inf")
        for _ in range(reps):
            api.tgp_fitness_mse(type_, val, size, X, y, n_outputs, max_len=max_len, config=c)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        table.append((best, cfg))
        if verbose:
            print(f"{best:9.3f} ms  {cfg}", flush=True)
    table.sort(key=lambda t: t[0])
    best_cfg = table[0][1]
    if store:
        with _lock:
            db = _load()
            db[_key(X.device, P, D, F, n_outputs, max_len)] = dict(best_cfg, ms=table[0][0])
            _store(db)
    return best_cfg, table
