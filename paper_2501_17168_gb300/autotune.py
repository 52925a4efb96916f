"""Launch-shape autotuner for the evaluation kernels.

Measures candidate launch shapes (points per lane, trees per block, points
per tile, tiles per item) of ``tgp_fitness_mse`` on the problem at hand with
CUDA events, and caches the fastest per GPU and shape bucket in a text file
(``$TGP_AUTOTUNE_CACHE``, default ``~/.cache/tgp_gb300/autotune.txt``) that
the C library reads itself: ``tgp_batch_plan(probs, n, cache_path, &plan)``
takes the stored shape for every problem without its own, and
``tgp_tune_cache_lookup`` reads one entry.  One entry per line:

    <GPU name, spaces as '_'>|P<lg P>_D<lg D>_F<F>_O<O>_L<lg max_len> \
        trees_per_block=<n> points_per_tile=<n> tiles_per_item=<n> points_per_lane=<n> ms=<t>

(all on one line; lg x = log2(x) rounded to the nearest integer; '#' starts a
comment; the last line of a key wins).

The candidates span the two schedules of the paper's adaptive parallelism
(Sec. III-C): many trees per block over small point tiles (population
parallelism, the paper's "hybrid" mode for small D) and few trees per block
over large point tiles (data parallelism, its mode for large D).
"""
from __future__ import annotations

import math
import os
import threading

SHAPE_FIELDS = ("trees_per_block", "points_per_tile", "tiles_per_item", "points_per_lane", "cta_width")

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("TGP_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tgp_gb300", "autotune.txt"))


def lg(x: int) -> int:
    """log2 rounded to the nearest integer (x < 1 counts as 1)."""
    return int(round(math.log2(max(int(x), 1))))


def bucket(P: int, D: int, F: int, O: int, max_len: int) -> str:
    return f"P{lg(P)}_D{lg(D)}_F{int(F)}_O{int(O)}_L{lg(max_len)}"


def key(gpu_name: str, P, D, F, O, max_len) -> str:
    return f"{gpu_name.replace(' ', '_')}|{bucket(P, D, F, O, max_len)}"


def _device_key(device, P, D, F, O, max_len) -> str:
    import torch
    return key(torch.cuda.get_device_name(device), P, D, F, O, max_len)


def candidates(P: int, D: int, O: int = 1):
    """The heuristic ({}) plus points per lane x tile widths x tree blocks:
    from one tree per block over wide tiles (the data-parallel schedule) to
    64 trees per block over one-chunk tiles (the population-parallel one;
    the wide CTAs of 28-32 warps want blocks of 32-64 trees), and at 8 points
    per lane each block of up to 32 trees also in the narrow CTAs."""
    out = [{}]  # the library's own shape heuristic
    for K in ((4,) if O > 1 else (8, 4)):
        ch = 32 * K
        for tp_mult in (1, 2, 4, 8):
            tp = ch * tp_mult
            if tp > 4096 or (tp > ch and tp // 2 >= D):
                continue
            for bt in (1, 4, 8, 16, 32, 64):
                if bt > P:
                    continue
                out.append({"points_per_lane": K, "points_per_tile": tp, "trees_per_block": bt})
                if K == 8 and bt <= 32:
                    # the narrow CTAs (several per SM) against the wide one
                    out.append({"points_per_lane": K, "points_per_tile": tp, "trees_per_block": bt,
                                "cta_width": 1})
    return out


def format_entry(k: str, cfg: dict, ms: float | None = None) -> str:
    fields = " ".join(f"{f}={int(cfg.get(f, 0))}" for f in SHAPE_FIELDS)
    return f"{k} {fields}" + (f" ms={ms:.6g}" if ms is not None else "")


def parse(text: str) -> dict:
    """{key: {shape fields..., 'ms': t}} of a cache file's text (last line wins)."""
    db = {}
    for line in text.splitlines():
        tok = line.split()
        if not tok or tok[0].startswith("#"):
            continue
        e = {}
        for t in tok[1:]:
            if "=" in t:
                n, v = t.split("=", 1)
                try:
                    e[n] = float(v) if n == "ms" else int(v)
                except ValueError:
                    pass
        db[tok[0]] = e
    return db


def load(path: str | None = None) -> dict:
    p = path or cache_path()
    try:
        with open(p) as f:
            return parse(f.read())
    except OSError:
        return {}


def store(entries: dict, path: str | None = None):
    """Merges {key: (cfg, ms)} into the cache file (atomic replace)."""
    p = path or cache_path()
    with _lock:
        db = load(p)
        for k, (cfg, ms) in entries.items():
            db[k] = dict({f: int(cfg.get(f, 0)) for f in SHAPE_FIELDS}, ms=ms)
        d = os.path.dirname(p)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = p + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            f.write("# tgp launch-shape cache: <gpu>|<bucket> shape fields (read by tgp_batch_plan)\n")
            for k in sorted(db):
                e = db[k]
                f.write(format_entry(k, e, e.get("ms")) + "\n")
        os.replace(tmp, p)


def lookup(device, P, D, F, O, max_len, path: str | None = None):
    e = load(path).get(_device_key(device, P, D, F, O, max_len))
    return None if e is None else {f: e.get(f, 0) for f in SHAPE_FIELDS}


def tune(type_, val, size, X, y, n_outputs=1, max_len=None, reps=3, cands=None, store_result=True,
         path: str | None = None, verbose=False):
    """Times every candidate on this problem; returns (best config, table).
    The heuristic ({}) is stored as the shape it resolves to, so that the
    cache entry always names a concrete shape."""
    import torch
    from . import api
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
    best_ms, best_cfg = table[0]
    if store_result and any(best_cfg.get(f) for f in SHAPE_FIELDS):
        store({_device_key(X.device, P, D, F, n_outputs, max_len): (best_cfg, best_ms)}, path)
    return best_cfg, table
