"""PyTorch-facing binding of the C ABI.

Same entry-point names as ``include/tgp.h``.  These functions only marshal
arguments: they check dtypes and shapes, allocate the outputs and the
workspace as torch device tensors (torch is the memory manager), and pass raw
device pointers plus the current CUDA stream to ``libtgp.so``.  Every step of
the evaluation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check, tgp_config, tgp_data, tgp_population

_WS: dict = {}


def _stream_handle(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def workspace(nbytes: int, device) -> torch.Tensor:
    """A cached uint8 workspace of at least nbytes on device (per stream)."""
    key = (torch.device(device).index, _stream_handle(device))
    ws = _WS.get(key)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
        _WS[key] = ws
    return ws


def _f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    return t


def make_population(type_, val, size, max_len: int | None = None) -> tgp_population:
    for name, t in (("type", type_), ("value", val), ("size", size)):
        _f32(t, name)
        if t.dim() != 2:
            raise ValueError(f"{name} must be [pop, ld]")
        if t.numel() > 0 and t.shape[1] > 1 and t.stride(1) != 1:
            raise ValueError(f"{name} must have unit column stride")
    if not type_.shape == val.shape == size.shape:
        raise ValueError("type, value and size must share their shape")
    if type_.numel() > 0 and not type_.stride() == val.stride() == size.stride():
        raise ValueError("type, value and size must share their strides")
    P, L = type_.shape
    ld = type_.stride(0) if P > 1 else L
    return tgp_population(type_.data_ptr(), val.data_ptr(), size.data_ptr(), P,
                          int(max_len if max_len is not None else L), max(ld, L))


def make_data(X) -> tgp_data:
    _f32(X, "X")
    if X.dim() != 2:
        raise ValueError("X must be [n_points, n_features]")
    D, F = X.shape
    if D > 0 and F > 1 and X.stride(1) != 1:
        raise ValueError("X must have unit column stride")
    ldx = X.stride(0) if D > 1 else F
    return tgp_data(X.data_ptr(), D, F, max(ldx, F))


def make_config(cfg) -> tgp_config | None:
    if cfg is None:
        return None
    if isinstance(cfg, tgp_config):
        return cfg
    ev0, ev1 = cfg.get("eval_begin_event"), cfg.get("eval_end_event")
    for ev in (ev0, ev1):
        if ev is not None and not ev.cuda_event:
            ev.record()  # torch creates the CUDA event lazily on its first record
    flags = int(cfg.get("flags", 0)) | (_lib.FLAG_SSE if cfg.get("sse") else 0)
    return tgp_config(int(cfg.get("trees_per_block", 0)), int(cfg.get("points_per_tile", 0)),
                      int(cfg.get("tiles_per_item", 0)), int(cfg.get("points_per_lane", 0)),
                      ev0.cuda_event if ev0 is not None else None,
                      ev1.cuda_event if ev1 is not None else None,
                      flags, int(cfg.get("max_wait_polls", 0)), int(cfg.get("cta_width", 0)))


def _cref(c):
    return ctypes.byref(c) if c is not None else None


def tgp_workspace_size(type_, val, size, X=None, n_outputs: int = 1, max_len=None, config=None) -> int:
    lib = _lib.load()
    pop = make_population(type_, val, size, max_len)
    data = make_data(X) if X is not None else None
    n = lib.tgp_workspace_size(ctypes.byref(pop), _cref(data), n_outputs, _cref(make_config(config)))
    if n == 0:
        raise _lib.TGPError(_lib.TGP_ERR_INVALID_ARG, "tgp_workspace_size")
    return int(n)


def tgp_validate(type_, val, size, n_features: int, n_outputs: int = 1, max_len=None) -> torch.Tensor:
    """Per-tree status bitmask (int32 [pop])."""
    lib = _lib.load()
    pop = make_population(type_, val, size, max_len)
    dev = type_.device
    st = torch.empty(pop.pop, dtype=torch.int32, device=dev)
    n = lib.tgp_workspace_size(ctypes.byref(pop), None, n_outputs, None)
    ws = workspace(n, dev)
    check(lib.tgp_validate(ctypes.byref(pop), n_features, n_outputs, st.data_ptr(), ws.data_ptr(),
                           ws.numel(), _stream_handle(dev)), "tgp_validate")
    return st


def tgp_eval_forward(type_, val, size, X, n_outputs: int = 1, max_len=None, config=None,
                     out=None, tree_status=None):
    """Forward outputs [pop, n_outputs, n_points] float32 and tree status."""
    lib = _lib.load()
    pop = make_population(type_, val, size, max_len)
    data = make_data(X)
    dev = X.device
    if out is None:
        out = torch.empty((pop.pop, n_outputs, data.n_points), dtype=torch.float32, device=dev)
    if tree_status is None:
        tree_status = torch.empty(pop.pop, dtype=torch.int32, device=dev)
    cfg = make_config(config)
    n = lib.tgp_workspace_size(ctypes.byref(pop), ctypes.byref(data), n_outputs, _cref(cfg))
    if n == 0:
        raise _lib.TGPError(_lib.TGP_ERR_INVALID_ARG, "tgp_workspace_size")
    ws = workspace(n, dev)
    check(lib.tgp_eval_forward_cfg(ctypes.byref(pop), ctypes.byref(data), n_outputs, out.data_ptr(),
                                   tree_status.data_ptr(), ws.data_ptr(), ws.numel(),
                                   _stream_handle(dev), _cref(cfg)), "tgp_eval_forward")
    return out, tree_status


def tgp_fitness_mse(type_, val, size, X, y, n_outputs: int = 1, max_len=None, config=None,
                    mse=None, tree_status=None):
    """Per-tree, per-output MSE [pop, n_outputs] float64 and tree status."""
    lib = _lib.load()
    pop = make_population(type_, val, size, max_len)
    data = make_data(X)
    _f32(y, "y")
    if not y.is_contiguous() or y.numel() != data.n_points * n_outputs:
        raise ValueError("y must be a contiguous [n_points, n_outputs] float32 tensor")
    dev = X.device
    if mse is None:
        mse = torch.empty((pop.pop, n_outputs), dtype=torch.float64, device=dev)
    if tree_status is None:
        tree_status = torch.empty(pop.pop, dtype=torch.int32, device=dev)
    cfg = make_config(config)
    n = lib.tgp_workspace_size(ctypes.byref(pop), ctypes.byref(data), n_outputs, _cref(cfg))
    if n == 0:
        raise _lib.TGPError(_lib.TGP_ERR_INVALID_ARG, "tgp_workspace_size")
    ws = workspace(n, dev)
    check(lib.tgp_fitness_mse_cfg(ctypes.byref(pop), ctypes.byref(data), y.data_ptr(), n_outputs,
                                  mse.data_ptr(), tree_status.data_ptr(), ws.data_ptr(), ws.numel(),
                                  _stream_handle(dev), _cref(cfg)), "tgp_fitness_mse")
    return mse, tree_status


def tgp_check_device_error(device=None):
    """Raises if a bounded device-side wait gave up during the last call."""
    lib = _lib.load()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    ws = _WS.get((dev.index, _stream_handle(dev)))
    if ws is None:
        return
    check(lib.tgp_check_device_error(ws.data_ptr(), ws.numel(), _stream_handle(dev)),
          "tgp_check_device_error")


def population_to(pop, device) -> tuple:
    """workloads.Population -> (type, value, size) float32 device tensors."""
    return tuple(torch.from_numpy(a).to(device) for a in (pop.type, pop.val, pop.size))


def tgp_eval_backward(type_, val, size, X, y, grad_mse, n_outputs: int = 1, max_len=None,
                      want_mse: bool = True, want_grad_value: bool = True, want_grad_X: bool = True,
                      grad_X=None, tree_status=None, config=None):
    """Reverse-mode gradient of sum(grad_mse * MSE).

    Returns (mse [pop, O] float64 or None, grad_value [pop, ld] float32 or None,
    grad_X [n_points, n_features] float32 or None, tree status).  grad_X, when
    given, is accumulated into; otherwise a zeroed tensor is allocated.
    """
    lib = _lib.load()
    pop = make_population(type_, val, size, max_len)
    data = make_data(X)
    _f32(y, "y")
    if not y.is_contiguous() or y.numel() != data.n_points * n_outputs:
        raise ValueError("y must be a contiguous [n_points, n_outputs] float32 tensor")
    dev = X.device
    g = grad_mse.to(device=dev, dtype=torch.float64).contiguous()
    if g.numel() != pop.pop * n_outputs:
        raise ValueError("grad_mse must have pop * n_outputs elements")
    mse = torch.empty((pop.pop, n_outputs), dtype=torch.float64, device=dev) if want_mse else None
    gv = torch.empty(type_.shape, dtype=torch.float32, device=dev) if want_grad_value else None
    if want_grad_X and grad_X is None:
        grad_X = torch.zeros(X.shape, dtype=torch.float32, device=dev)
    if not want_grad_X:
        grad_X = None
    if grad_X is not None and (grad_X.shape != X.shape or not grad_X.is_contiguous()):
        raise ValueError("grad_X must be a contiguous tensor shaped like X")
    if tree_status is None:
        tree_status = torch.empty(pop.pop, dtype=torch.int32, device=dev)
    n = lib.tgp_workspace_size(ctypes.byref(pop), ctypes.byref(data), n_outputs, None)
    if n == 0:
        raise _lib.TGPError(_lib.TGP_ERR_INVALID_ARG, "tgp_workspace_size")
    ws = workspace(n, dev)
    ptr = lambda t: t.data_ptr() if t is not None else None
    check(lib.tgp_eval_backward_cfg(ctypes.byref(pop), ctypes.byref(data), y.data_ptr(), n_outputs,
                                    g.data_ptr(), ptr(mse), ptr(gv), ptr(grad_X), tree_status.data_ptr(),
                                    ws.data_ptr(), ws.numel(), _stream_handle(dev),
                                    _cref(make_config(config))), "tgp_eval_backward")
    return mse, gv, grad_X, tree_status


class BatchProblem:
    """One problem of a batched fitness call (device tensors)."""

    def __init__(self, type_, val, size, X, y, n_outputs=1, max_len=None, config=None):
        self.tensors = (type_, val, size, X, y)
        self.n_outputs = n_outputs
        self.pop = make_population(type_, val, size, max_len)
        self.data = make_data(X)
        _f32(y, "y")
        if not y.is_contiguous() or y.numel() != self.data.n_points * n_outputs:
            raise ValueError("y must be a contiguous [n_points, n_outputs] float32 tensor")
        dev = X.device
        self.mse = torch.empty((self.pop.pop, n_outputs), dtype=torch.float64, device=dev)
        self.status = torch.empty(self.pop.pop, dtype=torch.int32, device=dev)
        cfg = make_config(config)
        self.cfg = cfg if cfg is not None else tgp_config()

    def c_struct(self):
        return _lib.tgp_problem(self.pop, self.data, self.tensors[4].data_ptr(), self.n_outputs,
                                self.mse.data_ptr(), self.status.data_ptr(), self.cfg)


def tgp_batch_workspace_size(problems) -> int:
    arr = (_lib.tgp_problem * len(problems))(*[p.c_struct() for p in problems])
    n = _lib.load().tgp_batch_workspace_size(arr, len(problems))
    if n == 0:
        raise _lib.TGPError(_lib.TGP_ERR_INVALID_ARG, "tgp_batch_workspace_size")
    return int(n)


def tgp_batch_fitness_mse(problems, ws=None):
    """MSE of every problem in one batched launch; fills problem.mse/status."""
    lib = _lib.load()
    arr = (_lib.tgp_problem * len(problems))(*[p.c_struct() for p in problems])
    dev = problems[0].tensors[3].device
    n = lib.tgp_batch_workspace_size(arr, len(problems))
    if n == 0:
        raise _lib.TGPError(_lib.TGP_ERR_INVALID_ARG, "tgp_batch_workspace_size")
    if ws is None:
        ws = workspace(n, dev)
    elif ws.numel() < n:
        raise ValueError("workspace too small")
    check(lib.tgp_batch_fitness_mse(arr, len(problems), ws.data_ptr(), ws.numel(), _stream_handle(dev)),
          "tgp_batch_fitness_mse")
    return [p.mse for p in problems]


class BatchPlan:
    """A batch planned once on the host (tgp_batch_plan) and run any number of
    times (tgp_batch_run, legal in CUDA graph capture).  `tune_cache` is the
    autotuner's cache file (None: the library's heuristic for every problem
    without its own shape)."""

    def __init__(self, problems, tune_cache=None):
        lib = _lib.load()
        self.problems = list(problems)   # keeps the tensors alive
        arr = (_lib.tgp_problem * len(self.problems))(*[p.c_struct() for p in self.problems])
        h = ctypes.c_void_p()
        path = tune_cache.encode() if tune_cache else None
        check(lib.tgp_batch_plan(arr, len(self.problems), path, ctypes.byref(h)), "tgp_batch_plan")
        self._h = h
        self.ws_bytes = int(lib.tgp_batch_plan_workspace_size(h))
        self.device = self.problems[0].tensors[3].device
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=self.device)

    def shape(self, i: int):
        """(launch shape dict, from_cache) the plan chose for problem i."""
        c = tgp_config()
        fc = ctypes.c_int32()
        check(_lib.load().tgp_batch_plan_shape(self._h, i, ctypes.byref(c), ctypes.byref(fc)),
              "tgp_batch_plan_shape")
        return ({"trees_per_block": c.trees_per_block, "points_per_tile": c.points_per_tile,
                 "tiles_per_item": c.tiles_per_item, "points_per_lane": c.points_per_lane},
                bool(fc.value))

    def run(self):
        check(_lib.load().tgp_batch_run(self._h, self.ws.data_ptr(), self.ws.numel(),
                                        _stream_handle(self.device)), "tgp_batch_run")
        return [p.mse for p in self.problems]

    def check_device_error(self):
        check(_lib.load().tgp_check_device_error(self.ws.data_ptr(), self.ws.numel(),
                                                 _stream_handle(self.device)),
              "tgp_check_device_error")

    def close(self):
        if self._h:
            _lib.load().tgp_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------ genetic operators
def _i32(t, name, n=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int32:
        raise TypeError(f"{name} must be a CUDA int32 tensor")
    if not t.is_contiguous() or (n is not None and t.numel() != n):
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return t


def tgp_subtree_exchange(old, old_index, node, donor=None, donor_index=None, donor_node=None,
                         mode: int = _lib.PICK_RANDOM, max_size: int = 512, out_ld=None,
                         apply_word=None, apply_below: int = 0, old_max_len=None,
                         donor_max_len=None, out=None, status=None):
    """Subtree exchange (Sec. III-B) of ``len(old_index)`` children.

    ``old`` / ``donor`` are (type, value, size) tuples of float32 [P, ld]
    device tensors; ``old_index`` / ``donor_index`` int32 rows; ``node`` /
    ``donor_node`` / ``apply_word`` int32 tensors read as uint32 words.
    Returns ((type, value, size) of the children [n, out_ld], status int32 [n]).
    """
    lib = _lib.load()
    n = old_index.numel()
    op = make_population(*old, old_max_len)
    dp = make_population(*donor, donor_max_len) if donor is not None else None
    dev = old[0].device
    _i32(old_index, "old_index", n)
    _i32(node, "node", n)
    if mode != _lib.PICK_HOIST:
        if dp is None or donor_index is None:
            raise ValueError("crossover and subtree mutation need a donor population and rows")
        _i32(donor_index, "donor_index", n)
    for t, name in ((donor_node, "donor_node"), (apply_word, "apply_word")):
        if t is not None:
            _i32(t, name, n)
    ld = int(out_ld if out_ld is not None else max(max_size, op.max_len))
    if out is None:
        out = tuple(torch.empty((n, ld), dtype=torch.float32, device=dev) for _ in range(3))
    for t in out:
        _f32(t, "out")
        if t.shape != (n, ld) or not t.is_contiguous():
            raise ValueError(f"out tensors must be contiguous float32 [{n}, {ld}]")
    if status is None:
        status = torch.empty(n, dtype=torch.int32, device=dev)
    _i32(status, "status", n)
    ptr = lambda t: t.data_ptr() if t is not None else None
    check(lib.tgp_subtree_exchange(ctypes.byref(op), _cref(dp), old_index.data_ptr(),
                                   node.data_ptr(), ptr(donor_index), ptr(donor_node),
                                   ptr(apply_word), int(apply_below) & 0xFFFFFFFF, n, int(mode),
                                   int(max_size), out[0].data_ptr(), out[1].data_ptr(),
                                   out[2].data_ptr(), ld, status.data_ptr(), _stream_handle(dev)),
          "tgp_subtree_exchange")
    return out, status


def tgp_tournament_select(fitness, words, minimize: bool = True, winners=None):
    """Winner row per selection; ``fitness`` float64 [P] (or a column view
    with a stride), ``words`` int32 [n, t] read as uint32."""
    lib = _lib.load()
    if fitness.dtype != torch.float64 or not fitness.is_cuda or fitness.dim() != 1:
        raise TypeError("fitness must be a 1-D CUDA float64 tensor")
    if words.dim() != 2:
        raise ValueError("words must be [n, tournament_size]")
    _i32(words, "words")
    n, t = words.shape
    if winners is None:
        winners = torch.empty(n, dtype=torch.int32, device=words.device)
    _i32(winners, "winners", n)
    check(lib.tgp_tournament_select(fitness.data_ptr(), max(fitness.stride(0), 1), fitness.numel(),
                                    words.data_ptr(), n, t, int(bool(minimize)),
                                    winners.data_ptr(), _stream_handle(words.device)),
          "tgp_tournament_select")
    return winners


def tgp_accuracy_from_outputs(out, labels):
    """(accuracy float64 [P], correct int64 [P]) of forward outputs [P, C, D]."""
    lib = _lib.load()
    _f32(out, "out")
    if out.dim() != 3 or not out.is_contiguous():
        raise ValueError("out must be a contiguous [pop, n_classes, n_points] tensor")
    P, C, D = out.shape
    _i32(labels, "labels", D)
    acc = torch.empty(P, dtype=torch.float64, device=out.device)
    cnt = torch.empty(P, dtype=torch.int64, device=out.device)
    check(lib.tgp_accuracy_from_outputs(out.data_ptr(), P, C, D, labels.data_ptr(), cnt.data_ptr(),
                                        acc.data_ptr(), _stream_handle(out.device)),
          "tgp_accuracy_from_outputs")
    return acc, cnt


def tgp_fitness_accuracy(type_, val, size, X, labels, n_classes: int, max_len=None):
    """(accuracy float64 [P], correct int64 [P], tree status int32 [P])."""
    lib = _lib.load()
    pop = make_population(type_, val, size, max_len)
    data = make_data(X)
    _i32(labels, "labels", data.n_points)
    dev = X.device
    n = lib.tgp_accuracy_workspace_size(ctypes.byref(pop), ctypes.byref(data), n_classes)
    if n == 0:
        raise _lib.TGPError(_lib.TGP_ERR_INVALID_ARG, "tgp_accuracy_workspace_size")
    ws = workspace(n, dev)
    acc = torch.empty(pop.pop, dtype=torch.float64, device=dev)
    cnt = torch.empty(pop.pop, dtype=torch.int64, device=dev)
    st = torch.empty(pop.pop, dtype=torch.int32, device=dev)
    check(lib.tgp_fitness_accuracy(ctypes.byref(pop), ctypes.byref(data), labels.data_ptr(),
                                   n_classes, acc.data_ptr(), cnt.data_ptr(), st.data_ptr(),
                                   ws.data_ptr(), ws.numel(), _stream_handle(dev)),
          "tgp_fitness_accuracy")
    return acc, cnt, st
