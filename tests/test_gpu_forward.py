"""GPU parity of the forward pass and MSE fitness against the FP64 oracle.

Everything goes through the C ABI (ctypes binding, torch only for device
memory).  Sizes are chosen so the oracle finishes in seconds while still
spanning several tiles, chunks and a ragged tail; the full-size sr_scale
workload is checked on sampled trees and points in the launch shape the
benchmark uses.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_17168_gb300 import api, workloads as W
from paper_2501_17168_gb300 import _lib
from parity import (PointStats, assert_mse_strict_floor, assert_strict_floor, compare_mse,
                    compare_points)

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_17168_gb300 import build
    build.build_all()
    _lib.load()


def dev_pop(p):
    return api.population_to(p, DEV)


def gpu_forward(p, X, O=1, config=None):
    t, v, s = dev_pop(p)
    out, st = api.tgp_eval_forward(t, v, s, torch.from_numpy(X).to(DEV), O, max_len=p.max_len,
                                   config=config)
    api.tgp_check_device_error()
    return out.cpu().numpy(), st.cpu().numpy()


def gpu_mse(p, X, y, O=1, config=None):
    t, v, s = dev_pop(p)
    m, st = api.tgp_fitness_mse(t, v, s, torch.from_numpy(X).to(DEV),
                                torch.from_numpy(np.ascontiguousarray(y, np.float32)).to(DEV), O,
                                max_len=p.max_len, config=config)
    api.tgp_check_device_error()
    return m.cpu().numpy(), st.cpu().numpy()


def targets(orc, prob, X=None, noise=None):
    X = prob.X if X is None else X
    noise = prob.noise if noise is None else noise
    out, st = orc.evaluate(prob.gt.type, prob.gt.val, prob.gt.size, X, n_outputs=1)
    y = np.stack([out[k, 0] for k in range(prob.gt.pop)], 1) + noise.astype(np.float64)
    return y.astype(np.float32)


def check_forward(orc, p, X, O=1, config=None, floor=True):
    """Every usable point within the bar (or within 2x the oracle's bound
    where no FP32 evaluation can meet it), and a strict fraction no lower
    than a float32 restatement's on the same points (less the margin the
    SFU approximations cost)."""
    g, gst = gpu_forward(p, X, O, config)
    ref, err, st = orc.evaluate(p.type, p.val, p.size, X, n_outputs=O, with_err=True,
                                max_len=p.max_len)
    np.testing.assert_array_equal(gst, st)
    ok = st == 0
    assert np.isnan(g[~ok]).all()
    stats = compare_points(g[ok], ref[ok], err[ok])
    assert stats.failed == 0, (stats, stats.examples)
    if floor:
        assert_strict_floor(g[ok], ref[ok], err[ok], p.type[ok], p.val[ok], p.size[ok], X, O)
    return stats


# ------------------------------------------------------------------ workloads
def test_sr_small_forward_and_mse(orc):
    prob = W.sr_small()
    stats = check_forward(orc, prob.pop, prob.X)
    y = targets(orc, prob)
    m, st = gpu_mse(prob.pop, prob.X, y)
    ref, allow, ost = orc.mse(prob.pop.type, prob.pop.val, prob.pop.size, prob.X, y, rel_tol=1e-5)
    r = compare_mse(m, ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
    assert_mse_strict_floor(m, ref, allow, prob.pop.type, prob.pop.val, prob.pop.size, prob.X, y)


@pytest.mark.parametrize("cfg", [None,
                                 {"points_per_lane": 4},
                                 {"points_per_lane": 8, "trees_per_block": 3, "points_per_tile": 512,
                                  "tiles_per_item": 2},
                                 {"points_per_lane": 4, "trees_per_block": 1, "points_per_tile": 128,
                                  "tiles_per_item": 5}])
def test_tiling_shapes_ragged_tail(orc, cfg):
    # 70 trees of length up to 255 over 1,234 points: several tiles, chunks
    # and tree blocks, and a ragged last tile
    p = W.random_population(101, 70, 255, (1, 255), max_depth=8, n_features=16)
    X = np.random.default_rng(1).standard_normal((1234, 16)).astype(np.float32)
    check_forward(orc, p, X, config=cfg)
    y = np.random.default_rng(2).standard_normal((1234, 1)).astype(np.float32)
    m, st = gpu_mse(p, X, y, config=cfg)
    ref, allow, ost = orc.mse(p.type, p.val, p.size, X, y, rel_tol=1e-5)
    r = compare_mse(m, ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r


def test_sr_scale_full_size_sampled(orc):
    prob = W.sr_scale()
    P, D = prob.pop.pop, prob.D
    # targets from the ground-truth tree (oracle), full size
    y = targets(orc, prob)
    m, st = gpu_mse(prob.pop, prob.X, y)
    assert (st == 0).all()
    pick = np.arange(0, P, 50)
    sub = prob.pop.take(pick)
    ref, allow, ost = orc.mse(sub.type, sub.val, sub.size, prob.X, y, rel_tol=1e-5)
    r = compare_mse(m[pick], ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
    assert_mse_strict_floor(m[pick], ref, allow, sub.type, sub.val, sub.size, prob.X, y)
    # per-point values on every 10th tree and every 97th point
    Xs = np.ascontiguousarray(prob.X[::97])
    g, gst = gpu_forward(prob.pop, Xs)
    sel = np.arange(0, P, 10)
    refp, err, _ = orc.evaluate(prob.pop.type[sel], prob.pop.val[sel], prob.pop.size[sel], Xs,
                                with_err=True)
    stats = compare_points(g[sel], refp, err)
    assert stats.failed == 0, (stats, stats.examples)
    assert_strict_floor(g[sel], refp, err, prob.pop.type[sel], prob.pop.val[sel], prob.pop.size[sel], Xs)
    assert stats.n >= 0.9 * len(sel) * Xs.shape[0], stats


# ------------------------------------------------------------------ examples
def test_paper_sigmoid_and_modi_examples():
    sig = W.encode(["pdiv", ("c", 1.0), "add", ("c", 1.0), "cexp", "sub", ("c", 0.0), ("x", 0)])
    x = np.linspace(-10, 10, 301, dtype=np.float32)[:, None]
    g, st = gpu_forward(sig, x)
    ref = 1 / (1 + np.exp(-x[:, 0].astype(np.float64)))
    assert st[0] == 0
    assert np.max(np.abs(g[0, 0] - ref) / np.maximum(np.abs(ref), 1)) <= 1e-5
    modi = W.encode([("mul", 0), "pdiv", ("x", 0), ("max", 1), ("x", 1), ("x", 2), ("add", 2), ("x", 4),
                     ("sub", 1), ("x", 3), ("c", 0.5)])
    X = np.random.default_rng(3).uniform(0.5, 3, (777, 5)).astype(np.float32)
    g, st = gpu_forward(modi, X, O=3)
    a, b, c, d, e = (X[:, i].astype(np.float64) for i in range(5))
    for k, want in enumerate([a / c * 0.5, np.maximum(b, c) + (d - 0.5), e + 0.5]):
        assert np.max(np.abs(g[0, k] - want) / np.maximum(np.abs(want), 1)) <= 1e-5


def test_guards_bit_exact():
    thr = np.float32(1e-6)
    up, dn = np.nextafter(thr, np.float32(1)), np.nextafter(thr, np.float32(0))
    bs = np.array([thr, -thr, up, -up, dn, -dn, 0, -0.0, 1e-40, -1e-40, 2.0, -3.0], np.float32)
    X = np.stack([np.full_like(bs, 3.0), bs], 1)
    P = W.stack([W.encode(["pdiv", ("x", 0), ("x", 1)]), W.encode(["plog", ("x", 1)])])
    g, st = gpu_forward(P, X)
    for i, b in enumerate(bs):
        if abs(float(b)) > float(thr):
            assert g[0, 0, i] != 1.0 or abs(3.0 / float(b) - 1.0) < 1e-5
            assert g[1, 0, i] != 0.0
        else:
            assert g[0, 0, i] == 1.0    # guard branch: exactly 1
            assert g[1, 0, i] == 0.0    # guard branch: exactly 0


def test_clamped_exp_branch():
    p = W.encode(["cexp", ("x", 0)])
    X = np.array([[79.0], [80.0], [81.0], [1e30], [np.inf], [-100.0]], np.float32)
    g, st = gpu_forward(p, X)
    e80 = np.float32(np.exp(80.0))
    assert g[0, 0, 2] == g[0, 0, 1] == g[0, 0, 3] == g[0, 0, 4]
    assert abs(float(g[0, 0, 1]) / float(e80) - 1) < 1e-5
    assert g[0, 0, 5] == 0.0 or g[0, 0, 5] < 1e-38


# ------------------------------------------------------------------ edge cases
def test_status_bit_exact_on_malformed_trees(orc):
    base = W.encode(["add", ("x", 0), "sin", ("c", 1.0)], 6)
    rows = []
    muts = [lambda t, v, s: None,
            lambda t, v, s: s.__setitem__((0, 0), 7),
            lambda t, v, s: s.__setitem__((0, 0), np.nan),
            lambda t, v, s: t.__setitem__((0, 1), 5),
            lambda t, v, s: v.__setitem__((0, 0), 5),
            lambda t, v, s: v.__setitem__((0, 0), 12),
            lambda t, v, s: v.__setitem__((0, 0), 256),
            lambda t, v, s: v.__setitem__((0, 1), 1),
            lambda t, v, s: v.__setitem__((0, 1), 0.5),
            lambda t, v, s: v.__setitem__((0, 3), np.inf),
            lambda t, v, s: s.__setitem__((0, 2), 1),
            lambda t, v, s: (t.__setitem__((0, 0), 19), v.__setitem__((0, 0), 512)),
            lambda t, v, s: (t.__setitem__((0, 1), 7), v.__setitem__((0, 0), 9)),
            lambda t, v, s: (s.__setitem__((0, 1), 0), s.__setitem__((0, 3), -1))]
    for m in muts:
        t, v, s = base.type.copy(), base.val.copy(), base.size.copy()
        m(t, v, s)
        rows.append((t, v, s))
    P = W.Population(np.concatenate([r[0] for r in rows]), np.concatenate([r[1] for r in rows]),
                     np.concatenate([r[2] for r in rows]), 6)
    X = np.random.default_rng(4).standard_normal((300, 1)).astype(np.float32)
    g, st = gpu_forward(P, X)
    ost, _ = orc.validate(P.type, P.val, P.size, 1, 1, 6)
    np.testing.assert_array_equal(st, ost)
    assert (st[1:] != 0).all() and st[0] == 0
    tv = api.tgp_validate(*dev_pop(P), n_features=1, n_outputs=1, max_len=6).cpu().numpy()
    np.testing.assert_array_equal(tv, ost)


def test_random_corruptions_status(orc):
    p = W.random_population(7, 200, 40, (1, 40), n_features=3)
    rng = np.random.default_rng(5)
    t, v, s = p.type.copy(), p.val.copy(), p.size.copy()
    for k in range(200):
        i = rng.integers(0, 40)
        which = rng.integers(0, 3)
        arr = (t, v, s)[which]
        arr[k, i] = rng.choice([0, 1, 2, 3, 18, 19, -1, 2.5, 7, 300, np.nan, rng.integers(0, 10)])
    P = W.Population(t, v, s, 40)
    X = np.random.default_rng(6).standard_normal((64, 3)).astype(np.float32)
    g, st = gpu_forward(P, X)
    ost, _ = orc.validate(t, v, s, 3, 1, 40)
    np.testing.assert_array_equal(st, ost)


def test_leaves_only_and_long_trees(orc):
    leaves = W.stack([W.encode([("x", 0)], 9), W.encode([("c", -1.25)], 9)])
    chain = W.encode(["sin"] * 1022 + [("x", 0)])                     # deepest unary chain
    full = W.random_population(9, 4, 1023, (1023, 1023), max_depth=9, n_features=2,
                               fset=(0, 1, 2, 3, 4))                  # full binary, 512 leaves
    X = np.random.default_rng(7).uniform(-1, 1, (300, 2)).astype(np.float32)
    check_forward(orc, leaves, X)
    # a chain of 1,022 sines adds the sine approximation's absolute error
    # (2^-20.9) at every link: every point stays within 2x the oracle's bound
    # but few within 1e-5, where a correctly rounded sine stays within it
    st = check_forward(orc, chain, X, floor=False)
    assert st.n >= 290, st
    p = W.Population(full.type, full.val, full.size, 1024)
    p = W.stack([p], ld=1024)
    check_forward(orc, W.Population(p.type, p.val, p.size, 1024), X)


def test_deep_modi_trees_use_every_stack_level(orc):
    # full binary Modi trees of 511 nodes need 8 register levels: three in
    # registers, the shared-memory stack entry and local-memory entries, with
    # Modi nodes (and their stack-combining forms) at every depth
    p = W.random_population(14, 6, 511, (511, 511), max_depth=8, n_features=3, n_outputs=3,
                            modi=True, modi_max=16, fset=(0, 1, 2, 3, 4))
    X = np.random.default_rng(11).uniform(-1, 1, (500, 3)).astype(np.float32)
    check_forward(orc, p, X, O=3)
    y = np.random.default_rng(12).standard_normal((500, 3)).astype(np.float32)
    m, st = gpu_mse(p, X, y, O=3)
    ref, allow, ost = orc.mse(p.type, p.val, p.size, X, y, n_outputs=3, rel_tol=1e-5)
    r = compare_mse(m, ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r


def test_deepest_modi_trees_fill_the_memory_stack(orc):
    # full binary Modi trees of 1,023 nodes need 10 levels: three in
    # registers and all seven memory-stack entries, which the Modi kernel
    # keeps in local memory
    p = W.random_population(17, 3, 1023, (1023, 1023), max_depth=9, n_features=2, n_outputs=2,
                            modi=True, modi_max=12, fset=(0, 1, 2, 3, 4))
    p = W.stack([p], ld=1024)
    p = W.Population(p.type, p.val, p.size, 1024)
    X = np.random.default_rng(13).uniform(-1, 1, (300, 2)).astype(np.float32)
    check_forward(orc, p, X, O=2)


def test_empty_population_and_points():
    p = W.random_population(3, 5, 10, n_features=2)
    X0 = np.zeros((0, 2), np.float32)
    g, st = gpu_forward(p, X0)
    assert g.shape == (5, 1, 0) and (st == 0).all()
    empty = W.Population(np.zeros((0, 10), np.float32), np.zeros((0, 10), np.float32),
                         np.zeros((0, 10), np.float32), 10)
    t, v, s = dev_pop(empty)
    X = torch.zeros((50, 2), device=DEV)
    out, st = api.tgp_eval_forward(t, v, s, X, 1, max_len=10)
    assert out.shape == (0, 1, 50)
    y = torch.zeros((50, 1), device=DEV)
    m, st = api.tgp_fitness_mse(t, v, s, X, y, 1, max_len=10)
    assert m.shape == (0, 1)


@pytest.mark.parametrize("cfg", [None, {"trees_per_block": 3, "points_per_tile": 256}])
def test_multi_output_modi_population(orc, cfg):
    prob = W.modi(pop=150, D=2000)
    p = prob.pop
    check_forward(orc, p, prob.X, O=8, config=cfg)
    y = np.random.default_rng(8).standard_normal((2000, 8)).astype(np.float32)
    m, st = gpu_mse(p, prob.X, y, O=8, config=cfg)
    ref, allow, ost = orc.mse(p.type, p.val, p.size, prob.X, y, n_outputs=8, rel_tol=1e-5)
    r = compare_mse(m, ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r


def test_single_output_with_modi_nodes(orc):
    # one output, a mix of plain trees (root value) and Modi trees (sums)
    plain = W.random_population(12, 30, 63, n_features=3)
    modi = W.random_population(13, 30, 63, (5, 63), n_features=3, n_outputs=1, modi=True, modi_max=4)
    P = W.stack([plain, modi])
    X = np.random.default_rng(9).standard_normal((700, 3)).astype(np.float32)
    check_forward(orc, P, X, O=1)
    check_forward(orc, plain, X, O=1)


def test_repeatable_bitwise():
    prob = W.sr_small()
    y = np.random.default_rng(10).standard_normal((256, 1)).astype(np.float32)
    a, _ = gpu_mse(prob.pop, prob.X, y)
    b, _ = gpu_mse(prob.pop, prob.X, y)
    np.testing.assert_array_equal(a, b)


def test_widest_feature_set(orc):
    # 256 features: the 8-points-per-lane X tile does not fit in shared
    # memory, the heuristic falls back to 4 points per lane
    p = W.random_population(15, 20, 63, (1, 63), max_depth=6, n_features=256)
    X = np.random.default_rng(13).standard_normal((700, 256)).astype(np.float32)
    check_forward(orc, p, X)
    y = np.random.default_rng(14).standard_normal((700, 1)).astype(np.float32)
    m, st = gpu_mse(p, X, y)
    ref, allow, ost = orc.mse(p.type, p.val, p.size, X, y, rel_tol=1e-5)
    r = compare_mse(m, ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r


def test_sixteen_outputs_and_single_point(orc):
    # the largest number of outputs, and a data set of one point
    p = W.random_population(16, 40, 127, (5, 127), max_depth=8, n_features=3, n_outputs=16,
                            modi=True, modi_max=20)
    X = np.random.default_rng(15).uniform(-1, 1, (600, 3)).astype(np.float32)
    check_forward(orc, p, X, O=16)
    y = np.random.default_rng(16).standard_normal((600, 16)).astype(np.float32)
    m, st = gpu_mse(p, X, y, O=16)
    ref, allow, ost = orc.mse(p.type, p.val, p.size, X, y, n_outputs=16, rel_tol=1e-5)
    r = compare_mse(m.ravel(), ref.ravel(), allow.ravel())
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
    q = W.random_population(17, 30, 63, n_features=2)
    X1 = np.array([[0.25, -0.5]], np.float32)
    check_forward(orc, q, X1)
