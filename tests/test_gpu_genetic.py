"""GPU parity of the genetic operators against the oracle (bit-exact: every
output is a copied element, an exact size update, an index or a count).

Covers the subtree exchange in its three node-choice modes (crossover,
subtree mutation, hoist) with operator probabilities, explicit positions,
bad indices and malformed trees, ragged child counts and row widths, the
full-size 100,000-child crossover on sampled rows, tournament selection with
ties / NaN / infinities, and classification accuracy (from outputs and fused
with the forward kernels, including the chunked path) on data of the paper's
classification shapes.  The last test runs one whole generation (fitness ->
selection -> crossover -> mutation) eagerly and from a captured CUDA graph.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_17168_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_17168_gb300 import build
    build.build_all()
    _lib.load()


@pytest.fixture(scope="module")
def gen(orc):
    from oracle import genetic
    return genetic


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _w(a):
    """uint32 words as the int32 device tensor the binding takes."""
    return _dev(np.asarray(a, np.uint32).view(np.int32))


def _pop(p):
    return tuple(_dev(a) for a in (p.type, p.val, p.size))


def _np(t):
    return t.cpu().numpy()


def _same(a, b):
    return np.array_equal(np.asarray(a, np.float32), np.asarray(b, np.float32), equal_nan=True)


def _run(gen, old, donor, oi, k, di, j, mode, max_size, out_ld, aw=None, ab=0):
    (t, v, z), st = api.tgp_subtree_exchange(
        _pop(old), _dev(oi), _w(k), donor=_pop(donor) if donor is not None else None,
        donor_index=_dev(di) if di is not None else None,
        donor_node=_w(j) if j is not None else None, mode=mode, max_size=max_size, out_ld=out_ld,
        apply_word=_w(aw) if aw is not None else None, apply_below=ab, old_max_len=old.max_len,
        donor_max_len=donor.max_len if donor is not None else None)
    torch.cuda.synchronize()
    ref = gen.subtree_exchange((old.type, old.val, old.size),
                               (donor.type, donor.val, donor.size) if donor is not None else None,
                               oi, k, di, j, mode, max_size, out_ld, old.max_len,
                               donor.max_len if donor is not None else None, aw, ab)
    return (_np(t), _np(v), _np(z), _np(st)), ref


def _check(got, ref):
    for g, r, name in zip(got, ref, ("type", "value", "size", "status")):
        assert _same(g, r), f"{name} differs on {np.count_nonzero(~((g == r) | (np.isnan(g) & np.isnan(r))))} elements"


def test_exchange_modes_match_oracle(gen):
    g = W.genetic(1, pop=1500, max_size=200, len_range=(1, 199), n=3001, pool=300, pool_len=(1, 15))
    P = g.pop
    # one-point crossover between two parents of the population
    got, ref = _run(gen, P, P, g.old_index, g.node, g.donor_index, g.donor_node, _lib.PICK_RANDOM,
                    200, 203)
    _check(got, ref)
    st = got[3]
    assert (st == _lib.XCHG_DONE).sum() > 1000 and (st == _lib.XCHG_TOO_LARGE).sum() > 50
    # subtree mutation from the pool of new trees, with probability 0.1
    thr = int(0.1 * 2 ** 32)
    got, ref = _run(gen, P, g.pool, g.old_index, g.node, g.pool_index, None, _lib.PICK_RANDOM, 200,
                    200, g.apply, thr)
    _check(got, ref)
    assert 200 < (got[3] == _lib.XCHG_DONE).sum() < 400
    # hoist mutation
    got, ref = _run(gen, P, None, g.old_index, g.node, None, g.donor_node, _lib.PICK_HOIST, 200, 257)
    _check(got, ref)
    assert (got[3] == _lib.XCHG_DONE).all()
    # explicit positions, some out of range
    k = (g.node % 260).astype(np.uint32)
    j = (g.donor_node % 40).astype(np.uint32)
    got, ref = _run(gen, P, g.pool, g.old_index, k, g.pool_index, j, _lib.PICK_NODES, 200, 200)
    _check(got, ref)
    assert (got[3] == _lib.XCHG_BAD_INDEX).sum() > 100


def test_exchange_edge_cases(gen):
    leaf = W.encode([("x", 0)], 8)
    small = W.stack([leaf, W.encode(["sin", ("x", 1)], 8), W.encode(["add", ("x", 0), ("c", 1.0)], 8)])
    bad = W.Population(small.type.copy(), small.val.copy(), small.size.copy(), 8)
    bad.size[1, 0] = np.nan           # no length
    bad.size[2, 1] = 7.0              # subtree runs past the tree
    bad.size[2, 2] = 1.5              # not an integer
    oi = np.array([0, 1, 2, 3, -1, 2, 0, 1, 2], np.int32)
    di = np.array([0, 0, 0, 0, 0, 2, 2, 2, 5], np.int32)
    k = np.array([0, 0, 1, 0, 0, 2, 0, 1, 0], np.uint32)
    j = np.array([0, 0, 0, 0, 0, 0, 0, 0, 0], np.uint32)
    for max_size in (1, 2, 3, 8):
        for old, donor in ((small, small), (bad, small), (small, bad)):
            got, ref = _run(gen, old, donor, oi, k, di, j, _lib.PICK_NODES, max_size, 8)
            _check(got, ref)
    # no children, and trees of the largest supported length
    (t, v, z), st = api.tgp_subtree_exchange(_pop(small), _dev(np.zeros(0, np.int32)),
                                             _w(np.zeros(0, np.uint32)), donor=_pop(small),
                                             donor_index=_dev(np.zeros(0, np.int32)), max_size=8)
    assert st.numel() == 0
    big = W.random_population(3, 64, 1024, (900, 1024), max_depth=20, n_features=3)
    g = np.random.default_rng(0)
    n = 97
    oi = g.integers(0, 64, n).astype(np.int32)
    got, ref = _run(gen, big, big, oi, W.random_words(4, n), oi[::-1].copy(), W.random_words(5, n),
                    _lib.PICK_RANDOM, 1024, 1024)
    _check(got, ref)


def test_exchange_full_size_sampled(gen):
    """The benchmark's crossover: 100,000 children of trees up to 512 nodes."""
    g = W.genetic(0)
    P = g.pop
    (t, v, z), st = api.tgp_subtree_exchange(
        _pop(P), _dev(g.old_index), _w(g.node), donor=_pop(P), donor_index=_dev(g.donor_index),
        donor_node=_w(g.donor_node), mode=_lib.PICK_RANDOM, max_size=512, out_ld=512)
    torch.cuda.synchronize()
    idx = np.random.default_rng(1).choice(g.n, 600, replace=False)
    idx = np.concatenate([idx, [0, g.n - 1]])
    ref = gen.subtree_exchange((P.type, P.val, P.size), (P.type, P.val, P.size), g.old_index[idx],
                               g.node[idx], g.donor_index[idx], g.donor_node[idx], _lib.PICK_RANDOM,
                               512, 512)
    got = (_np(t[idx]), _np(v[idx]), _np(z[idx]), _np(st[idx]))
    _check(got, ref)
    # every child is valid and as long as its status says
    s = _np(st)
    assert set(np.unique(s)) <= {_lib.XCHG_DONE, _lib.XCHG_TOO_LARGE}
    vs = api.tgp_validate(t, v, z, 16, 1, max_len=512)
    assert int((vs != 0).sum()) == 0
    keep = s == _lib.XCHG_TOO_LARGE
    lens = _np(z[:, 0])
    assert (lens[keep] == P.size[g.old_index[keep], 0]).all()


def test_tournament_matches_oracle(gen):
    rng = np.random.default_rng(2)
    for P, t, n, spread in ((1, 20, 5, 0), (37, 1, 100, 0), (5000, 20, 10001, 0),
                            (500, 33, 999, 3), (200, 64, 515, 2), (1000, 100, 333, 0)):
        f = rng.standard_normal(P)
        if spread:
            f = rng.integers(0, spread, P).astype(np.float64)
        f[rng.random(P) < 0.1] = np.nan
        f[rng.random(P) < 0.05] = np.inf
        f[rng.random(P) < 0.05] = -np.inf
        words = W.random_words(P, (n, t))
        for mn in (True, False):
            got = api.tgp_tournament_select(_dev(f), _w(words), mn)
            assert (_np(got) == gen.tournament(f, words, mn)).all(), (P, t, mn)
    # a column of an MSE matrix (stride 2)
    m = rng.standard_normal((300, 2))
    words = W.random_words(9, (256, 20))
    got = api.tgp_tournament_select(_dev(m)[:, 1], _w(words))
    assert (_np(got) == gen.tournament(m[:, 1], words)).all()


def test_accuracy_from_outputs_matches_oracle(gen):
    rng = np.random.default_rng(3)
    for P, C, D in ((1, 1, 1), (7, 3, 178), (64, 10, 1484), (3, 16, 70000)):
        out = rng.integers(-3, 4, (P, C, D)).astype(np.float32)
        out[rng.random((P, C, D)) < 0.1] = np.nan
        out[rng.random((P, C, D)) < 0.02] = -np.inf
        out[:, :, :5] = np.nan
        lab = rng.integers(0, C, D).astype(np.int32)
        acc, cnt = api.tgp_accuracy_from_outputs(_dev(out), _dev(lab))
        racc, rcnt = gen.accuracy_from_outputs(out, lab)
        assert (_np(cnt) == rcnt).all() and (_np(acc) == racc).all()


@pytest.mark.parametrize("shape,pop,D", [("wine", 200, None), ("kidney", 300, None),
                                         ("breast", 100, None), ("yeast", 1000, None),
                                         ("yeast", 1700, 4700)])
def test_fitness_accuracy_matches_oracle(gen, shape, pop, D):
    # the last case (1700 trees x 10 classes x 4700 points, 320 MB of outputs)
    # takes the chunked path: two forward chunks of 3840 and 860 points
    prob = W.classification(0, shape, pop=pop, max_len=63, D=D)
    p = prob.pop
    acc, cnt, st = api.tgp_fitness_accuracy(*_pop(p), _dev(prob.X), _dev(prob.labels),
                                            prob.n_classes, max_len=p.max_len)
    torch.cuda.synchronize()
    racc, rcnt, amb, rst = gen.accuracy(p.type, p.val, p.size, prob.X, prob.labels,
                                        prob.n_classes, max_len=p.max_len)
    assert (_np(st) == rst).all()
    c = _np(cnt)
    ok = rst == 0
    assert (np.abs(c - rcnt)[ok] <= amb[ok]).all()
    assert np.mean(c[ok] == rcnt[ok]) > 0.8
    a = _np(acc)
    assert np.isnan(a[~ok]).all() and (a[ok] == c[ok] / prob.X.shape[0]).all()


def test_generation_graph_matches_eager_and_oracle(gen, orc):
    from paper_2501_17168_gb300 import evolve
    g = W.genetic(5, pop=256, max_size=512, len_range=(1, 63), pool=64, pool_len=(1, 15),
                  n_features=2)
    X = np.random.default_rng(5).uniform(-2, 2, (1000, 2)).astype(np.float32)
    gt = W.encode(["add", "mul", ("x", 0), ("x", 0), "sin", ("x", 1)])
    y, _ = orc.evaluate(gt.type, gt.val, gt.size, X)
    y = y[0, 0].astype(np.float32)[:, None]
    start = _pop(g.pop)
    torch.manual_seed(0)
    state = evolve.Generation(tuple(a.clone() for a in start), _dev(X), _dev(y), _pop(g.pool))
    state.step()                      # warm-up: allocates the cached workspace
    torch.cuda.synchronize()
    # capture one generation and replay it from the start population
    for a, b in zip(state.pop, start):
        a.copy_(b)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        state.step()
    for a, b in zip(state.pop, start):
        a.copy_(b)
    graph.replay()
    torch.cuda.synchronize()
    g_pop = [_np(a) for a in state.pop]
    g_mse, g_win = _np(state.mse)[:, 0], _np(state.winners)
    words = _np(state.words).view(np.uint32)
    pool_index = _np(state.pool_index)
    # eager recomputation with the graph's own random words
    for a, b in zip(state.pop, start):
        a.copy_(b)
    state.apply()
    torch.cuda.synchronize()
    for a, b in zip(state.pop, g_pop):
        assert _same(_np(a), b)
    # the oracle's generation on the same words
    P, t = 256, state.t
    pop0 = (g.pop.type, g.pop.val, g.pop.size)
    rmse, allow, _ = orc.mse(*pop0, X, y, rel_tol=1e-5, max_len=512)
    rmse = rmse[:, 0]
    wt = words[:2 * P * t].reshape(2 * P, t)
    k1, j1, a1, k2, a2 = (words[2 * P * t + i * P:2 * P * t + (i + 1) * P] for i in range(5))
    rwin = gen.tournament(rmse, wt)
    # winners may differ only between trees whose fitness the FP32 path cannot order
    with np.errstate(all="ignore"):
        tol = 1e-4 * np.maximum(np.abs(rmse[rwin]), np.abs(rmse[g_win])) + allow[rwin, 0] + allow[g_win, 0]
        tied = (np.abs(rmse[rwin] - rmse[g_win]) <= tol) | (~np.isfinite(rmse[rwin]) & ~np.isfinite(rmse[g_win]))
    diff = rwin != g_win
    assert (tied[diff]).all() and diff.mean() < 0.05
    fin = np.isfinite(allow[:, 0]) & (rmse < 1e30)
    assert (np.abs(g_mse - rmse)[fin] <= 1e-4 * np.abs(rmse[fin]) + allow[fin, 0]).all()
    c = gen.subtree_exchange(pop0, pop0, rwin[:P], k1, rwin[P:], j1, gen.RANDOM, 512, 512, 512, 512,
                             a1, state.thr_cross)
    m = gen.subtree_exchange(c[:3], (g.pool.type, g.pool.val, g.pool.size), np.arange(P), k2,
                             pool_index, None, gen.RANDOM, 512, 512, 512, g.pool.max_len, a2,
                             state.thr_mut)
    same = ~diff[:P] & ~diff[P:]
    for a, b in zip(g_pop, m[:3]):
        assert _same(a[same], b[same])
    assert same.mean() > 0.9
