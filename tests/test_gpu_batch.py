"""Batched uneven problems: one persistent launch over several populations and
datasets of different sizes gives the same results as one call per problem,
matches the oracle, mixes single-output and Modi problems, and replays
correctly from a captured CUDA graph."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_17168_gb300 import _lib, api, workloads as W
from parity import compare_mse

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_17168_gb300 import build
    build.build_all()
    _lib.load()


def _same(a, b):
    return bool(((a == b) | (torch.isnan(a) & torch.isnan(b))).all())


def _targets(orc, prob):
    out, _ = orc.evaluate(prob.gt.type, prob.gt.val, prob.gt.size, prob.X)
    return (out[0, 0] + prob.noise[:, 0]).astype(np.float32)[:, None]


def _dev(prob, y, O=1, config=None):
    t, v, s = api.population_to(prob.pop, DEV)
    return api.BatchProblem(t, v, s, torch.from_numpy(prob.X).to(DEV), torch.from_numpy(y).to(DEV), O,
                            max_len=prob.pop.max_len, config=config)


def test_batch_matches_per_problem_calls_and_oracle(orc):
    probs = W.batched_uneven(seed=0, scale=0.02)          # 8 problems, uneven P, D, F, lengths
    ys = [_targets(orc, p) for p in probs]
    bps = [_dev(p, y) for p, y in zip(probs, ys)]
    api.tgp_batch_fitness_mse(bps)
    torch.cuda.synchronize()
    api.tgp_check_device_error()
    for prob, y, bp in zip(probs, ys, bps):
        t, v, s, X, yd = bp.tensors
        ref_gpu, st = api.tgp_fitness_mse(t, v, s, X, yd, 1, max_len=prob.pop.max_len)
        np.testing.assert_array_equal(bp.mse.cpu().numpy(), ref_gpu.cpu().numpy())
        np.testing.assert_array_equal(bp.status.cpu().numpy(), st.cpu().numpy())
        sel = np.arange(0, prob.pop.pop, max(1, prob.pop.pop // 25))
        sub = prob.pop.take(sel)
        ref, allow, ost = orc.mse(sub.type, sub.val, sub.size, prob.X, y, rel_tol=1e-5)
        r = compare_mse(bp.mse.cpu().numpy()[sel], ref, allow)
        assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r


def test_batch_mixed_outputs(orc):
    a = W.sr_small(1)
    ya = _targets(orc, a)
    m = W.modi(pop=60, D=900, n_outputs=3)
    ym = np.random.default_rng(1).standard_normal((900, 3)).astype(np.float32)
    bps = [_dev(a, ya), _dev(m, ym, O=3)]
    api.tgp_batch_fitness_mse(bps)
    torch.cuda.synchronize()
    ref, allow, _ = orc.mse(m.pop.type, m.pop.val, m.pop.size, m.X, ym, n_outputs=3, rel_tol=1e-5)
    r = compare_mse(bps[1].mse.cpu().numpy(), ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
    ref, allow, _ = orc.mse(a.pop.type, a.pop.val, a.pop.size, a.X, ya, rel_tol=1e-5)
    r = compare_mse(bps[0].mse.cpu().numpy(), ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r


def test_batch_graph_capture_replay(orc):
    probs = W.batched_uneven(seed=1, n_problems=4, scale=0.01)
    ys = [_targets(orc, p) for p in probs]
    bps = [_dev(p, y) for p, y in zip(probs, ys)]
    n = api.tgp_batch_workspace_size(bps)
    ws = torch.empty(n, dtype=torch.uint8, device=DEV)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.tgp_batch_fitness_mse(bps, ws=ws)          # warm-up: kernel attributes set outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    first = [bp.mse.clone() for bp in bps]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        api.tgp_batch_fitness_mse(bps, ws=ws)
    for bp in bps:
        bp.mse.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    for a, bp in zip(first, bps):
        assert _same(a, bp.mse)
    # new data in the same buffers, replay again: results follow the data
    for bp in bps:
        bp.tensors[4].mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    for bp, prob in zip(bps, probs):
        t, v, s2, X, yd = bp.tensors
        ref, _ = api.tgp_fitness_mse(t, v, s2, X, yd, 1, max_len=prob.pop.max_len)
        assert _same(ref, bp.mse)


def test_batch_rejects_bad_arguments():
    p = W.sr_small(2)
    y = np.zeros((256, 1), np.float32)
    bp = _dev(p, y)
    assert _lib.load().tgp_batch_workspace_size(None, 1) == 0
    with pytest.raises(_lib.TGPError):
        api.tgp_batch_fitness_mse([bp] * 17)


def test_batch_of_mixed_cta_widths(orc):
    """A Modi problem whose sixteen output rows per warp cramp the wide CTA
    and a small Modi problem that fits it run in one batch: each keeps the
    kernel and shape it gets alone (the batch launches one persistent kernel
    per kernel and occupancy group), so each MSE has the bits of its own
    call, and matches the oracle."""
    rng = np.random.default_rng(41)
    wide = W.random_population(42, 60, 63, (5, 63), max_depth=6, n_features=96, n_outputs=16,
                               modi=True, modi_max=20, fset=(W.ADD, W.SUB, W.MUL, W.SIN))
    small = W.random_population(43, 50, 31, (5, 31), max_depth=5, n_features=3, n_outputs=2,
                                modi=True, modi_max=4, fset=(W.ADD, W.MUL, W.COS))
    cases = [(wide, rng.standard_normal((3000, 96)).astype(np.float32), 16),
             (small, rng.uniform(-1, 1, (2000, 3)).astype(np.float32), 2)]
    bps, ys = [], []
    for p, X, O in cases:
        y = rng.standard_normal((X.shape[0], O)).astype(np.float32)
        t, v, s = api.population_to(p, DEV)
        bps.append(api.BatchProblem(t, v, s, torch.from_numpy(X).to(DEV), torch.from_numpy(y).to(DEV), O,
                                    max_len=p.max_len))
        ys.append(y)
    api.tgp_batch_fitness_mse(bps)
    torch.cuda.synchronize()
    api.tgp_check_device_error()
    for (p, X, O), y, bp in zip(cases, ys, bps):
        t, v, s, Xd, yd = bp.tensors
        one, st = api.tgp_fitness_mse(t, v, s, Xd, yd, O, max_len=p.max_len)
        np.testing.assert_array_equal(bp.status.cpu().numpy(), st.cpu().numpy())
        assert _same(bp.mse, one)
        ref, allow, ost = orc.mse(p.type, p.val, p.size, X, y, n_outputs=O, rel_tol=1e-5)
        r = compare_mse(bp.mse.cpu().numpy(), ref, allow)
        assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
