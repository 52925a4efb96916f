"""The C ABI's call options on the GPU: the bounded wait's timeout path
(driven by a poll limit, without any fault), the SSE mode whose point-sharded
partial sums add up to the whole data set's MSE, and the batch plan that is
built once on the host (with the autotuner's cache) and run or replayed many
times."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_17168_gb300 import _lib, api, autotune, workloads as W
from parity import compare_mse

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_17168_gb300 import build
    build.build_all()
    _lib.load()


def _bits_equal(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    if a.shape != b.shape or a.dtype != b.dtype:
        return False
    iv = np.int64 if a.dtype == np.float64 else np.int32
    both_nan = np.isnan(a) & np.isnan(b)
    return bool((both_nan | (a.view(iv) == b.view(iv))).all())


def _problem(seed=3, P=150, D=5000, F=6):
    p = W.random_population(seed, P, 127, (1, 127), max_depth=8, n_features=F)
    X = np.random.default_rng(seed).standard_normal((D, F)).astype(np.float32)
    y = np.random.default_rng(seed + 1).standard_normal((D, 1)).astype(np.float32)
    t, v, s = api.population_to(p, DEV)
    return p, X, y, (t, v, s, torch.from_numpy(X).to(DEV), torch.from_numpy(y).to(DEV))


def test_bounded_wait_timeout_is_reported_and_the_next_call_is_exact():
    """A negative poll limit makes every CTA give up its wait for the program
    copies at once: the CTA-uniform exit returns every thread together after
    the copies land, the error word reports TGP_ERR_TIMEOUT, and the next
    normal call on the same workspace gives the normal results bit for bit."""
    p, X, y, (t, v, s, Xd, yd) = _problem()
    ref, st_ref = api.tgp_fitness_mse(t, v, s, Xd, yd, 1, max_len=127)
    api.tgp_check_device_error()
    torch.cuda.synchronize()
    for cfg in ({"max_wait_polls": -1}, {"max_wait_polls": -1, "trees_per_block": 2,
                                          "points_per_tile": 512}):
        api.tgp_fitness_mse(t, v, s, Xd, yd, 1, max_len=127, config=cfg)
        with pytest.raises(_lib.TGPError) as e:
            api.tgp_check_device_error()
        assert e.value.code == _lib.TGP_ERR_TIMEOUT
        api.tgp_check_device_error()          # the word was cleared by the read
    m2, st2 = api.tgp_fitness_mse(t, v, s, Xd, yd, 1, max_len=127)
    api.tgp_check_device_error()
    assert torch.equal(st2, st_ref)
    assert _bits_equal(m2, ref)
    # the forward path takes the same exit
    out_ref, _ = api.tgp_eval_forward(t, v, s, Xd, 1, max_len=127)
    api.tgp_eval_forward(t, v, s, Xd, 1, max_len=127, config={"max_wait_polls": -1})
    with pytest.raises(_lib.TGPError):
        api.tgp_check_device_error()
    out2, _ = api.tgp_eval_forward(t, v, s, Xd, 1, max_len=127)
    api.tgp_check_device_error()
    assert _bits_equal(out2, out_ref)


def test_sse_mode_point_shards_add_up_to_the_mse(orc):
    """TGP_FLAG_SSE returns the FP64 sum of squared residuals; the sums over
    disjoint point ranges add up to D times the whole set's MSE (up to the
    order of the additions), and match the oracle's SSE."""
    p, X, y, (t, v, s, Xd, yd) = _problem(seed=5, P=120, D=7001)
    D = X.shape[0]
    full, st = api.tgp_fitness_mse(t, v, s, Xd, yd, 1, max_len=127)
    whole_sse, _ = api.tgp_fitness_mse(t, v, s, Xd, yd, 1, max_len=127, config={"sse": True})
    torch.cuda.synchronize()
    ok = (st == 0).cpu().numpy()
    fm, ws_ = full.cpu().numpy()[:, 0], whole_sse.cpu().numpy()[:, 0]
    fin = ok & np.isfinite(fm)
    np.testing.assert_allclose(ws_[fin], fm[fin] * D, rtol=1e-13)
    parts = []
    for a, b in ((0, 2500), (2500, 2501), (2501, D)):
        m, _ = api.tgp_fitness_mse(t, v, s, Xd[a:b].contiguous(), yd[a:b].contiguous(), 1, max_len=127,
                                   config={"sse": True})
        parts.append(m.cpu().numpy()[:, 0])
    comb = sum(parts) / D
    with np.errstate(invalid="ignore"):
        rel = np.abs(comb - fm) / np.maximum(np.abs(fm), 1e-300)
    # FP32 chunk sums differ with the point partition: a few ulps of FP32
    assert (rel[fin & (fm < 1e30)] <= 1e-5).all(), np.nanmax(rel[fin & (fm < 1e30)])
    assert np.isnan(comb[~ok]).all()
    ref, allow, _ = orc.mse(p.type, p.val, p.size, X, y, rel_tol=1e-5)
    r = compare_mse(comb[:, None], ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r


def _bp(prob, y, config=None):
    t, v, s = api.population_to(prob.pop, DEV)
    return api.BatchProblem(t, v, s, torch.from_numpy(prob.X).to(DEV), torch.from_numpy(y).to(DEV), 1,
                            max_len=prob.pop.max_len, config=config)


def test_batch_plan_reads_the_tune_cache_and_replays(orc, tmp_path):
    probs = W.batched_uneven(seed=2, n_problems=4, scale=0.02)
    ys = []
    for pr in probs:
        out, _ = orc.evaluate(pr.gt.type, pr.gt.val, pr.gt.size, pr.X)
        ys.append((out[0, 0] + pr.noise[:, 0]).astype(np.float32)[:, None])
    bps = [_bp(pr, y) for pr, y in zip(probs, ys)]
    # a cache entry for problems 0 and 2 (a population-parallel and a
    # data-parallel shape), none for 1 and 3
    name = torch.cuda.get_device_name(0)
    shapes = {0: {"trees_per_block": 16, "points_per_tile": 256, "tiles_per_item": 1,
                  "points_per_lane": 8},
              2: {"trees_per_block": 1, "points_per_tile": 2048, "tiles_per_item": 2,
                  "points_per_lane": 8}}
    path = str(tmp_path / "tune.txt")
    autotune.store({autotune.key(name, probs[i].pop.pop, probs[i].D, probs[i].F, 1, probs[i].pop.max_len):
                    (sh, 1.0) for i, sh in shapes.items()}, path)
    plan = api.BatchPlan(bps, tune_cache=path)
    for i in range(4):
        sh, fc = plan.shape(i)
        assert fc == (i in shapes), (i, sh)
        if i in shapes:
            assert sh["trees_per_block"] == shapes[i]["trees_per_block"]
            assert sh["points_per_tile"] == shapes[i]["points_per_tile"]
    plan.run()
    torch.cuda.synchronize()
    plan.check_device_error()
    first = [bp.mse.clone() for bp in bps]
    # each problem equals its own call in the plan's shape, bit for bit
    for i, (pr, bp) in enumerate(zip(probs, bps)):
        t, v, s, X, yd = bp.tensors
        cfg = shapes.get(i)
        if cfg is not None:
            ref, st = api.tgp_fitness_mse(t, v, s, X, yd, 1, max_len=pr.pop.max_len, config=cfg)
            assert _bits_equal(ref, bp.mse), i
        sel = np.arange(0, pr.pop.pop, max(1, pr.pop.pop // 20))
        sub = pr.pop.take(sel)
        ref, allow, _ = orc.mse(sub.type, sub.val, sub.size, pr.X, ys[i], rel_tol=1e-5)
        r = compare_mse(bp.mse.cpu().numpy()[sel], ref, allow)
        assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, (i, r)
    # the same batch through the one-shot call with the same shapes
    bps2 = [_bp(pr, y, config=shapes.get(i)) for i, (pr, y) in enumerate(zip(probs, ys))]
    api.tgp_batch_fitness_mse(bps2)
    for a, b in zip(first, bps2):
        assert _bits_equal(a, b.mse)
    # captured once, replayed: results follow new data in the same buffers
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.run()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run()
    for bp in bps:
        bp.mse.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    for a, bp in zip(first, bps):
        assert _bits_equal(a, bp.mse)
    for bp in bps:
        bp.tensors[4].mul_(0.5)
    g.replay()
    plan.run()
    torch.cuda.synchronize()
    for i, (pr, bp) in enumerate(zip(probs, bps)):
        t, v, s, X, yd = bp.tensors
        cfg = shapes.get(i)
        if cfg is not None:
            ref, _ = api.tgp_fitness_mse(t, v, s, X, yd, 1, max_len=pr.pop.max_len, config=cfg)
            assert _bits_equal(ref, bp.mse)
    plan.close()


def test_batch_plan_without_cache_equals_one_shot_batch():
    probs = W.batched_uneven(seed=4, n_problems=3, scale=0.01)
    ys = [np.random.default_rng(i).standard_normal((pr.D, 1)).astype(np.float32)
          for i, pr in enumerate(probs)]
    bps = [_bp(pr, y) for pr, y in zip(probs, ys)]
    plan = api.BatchPlan(bps, tune_cache=os.devnull)
    assert not any(plan.shape(i)[1] for i in range(3))
    plan.run()
    torch.cuda.synchronize()
    first = [bp.mse.clone() for bp in bps]
    api.tgp_batch_fitness_mse(bps)
    torch.cuda.synchronize()
    for a, bp in zip(first, bps):
        assert _bits_equal(a, bp.mse)


def test_cta_width_option(orc):
    """cta_width picks the narrow CTAs (1) or one wide CTA per SM (2) for the
    single-output and the Modi kernel: the per-point outputs are the same
    bits (same interpreter, same points per lane), the MSE agrees up to the
    FP64 summation order of the tiles, and other values are refused."""
    p, X, y, (t, v, s, Xd, yd) = _problem(seed=21, P=200, D=6000)
    outs, mses = [], []
    for w in (0, 1, 2):
        o, _ = api.tgp_eval_forward(t, v, s, Xd, 1, max_len=p.max_len, config={"cta_width": w})
        m, st = api.tgp_fitness_mse(t, v, s, Xd, yd, 1, max_len=p.max_len, config={"cta_width": w})
        outs.append(o)
        mses.append(m.cpu().numpy())
    assert _bits_equal(outs[0], outs[1]) and _bits_equal(outs[0], outs[2])
    np.testing.assert_allclose(mses[1], mses[0], rtol=1e-12, atol=0)
    np.testing.assert_allclose(mses[2], mses[0], rtol=1e-12, atol=0)
    m = W.random_population(22, 80, 63, (9, 63), max_depth=6, n_features=6, n_outputs=3, modi=True,
                            modi_max=6)
    tm, vm, sm = api.population_to(m, DEV)
    y3 = torch.from_numpy(np.random.default_rng(23).standard_normal((6000, 3)).astype(np.float32)).to(DEV)
    got = [api.tgp_fitness_mse(tm, vm, sm, Xd, y3, 3, max_len=63, config={"cta_width": w})[0].cpu().numpy()
           for w in (1, 2)]
    np.testing.assert_allclose(got[1], got[0], rtol=1e-12, atol=0)
    ref, allow, _ = orc.mse(m.type, m.val, m.size, X, y3.cpu().numpy(), n_outputs=3, rel_tol=1e-5)
    r = compare_mse(got[1], ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
    with pytest.raises(_lib.TGPError) as e:
        api.tgp_fitness_mse(t, v, s, Xd, yd, 1, max_len=p.max_len, config={"cta_width": 3})
    assert e.value.code == _lib.TGP_ERR_INVALID_ARG
