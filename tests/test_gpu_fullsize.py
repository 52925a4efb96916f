"""Full-size GPU parity on sampled trees, in the launch shapes the benchmark
uses: the differentiation workload (10,000 trees x 200,000 points, fused MSE
and gradients), the Modi workload (20,000 trees x 1,000,000 points x 8
outputs) and the batched uneven workload (8 problems in one batched call).

The oracle cannot evaluate whole populations at these sizes, so each test
runs the full GPU call and checks a sample of trees against the oracle; for
the adjoint, the upstream gradient is non-zero only on the sampled trees,
which makes the X gradient (a sum over trees) checkable as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_17168_gb300 import _lib, api, workloads as W
from parity import compare_mse

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_17168_gb300 import build
    build.build_all()
    _lib.load()


def _targets(orc, prob):
    ys = []
    for k in range(prob.gt.pop):
        g = prob.gt.take([k])
        out, _ = orc.evaluate(g.type, g.val, g.size, prob.X)
        ys.append(out[0, 0])
    return (np.stack(ys, 1) + prob.noise.astype(np.float64)).astype(np.float32)


def test_diff_full_size_adjoint_sampled(orc):
    prob = W.diff()
    P, D = prob.pop.pop, prob.D
    y = _targets(orc, prob)
    # over 200,000 points few deep random trees are well conditioned at every
    # point, so sample widely and keep the well-conditioned ones
    pick = np.arange(7, P, P // 240)
    sub = prob.pop.take(pick)
    # trees whose forward is ill-conditioned at some point get no upstream gradient
    out, err, st = orc.evaluate(sub.type, sub.val, sub.size, prob.X, with_err=True)
    with np.errstate(all="ignore"):
        good = (st == 0) & (np.isfinite(out) & (2 * err <= 1e-5 * np.maximum(np.abs(out), 1.0))).all(axis=(1, 2))
    assert good.sum() >= 10, good.sum()
    rng = np.random.default_rng(5)
    g_sub = rng.uniform(0.5, 1.5, (len(pick), 1)) * good[:, None]
    g = np.zeros((P, 1))
    g[pick] = g_sub
    t, v, s = api.population_to(prob.pop, DEV)
    mse, gv, gx, gst = api.tgp_eval_backward(t, v, s, torch.from_numpy(prob.X).to(DEV),
                                             torch.from_numpy(y).to(DEV),
                                             torch.from_numpy(g).to(DEV), 1, max_len=prob.pop.max_len)
    api.tgp_check_device_error()
    mse, gv, gx, gst = (x.cpu().numpy() for x in (mse, gv, gx, gst))
    rm, rgv, rgx, rst = orc.grad(sub.type, sub.val, sub.size, prob.X, y, g_sub, max_len=sub.max_len)
    np.testing.assert_array_equal(gst[pick], rst)
    # fused MSE of the sampled trees
    ref, allow, _ = orc.mse(sub.type, sub.val, sub.size, prob.X, y, rel_tol=1e-5)
    r = compare_mse(mse[pick], ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
    # constant gradients of the sampled, included trees
    const = sub.type == W.CONST
    sel = good[:, None] & const
    _check_grad(gv[pick][sel], rgv[sel])
    assert sel.sum() >= 20
    # X gradient: the sum over the sampled trees (every other tree has g = 0)
    _check_grad(gx, rgx)


def _check_grad(gpu, ref):
    """Elementwise |gpu - ref| <= 1e-3 max(|ref|, 1); a derivative chain can
    overflow although the forward values stay finite, so elements whose
    reference is non-finite or above 1e30 must be so on the GPU too."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    with np.errstate(all="ignore"):
        div_ref = ~np.isfinite(ref) | (np.abs(ref) > 1e30)
        div_gpu = ~np.isfinite(gpu) | (np.abs(gpu) > 1e30)
        assert (div_ref == div_gpu).all(), (int(div_ref.sum()), int(div_gpu.sum()))
        d = np.abs(gpu - ref)[~div_ref]
        bad = d > TOL_GRAD * np.maximum(np.abs(ref[~div_ref]), 1.0)
    assert not bad.any(), (int(bad.sum()), float(d.max()))
    assert div_ref.mean() < 0.01, float(div_ref.mean())


def test_modi_full_size_forward_sampled(orc):
    prob = W.modi()
    P, O = prob.pop.pop, prob.n_outputs
    y = _targets(orc, prob)
    t, v, s = api.population_to(prob.pop, DEV)
    m, st = api.tgp_fitness_mse(t, v, s, torch.from_numpy(prob.X).to(DEV), torch.from_numpy(y).to(DEV),
                                O, max_len=prob.pop.max_len)
    api.tgp_check_device_error()
    m, st = m.cpu().numpy(), st.cpu().numpy()
    assert (st == 0).all()
    pick = np.arange(3, P, P // 10)
    sub = prob.pop.take(pick)
    ref, allow, ost = orc.mse(sub.type, sub.val, sub.size, prob.X, y, n_outputs=O, rel_tol=1e-5)
    r = compare_mse(m[pick].ravel(), ref.ravel(), allow.ravel())
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
    assert r["n"] >= len(pick) * O // 2, r


def test_batched_uneven_full_size_sampled(orc):
    probs = W.batched_uneven(0)
    bps, ys = [], []
    for pr in probs:
        y = _targets(orc, pr)
        ys.append(y)
        t, v, s = api.population_to(pr.pop, DEV)
        bps.append(api.BatchProblem(t, v, s, torch.from_numpy(pr.X).to(DEV), torch.from_numpy(y).to(DEV), 1,
                                    max_len=pr.pop.max_len))
    api.tgp_batch_fitness_mse(bps)
    api.tgp_check_device_error()
    batched = [bp.mse.clone() for bp in bps]
    for bp, mb in zip(bps, batched):
        tt, vv, ss, Xp, yp = bp.tensors
        m1, _ = api.tgp_fitness_mse(tt, vv, ss, Xp, yp, 1, max_len=bp.pop.max_len)
        # same kernels and shapes: one call per problem gives the same bits
        assert bool(((m1 == mb) | (torch.isnan(m1) & torch.isnan(mb))).all())
    for pr, y, mb in zip(probs, ys, batched):
        pick = np.arange(1, pr.pop.pop, max(1, pr.pop.pop // 4))
        sub = pr.pop.take(pick)
        ref, allow, _ = orc.mse(sub.type, sub.val, sub.size, pr.X, y, rel_tol=1e-5)
        r = compare_mse(mb.cpu().numpy()[pick], ref, allow)
        assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, (pr.pop.pop, pr.D, r)
