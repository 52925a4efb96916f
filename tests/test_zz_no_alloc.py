"""tgp_fitness_mse_noalloc -- the fitness call for callers that cannot
allocate device memory (for example a plain C host without a device
allocator, or a plugin whose host application owns all device memory).

It is called here through the C ABI and must give the same statuses and MSE
values as tgp_fitness_mse with a caller workspace, on two calls in a row
(the scratch array is reused and must be cleared where it matters).  This
file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_17168_gb300 import _lib, api, build, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def lib():
    build.build_all()
    return _lib.load()


def _noalloc(lib, t, v, s, X, y, O, max_len):
    pop = api.make_population(t, v, s, max_len)
    data = api.make_data(X)
    mse = torch.full((pop.pop, O), -1.0, dtype=torch.float64, device=DEV)
    st = torch.full((pop.pop,), -1, dtype=torch.int32, device=DEV)
    rc = lib.tgp_fitness_mse_noalloc(ctypes.byref(pop), ctypes.byref(data), y.data_ptr(), O,
                                     mse.data_ptr(), st.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    return rc, mse, st


def _same(a, b):
    """Bit-equal up to NaN payloads: both calls run the same kernels in the
    same launch shape with fixed-order reductions, so any difference (a stale
    value left in the shared scratch included) is a fault."""
    a, b = a.cpu().numpy(), b.cpu().numpy()
    both_nan = np.isnan(a) & np.isnan(b)
    return bool((both_nan | (a.view(np.int64) == b.view(np.int64))).all())


def test_noalloc_matches_workspace_call_twice(lib):
    problems = []
    p = W.random_population(41, 300, 127, n_features=5)
    t = list(p.type); t[7][0] = 9.0                          # one malformed tree
    p = W.Population(np.stack(t), p.val, p.size, 127)
    X = np.random.default_rng(1).standard_normal((3000, 5)).astype(np.float32)
    y = np.random.default_rng(2).standard_normal((3000, 1)).astype(np.float32)
    problems.append((p, X, y, 1))
    m = W.modi(pop=120, D=1500, n_outputs=4)
    y4 = np.random.default_rng(3).standard_normal((1500, 4)).astype(np.float32)
    problems.append((m.pop, m.X, y4, 4))
    for call in range(2):
        for pop, Xn, yn, O in problems:
            tt, vv, ss = api.population_to(pop, DEV)
            Xd = torch.from_numpy(Xn).to(DEV)
            yd = torch.from_numpy(yn).to(DEV)
            ref, st_ref = api.tgp_fitness_mse(tt, vv, ss, Xd, yd, O, max_len=pop.max_len)
            rc, mse, st = _noalloc(lib, tt, vv, ss, Xd, yd, O, pop.max_len)
            torch.cuda.synchronize()
            assert rc == _lib.TGP_OK, lib.tgp_status_string(rc)
            # the no-allocation call's own error word (no bounded wait gave up)
            rc = lib.tgp_check_device_error_noalloc(torch.cuda.current_stream().cuda_stream)
            assert rc == _lib.TGP_OK, lib.tgp_status_string(rc)
            assert torch.equal(st, st_ref)
            assert _same(mse, ref), (call, O)


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    # 20,000 trees of up to 255 nodes need about 41 MB of programs alone
    P, L = 20000, 255
    t = torch.zeros((P, L), device=DEV)
    v = torch.zeros((P, L), device=DEV)
    s = torch.ones((P, L), device=DEV)
    X = torch.zeros((10, 1), device=DEV)
    y = torch.zeros((10, 1), device=DEV)
    assert api.tgp_workspace_size(t, v, s, X, 1) > _lib.NOALLOC_WS_BYTES
    rc, mse, st = _noalloc(lib, t, v, s, X, y, 1, L)
    torch.cuda.synchronize()
    assert rc == _lib.TGP_ERR_WORKSPACE
    assert (st == -1).all()          # nothing was launched
