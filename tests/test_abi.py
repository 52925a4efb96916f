"""The C ABI library: builds for sm_103a, loads, exports every entry point
declared in include/tgp.h, and rejects bad arguments on the host before any
device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2501_17168_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "tgp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tgp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("tgp_eval_forward", "tgp_fitness_mse", "tgp_validate", "tgp_workspace_size",
              "tgp_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_declares_every_header_symbol():
    assert set(_declared()) <= set(_lib.declared_symbols())


def test_status_strings(lib):
    assert lib.tgp_status_string(0) == b"TGP_OK"
    assert lib.tgp_status_string(3) == b"TGP_ERR_WORKSPACE"
    assert b"sm_103a" in lib.tgp_version()


def test_host_argument_checks_need_no_device(lib):
    P = ctypes.POINTER
    pop = _lib.tgp_population(None, None, None, 4, 8, 8)      # null arrays with pop > 0
    data = _lib.tgp_data(None, 0, 1, 1)
    assert lib.tgp_fitness_mse(ctypes.byref(pop), ctypes.byref(data), None, 1, None, None, None, 0,
                               None) == _lib.TGP_ERR_INVALID_ARG
    pop = _lib.tgp_population(None, None, None, 0, 2000, 2000)  # max_len beyond the limit
    assert lib.tgp_eval_forward(ctypes.byref(pop), ctypes.byref(data), 1, None, None, None, 0,
                                None) == _lib.TGP_ERR_INVALID_ARG
    pop = _lib.tgp_population(None, None, None, 0, 8, 4)        # ld < max_len
    assert lib.tgp_workspace_size(ctypes.byref(pop), None, 1, None) == 0
    pop = _lib.tgp_population(None, None, None, 0, 8, 8)
    assert lib.tgp_validate(ctypes.byref(pop), 0, 1, None, None, 0, None) == _lib.TGP_ERR_INVALID_ARG
    assert lib.tgp_validate(ctypes.byref(pop), 1, 99, None, None, 0, None) == _lib.TGP_ERR_INVALID_ARG


def test_genetic_operator_argument_checks_need_no_device(lib):
    u32 = ctypes.c_uint32
    old = _lib.tgp_population(0x10000, 0x20000, 0x30000, 4, 8, 8)   # fake, never dereferenced
    idx, words = ctypes.c_void_p(0x40000), ctypes.c_void_p(0x50000)
    outs = [ctypes.c_void_p(0x60000), ctypes.c_void_p(0x70000), ctypes.c_void_p(0x80000)]

    def xchg(mode=_lib.PICK_RANDOM, n=2, max_size=8, out_ld=8, o=outs, donor=old):
        return lib.tgp_subtree_exchange(ctypes.byref(old), ctypes.byref(donor), idx, words, idx,
                                        words, None, u32(0), n, mode, max_size, *o, out_ld, None,
                                        None)

    assert xchg(mode=7) == _lib.TGP_ERR_INVALID_ARG
    assert xchg(max_size=0) == _lib.TGP_ERR_INVALID_ARG
    assert xchg(max_size=2000, out_ld=2000) == _lib.TGP_ERR_INVALID_ARG   # beyond TGP_MAX_LEN
    assert xchg(max_size=16, out_ld=8) == _lib.TGP_ERR_INVALID_ARG        # row narrower than the limit
    assert xchg(max_size=4, out_ld=4) == _lib.TGP_ERR_INVALID_ARG         # narrower than old rows
    assert xchg(n=0) == _lib.TGP_OK
    assert xchg(n=-1) == _lib.TGP_ERR_INVALID_ARG
    clash = [ctypes.c_void_p(0x10040), outs[1], outs[2]]                 # inside old.type
    assert xchg(o=clash) == _lib.TGP_ERR_INVALID_ARG
    same = [outs[0], outs[0], outs[2]]
    assert xchg(o=same) == _lib.TGP_ERR_INVALID_ARG
    nulls = [None, outs[1], outs[2]]
    assert xchg(o=nulls) == _lib.TGP_ERR_INVALID_ARG
    fit = ctypes.c_void_p(0x90000)
    assert lib.tgp_tournament_select(fit, 1, 10, words, 4, 0, 1, idx, None) == _lib.TGP_ERR_INVALID_ARG
    assert lib.tgp_tournament_select(fit, 1, 0, words, 4, 3, 1, idx, None) == _lib.TGP_ERR_INVALID_ARG
    assert lib.tgp_tournament_select(fit, 0, 10, words, 4, 3, 1, idx, None) == _lib.TGP_ERR_INVALID_ARG
    assert lib.tgp_tournament_select(fit, 1, 10, words, 0, 3, 1, idx, None) == _lib.TGP_OK
    assert lib.tgp_accuracy_from_outputs(fit, 4, 0, 10, idx, idx, None, None) == _lib.TGP_ERR_INVALID_ARG
    assert lib.tgp_accuracy_from_outputs(fit, 4, 3, 0, idx, idx, None, None) == _lib.TGP_ERR_INVALID_ARG
    assert lib.tgp_accuracy_from_outputs(fit, 0, 3, 10, idx, idx, None, None) == _lib.TGP_OK
    data = _lib.tgp_data(0xA0000, 0, 2, 2)
    assert lib.tgp_accuracy_workspace_size(ctypes.byref(old), ctypes.byref(data), 3) == 0
    assert lib.tgp_fitness_accuracy(ctypes.byref(old), ctypes.byref(data), idx, 3, idx, None, None,
                                    None, 0, None) == _lib.TGP_ERR_INVALID_ARG


def test_header_compiles_as_c_and_a_c_client_runs(lib, tmp_path):
    """include/tgp.h is plain C11: a C client compiles with -Wall -Werror,
    links the library and runs its host-side checks (no GPU needed)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    exe = tmp_path / "abi_smoke"
    build_dir = os.path.dirname(_lib.LIB_PATH)
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_smoke.c"),
           "-o", str(exe), "-L", build_dir, "-ltgp", f"-Wl,-rpath,{build_dir}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "ok"


def test_autotune_cache_round_trip_through_the_c_reader(lib, tmp_path):
    """The autotuner's cache file (written in Python) is what the C planner
    reads: keys, candidates, store, lookup and the C parser agree."""
    from paper_2501_17168_gb300 import autotune
    assert autotune.lg(1) == 0 and autotune.lg(0) == 0 and autotune.lg(5000) == 12
    assert autotune.lg(100_000) == 17 and autotune.lg(255) == 8 and autotune.lg(181) == 7
    k = autotune.key("NVIDIA GB300", 5000, 100_000, 16, 1, 255)
    assert k == "NVIDIA_GB300|P12_D17_F16_O1_L8"
    # candidates: the heuristic first, both schedules (1 and up to 64 trees
    # per block), tiles that are multiples of a warp's chunk and no wider
    # than needed, one points-per-lane value for Modi populations
    c = autotune.candidates(5000, 100_000, 1)
    assert c[0] == {}
    bts = {x["trees_per_block"] for x in c[1:]}
    assert {1, 32, 64} <= bts
    for x in c[1:]:
        assert x["points_per_tile"] % (32 * x["points_per_lane"]) == 0
        assert x["points_per_tile"] <= 4096
    small = autotune.candidates(3, 100, 1)
    assert all(x["trees_per_block"] <= 3 for x in small[1:])
    assert all(x["points_per_tile"] // 2 < 100 or x["points_per_tile"] == 32 * x["points_per_lane"]
               for x in small[1:])
    assert {x["points_per_lane"] for x in autotune.candidates(100, 1000, 8)[1:]} == {4}
    assert {x.get("cta_width", 0) for x in c[1:] if x["points_per_lane"] == 8} == {0, 1}
    assert all(x.get("cta_width", 0) == 0 for x in autotune.candidates(100, 1000, 8)[1:])
    path = str(tmp_path / "tune.txt")
    autotune.store({k: ({"trees_per_block": 8, "points_per_tile": 512, "points_per_lane": 8}, 2.0)}, path)
    autotune.store({k: ({"trees_per_block": 28, "points_per_tile": 1024, "tiles_per_item": 3,
                         "points_per_lane": 8}, 1.0),
                    "other|P1_D1_F1_O1_L1": ({"trees_per_block": 1, "points_per_tile": 128,
                                               "points_per_lane": 4}, 5.0)}, path)
    db = autotune.load(path)
    assert db[k]["trees_per_block"] == 28 and db[k]["ms"] == 1.0
    cfg = _lib.tgp_config()
    assert lib.tgp_tune_cache_lookup(path.encode(), k.encode(), ctypes.byref(cfg)) == _lib.TGP_OK
    assert (cfg.trees_per_block, cfg.points_per_tile, cfg.tiles_per_item, cfg.points_per_lane) == \
        (28, 1024, 3, 8)
    assert lib.tgp_tune_cache_lookup(path.encode(), b"other|P1_D1_F1_O1_L1", ctypes.byref(cfg)) == 0
    assert cfg.points_per_lane == 4 and cfg.trees_per_block == 1
    assert lib.tgp_tune_cache_lookup(path.encode(), b"missing", ctypes.byref(cfg)) == \
        _lib.TGP_ERR_INVALID_ARG
    # a malformed value drops the entry in both readers' view of validity
    with open(path, "a") as f:
        f.write(k + " trees_per_block=-3 points_per_tile=512\n")
    assert lib.tgp_tune_cache_lookup(path.encode(), k.encode(), ctypes.byref(cfg)) == \
        _lib.TGP_ERR_INVALID_ARG
