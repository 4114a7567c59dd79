"""The C-ABI library builds, loads and exports every entry point that
include/bf.h declares; argument checks that return before any CUDA call
work without a GPU (CPU only)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bf.h")


@pytest.fixture(scope="module")
def bf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1412_4907_gb300 as m
    return m


def declared():
    hdr = open(HEADER).read()
    return set(re.findall(r"^(?:bf_status|const char \*|double)\s*(bf_\w+)\(", hdr, re.M))


def test_every_declared_symbol_is_exported(bf):
    names = declared()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", bf.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (bf_\w+)$", out, re.M))
    assert names <= exported, names - exported
    assert names == set(bf.SIGNATURES), names ^ set(bf.SIGNATURES)
    lib = ctypes.CDLL(bf.LIB_PATH)
    for n in names:
        assert getattr(lib, n) is not None


def test_library_targets_sm103a(bf):
    import __graft_entry__
    assert "arch=compute_103a,code=sm_103a" in __graft_entry__._build_module().ARCH


def _create(bf, **kw):
    args = dict(pos=np.zeros((4, 3)), freqs=np.array([4e8]), dirs=np.array([[0.0, 0.0, 1.0]]),
                dtype=bf.BF_C16F, t_int=64, layout=bf.BF_LAYOUT_CTN)
    args.update(kw)
    return bf.bf_plan_create(args["pos"], args["freqs"], args["dirs"], args["dtype"], args["t_int"],
                             args["layout"])


@pytest.mark.parametrize("kw,status", [
    (dict(pos=np.zeros((0, 3))), 1),
    (dict(dirs=np.array([[0.0, 0.5, 0.5]])), 1),
    (dict(dirs=np.array([[np.nan, 0.0, 1.0]])), 1),
    (dict(freqs=np.array([-1.0])), 1),
    (dict(freqs=np.array([np.inf])), 1),
    (dict(pos=np.array([[np.nan, 0, 0]] * 4)), 1),
    (dict(dtype=17), 1),
    (dict(layout=5), 1),
    (dict(t_int=0), 1),
    (dict(pos=np.zeros((5, 3))), 5),                         # 16-bit rows of 20 bytes: no TMA
    (dict(pos=np.zeros((4, 3)), dtype=3), 5),                 # FP8 with N % 8 != 0
    (dict(t_int=100), 5),                                     # lcm(16, 100) > 256 on tensor cores
])
def test_plan_create_rejects_before_touching_the_device(bf, kw, status):
    with pytest.raises(bf.BFError) as ei:
        _create(bf, **kw)
    assert ei.value.status == status
    assert bf.bf_last_error()


def test_null_and_bad_handles(bf):
    lib = bf._lib
    assert lib.bf_destroy(None) == bf.BF_OK
    assert lib.bf_sync(None) == bf.BF_ERR_ARG
    assert lib.bf_execute(None, None, 0, None, None) == bf.BF_ERR_ARG
    assert lib.bf_weights(None, None) == bf.BF_ERR_ARG
    assert lib.bf_plan_query(None, None, None, None, None) == bf.BF_ERR_ARG
    b = ctypes.c_void_p()
    assert lib.bf_batch_create(ctypes.byref(b), None, 0, 0) == bf.BF_ERR_ARG
    assert lib.bf_batch_create(None, None, 1, 0) == bf.BF_ERR_ARG
    assert lib.bf_batch_set(None, 0, None, 0, None) == bf.BF_ERR_ARG
    assert lib.bf_batch_execute(None, None) == bf.BF_ERR_ARG
    assert lib.bf_batch_replay(None, None) == bf.BF_ERR_ARG
    assert lib.bf_batch_sync(None) == bf.BF_ERR_ARG
    assert lib.bf_batch_query(None, None, None, None) == bf.BF_ERR_ARG
    assert lib.bf_batch_destroy(None) == bf.BF_OK
    assert lib.bf_plan_set_weight_buffers(None, 2) == bf.BF_ERR_ARG
    assert lib.bf_server_create(ctypes.byref(b), None, 1, 1 << 20, 2, 0) == bf.BF_ERR_ARG
    assert lib.bf_server_create(ctypes.byref(b), None, 1, 1 << 20, 0, 0) == bf.BF_ERR_ARG
    assert lib.bf_server_submit(None, 0, None, 1, None, None) == bf.BF_ERR_ARG
    n = ctypes.c_int()
    assert lib.bf_server_poll(None, None, 0, ctypes.byref(n), 0) == bf.BF_ERR_ARG
    assert lib.bf_server_drain(None, 0) == bf.BF_ERR_ARG
    assert lib.bf_server_pause(None, 1) == bf.BF_ERR_ARG
    assert lib.bf_server_stats(None, None) == bf.BF_ERR_ARG
    assert lib.bf_server_destroy(None) == bf.BF_OK
    assert lib.bf_server_now() > 0.0
    assert lib.bf_selftest_timeout(0.0, None) == bf.BF_ERR_ARG
    assert lib.bf_selftest_timeout(1e9, None) == bf.BF_ERR_ARG
    out = ctypes.c_void_p(123)
    assert lib.bf_plan_create(ctypes.byref(out), 0, None, None, 0, None, 0, None, 0, 0, 0, None) == bf.BF_ERR_ARG
    assert out.value is None
    assert lib.bf_plan_create(None, 4, None, None, 1, None, 1, None, 0, 1, 0, None) == bf.BF_ERR_ARG


def test_corner_turn_argument_checks(bf):
    with pytest.raises(bf.BFError) as ei:
        bf.bf_corner_turn(0, bf.BF_C16F, 0, bf.BF_C16F, 4, 1, 8)
    assert ei.value.status == bf.BF_ERR_ARG
    with pytest.raises(bf.BFError) as ei:
        bf.bf_corner_turn(16, bf.BF_C16F, 32, bf.BF_C16F, 4, 1, 8, perm=[0, 1, 1, 2])
    assert ei.value.status == bf.BF_ERR_ARG
    with pytest.raises(bf.BFError) as ei:
        bf.bf_corner_turn(16, bf.BF_C16F, 32, bf.BF_CI8, 4, 1, 8)
    assert ei.value.status == bf.BF_ERR_UNSUPPORTED


def test_binding_fails_loudly_without_the_library(tmp_path):
    """The product path has no fallback: with libbf.so absent the import raises."""
    code = ("import sys, os; sys.path.insert(0, %r);"
            "import paper_1412_4907_gb300 as m" % str(tmp_path))
    pkg = tmp_path / "paper_1412_4907_gb300"
    pkg.mkdir()
    src = open(os.path.join(ROOT, "paper_1412_4907_gb300", "__init__.py")).read()
    (pkg / "__init__.py").write_text(src)
    r = subprocess.run(["python", "-c", code], capture_output=True, text=True)
    assert r.returncode != 0 and "not built" in r.stderr


def test_planner_layouts_fit_shared_memory(bf):
    """Every tiling the planner picks keeps the kernel's shared-memory layout
    inside the allocation (checked on the host before any CUDA call)."""
    import itertools
    for n_ant, n_beam, dtype, t_int in itertools.product(
            (4, 8, 16, 32, 40, 64, 96, 128, 192, 256, 384, 512), (1, 65, 1024, 4096),
            (bf.BF_C16F, bf.BF_C16BF, bf.BF_C8E4M3, bf.BF_CI8, bf.BF_CI4), (1, 10, 16, 48, 64, 128, 256)):
        if dtype == bf.BF_C8E4M3 and n_ant % 8:
            continue
        pos = np.zeros((n_ant, 3))
        dirs = np.tile([0.0, 0.0, 1.0], (n_beam, 1))
        try:
            h = bf.bf_plan_create(pos, np.array([4e8]), dirs, dtype, t_int)
            bf.bf_destroy(h)          # a GPU is present: the plan was built
        except bf.BFError as e:
            assert "inconsistency" not in str(e), (n_ant, n_beam, dtype, t_int, str(e))
            assert e.status in (bf.BF_ERR_CUDA, bf.BF_ERR_UNSUPPORTED, bf.BF_ERR_NOMEM), str(e)
