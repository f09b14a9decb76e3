"""Host-side checks of the C ABI library (no GPU needed).

* the library builds for sm_103a and loads;
* it exports every function include/knnjoin.h declares;
* the ctypes struct layouts of the binding equal the header's;
* the exact-arithmetic header reproduces IEEE-754 double arithmetic bit for
  bit (canonical squared distance and square root) against the host CPU;
* calls without a GPU fail with a status, not a crash.
"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1810_04758_b300 as kj
from paper_1810_04758_b300 import build as kbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "knnjoin.h")


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return kj.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(knnjoin_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    assert set(names) == set(kj.EXPORTS), names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", kj.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (knnjoin_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_struct_layouts_match_header(tmp_path):
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-O0", "-o", str(exe), os.path.join(ROOT, "tests/native/layout_probe.c")],
                   check=True)
    lines = dict((l.split()[0], list(map(int, l.split()[1:])))
                 for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                         check=True).stdout.splitlines())
    assert lines["config"] == [ctypes.sizeof(kj.KnnjoinConfig), kj.KnnjoinConfig.width_mult.offset,
                               kj.KnnjoinConfig.hbm_budget_bytes.offset, kj.KnnjoinConfig.workers.offset,
                               kj.KnnjoinConfig.large_first.offset]
    assert lines["job"] == [ctypes.sizeof(kj.KnnjoinJob), kj.KnnjoinJob.out_dist.offset]
    assert lines["stats"] == [ctypes.sizeof(kj.KnnjoinStats), kj.KnnjoinStats.candidates.offset,
                              kj.KnnjoinStats.ms_index.offset, kj.KnnjoinStats.ms_wall.offset,
                              kj.KnnjoinStats.ms_pass.offset, kj.KnnjoinStats.pass_candidates.offset,
                              kj.KnnjoinStats.width_mult.offset, kj.KnnjoinStats.chunks.offset,
                              kj.KnnjoinStats.buffer_entries.offset]


def test_exact_arithmetic_matches_ieee_double_on_host(tmp_path):
    exe = tmp_path / "test_exact_host"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe),
                    os.path.join(ROOT, "tests/native/test_exact_host.cpp")], check=True)
    r = subprocess.run([str(exe), "400000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad=0" in r.stdout


def test_version_string(lib):
    assert kj.knnjoin_version().startswith("knnjoin-b300")


def test_create_without_gpu_returns_status(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = kj.KnnjoinConfig()
    out = ctypes.c_void_p()
    st = lib.knnjoin_create(ctypes.byref(cfg), ctypes.byref(out))
    assert st in (kj.KNN_ERR_CUDA, kj.KNN_ERR_INVALID)
    assert not out.value


def test_null_context_is_rejected(lib):
    assert lib.knnjoin_self_join(None, None, 10, 2, 3, None, None) == kj.KNN_ERR_INVALID
    assert lib.knnjoin_poll(None, 1) == kj.KNN_ERR_INVALID
    lib.knnjoin_destroy(None)


def test_null_handles_of_the_newer_entry_points(lib):
    # no context / no index: rejected without touching a GPU
    out = (ctypes.c_int64 * 3)()
    rows = (ctypes.c_int64 * 1)(0)
    assert lib.knnjoin_fp32_mismatch(None, None, 10, 2, 3, None, rows, 1, out) == kj.KNN_ERR_INVALID
    assert lib.knnjoin_self_join_rows(None, None, 10, 2, 3, 0, 5, None, None) == kj.KNN_ERR_INVALID
    ix = ctypes.c_void_p()
    assert lib.knnjoin_index_create(None, None, 10, 2, 3, ctypes.byref(ix)) == kj.KNN_ERR_INVALID
    assert lib.knnjoin_index_query(None, None, 1, 3, None, None) == kj.KNN_ERR_INVALID
    assert lib.knnjoin_index_stats(None, None) == kj.KNN_ERR_INVALID
    lib.knnjoin_index_destroy(None)


@pytest.mark.parametrize("n,world,rank", [(5, 0, 0), (5, 2, 2), (5, 2, -1), (3, 4, 0)])
def test_shard_rows_rejects_bad_arguments(n, world, rank):
    with pytest.raises(ValueError):
        kj.shard_rows(n, world, rank)


@pytest.mark.parametrize("workload", ["batched", "served", "join", "index"])
def test_reference_arm_reports_unavailable_workloads(workload):
    # the CPU oracle is timed on the unif/expo workloads only; the others
    # print one JSON line saying so and exit 0 (no GPU needed)
    import json
    import subprocess
    import sys
    root = os.path.dirname(HEADER).rsplit(os.sep, 1)[0]
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--workload", workload], capture_output=True, text=True, timeout=120, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference" and "unavailable" in line
