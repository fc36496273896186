"""The LBM_CHECK debug build (``csrc/check.cuh``), a device memory checker
built into the library.

``liblbm_check.so`` tests every global load, store and atomic of every kernel
against the buffers its launch was given (extent, read / write use, natural
alignment) and refuses, counts and records what fails instead of making the
access. ``tests/check_workloads.py`` runs every kernel family (all step
kernels and wall forms, 16-bit storage, on-site walls, graph replay,
streaming and push, moments with and without allocation, the host pipeline,
both adjoint forms, the batched persistent, per-launch and sequence kernels
and their adjoints) on small ragged lattices, once under each library in a
process of its own. The tests check that
* the checked build refuses no access in any workload;
* both builds give the same bits for every output (the checks change no
  arithmetic), so what was checked is what the normal build computes;
* at the benchmark's sizes (384^3 steps in FP32 and FP16, halfway and
  on-site walls, the 1024^3 FP32 cavity, the 64-cavity batch with its
  persistent, sequence and reverse-sequence kernels) no access is refused
  either;
* with every table range ended 64 bytes early (lbm_check_narrow) a plain
  step's accesses to those tails are refused and the first one is reported
  with its address inside one of the two f buffers' tails: refusals are
  detected, and the refused accesses are not made, so every access that is
  made stays inside its real buffer;
* the same narrowing makes the tensor-copy staged kernel skip the copies
  that read a tail, and its bounded waits end the step with LBM_ETIMEOUT
  (reported by lbm_sync) instead of hanging.
"""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = os.path.join(ROOT, "tests", "check_workloads.py")


@pytest.fixture(scope="module")
def libs():
    from paper_1309_1983_gb300 import build as B
    return B.build(), B.build(check=True)


def _run(out, lib, *extra):
    env = dict(os.environ)
    env.pop("LBM_LIBRARY", None)
    if lib:
        env["LBM_LIBRARY"] = lib
    r = subprocess.run([sys.executable, SCRIPT, str(out), *extra], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    with open(out) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def runs(libs, tmp_path_factory):
    d = tmp_path_factory.mktemp("check_build")
    return _run(d / "normal.json", None), _run(d / "checked.json", libs[1])


def _workloads(res):
    return {k: v for k, v in res.items() if isinstance(v, dict)}


def test_checked_build_refuses_no_access(runs):
    _, chk = runs
    assert chk["checked"] and chk["library"] == "liblbm_check.so"
    w = _workloads(chk)
    assert len(w) >= 60, sorted(w)
    bad = {k: v["refused"] for k, v in w.items() if v["refused"]}
    assert not bad, bad


def test_checked_build_computes_the_same_bits(runs):
    plain, chk = runs
    assert not plain["checked"]
    a, b = _workloads(plain), _workloads(chk)
    assert sorted(a) == sorted(b)
    diff = sorted(k for k in a if a[k]["digest"] != b[k]["digest"])
    assert not diff, diff


def test_narrowed_tables_are_refused_and_reported(libs, tmp_path):
    res = _run(tmp_path / "narrow.json", libs[1], "--narrow", "64")["narrow"]
    assert res["refused"] > 0, res
    assert any(lo <= res["first"] < hi for lo, hi in res["tails"]), res
    assert res["bytes"] in (4, 8) and res["kind"] in (1, 2), res


def test_refused_tensor_copy_ends_in_a_timeout_not_a_hang(libs, tmp_path):
    """A tensor copy that the check build refuses is never issued, so its
    pipeline stage never completes: the bounded mbarrier waits end the launch
    and the next lbm_sync reports LBM_ETIMEOUT."""
    from paper_1309_1983_gb300 import capi
    res = _run(tmp_path / "narrow_tma.json", libs[1], "--narrow-tma", "64")["narrow_tma"]
    assert res["refused"] > 0, res
    assert any(lo <= res["first"] < hi for lo, hi in res["tails"]), res
    assert res["bytes"] in (2, 4) and res["kind"] in (1, 2), res
    assert res["sync"] == capi.LBM_ETIMEOUT, res


def test_checked_build_refuses_no_access_at_full_size(libs, tmp_path):
    import torch
    torch.cuda.empty_cache()  # the child needs 163 GB for the 1024^3 lattice
    res = _run(tmp_path / "large.json", libs[1], "--large")["large"]
    assert set(res) == {"periodic_384_f32", "cavity_384_f16", "onsite_384_f16",
                        "cavity_1024_f32", "batch_64_cavities"}, res
    bad = {k: v["refused"] for k, v in res.items() if v["refused"]}
    assert not bad, bad
