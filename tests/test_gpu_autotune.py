"""The launch-shape autotuners (lbm_autotune, lbm_batch_autotune): the
chosen shape is a legal candidate, it is applied, the cache is written and a
cache hit applies it without running a step; results do not depend on the
shape."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_1983_gb300 import build as B
    B.build()


def test_lattice_autotune_cache_and_results(tmp_path):
    from paper_1309_1983_gb300 import autotune
    from paper_1309_1983_gb300.lattice import Lattice
    cache = str(tmp_path / "tune.txt")
    L = Lattice(40, 24, 16, 0.6, walls=(True, True, True), lid=(0.05, 0.0, 0.0))
    L.init_equilibrium()
    bx, by, ms = autotune.tune_lattice(L, steps=3, cache_path=cache)
    assert bx in (32, 64) and by in (1, 2, 4, 8) and 64 <= bx * by <= 256, (bx, by)
    assert ms > 0
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and "lattice/40x24x16/" in lines[0]
    assert lines[0].split("\t")[1:3] == [str(bx), str(by)]
    # a hit runs nothing: the state is unchanged
    before = L.get_f()
    assert autotune.tune_lattice(L, steps=3, cache_path=cache)[:2] == (bx, by)
    np.testing.assert_array_equal(L.get_f(), before)
    assert len(open(cache).read().splitlines()) == 1
    # the tuned shape gives the same bits as the default one
    L.init_equilibrium()
    L.step(20)
    ref = Lattice(40, 24, 16, 0.6, walls=(True, True, True), lid=(0.05, 0.0, 0.0))
    ref.init_equilibrium()
    ref.step(20)
    np.testing.assert_array_equal(L.get_f(), ref.get_f())
    # a second problem adds its own line
    L2 = Lattice(33, 8, 8, 0.7)
    L2.init_equilibrium()
    autotune.tune_lattice(L2, steps=2, cache_path=cache)
    assert len(open(cache).read().splitlines()) == 2


def test_batch_autotune_cache(tmp_path):
    from paper_1309_1983_gb300 import autotune
    from paper_1309_1983_gb300.batch import Batch
    cache = str(tmp_path / "tune.txt")
    dims = [(17, 5, 9), (33, 16, 4), (8, 8, 8)]
    B = Batch(dims, [0.6, 0.7, 0.8], [0.02, 0.05, 0.03])
    B.init_rest()
    t, bps, ms = autotune.tune_batch(B, steps=3, cache_path=cache)
    assert t in (64, 128, 256) and bps in (0, 2, 4, 6, 8) and ms > 0
    assert B.info()["threads"] == t
    line = open(cache).read().splitlines()
    assert len(line) == 1 and line[0].split("\t")[1:3] == [str(t), str(bps)]
    B.init_rest()
    B.step(4)
    before = [B.get_f(d) for d in range(3)]
    assert autotune.tune_batch(B, steps=3, cache_path=cache)[:2] == (t, bps)
    for d in range(3):
        np.testing.assert_array_equal(B.get_f(d), before[d])
    torch.cuda.synchronize()
