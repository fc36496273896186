"""The tensor-copy staged step kernel (LBM_KERNEL_TMA, 16-bit storage).

Its arithmetic is the two-node kernel's, so it must reproduce the one-node
kernel's values exactly (the one-node kernel is itself checked against the
FP64 oracle in test_gpu_forward.py and test_gpu_storage16.py); one case is
also compared with the oracle directly. The shapes cover one, several and
ragged x tiles of 64 nodes (rows of 1, 3, 37, 64, 129, 130, 200 and 384
nodes), ragged y tiles (row counts not a multiple of the tile's 2, 4 or 8
rows), one-node axes (the periodic wrap of a source onto the node itself),
every geometry (walls on each axis, the moving lid), a body force and the
fused moments, plain launches and graph replay.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1309_1983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_1983_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()


GEOMS = {
    "periodic": dict(walls=(0, 0, 0), lid=None),
    "walls_x": dict(walls=(1, 0, 0), lid=None),
    "walls_y": dict(walls=(0, 1, 0), lid=None),
    "walls_z": dict(walls=(0, 0, 1), lid=None),
    "cavity": dict(walls=(1, 1, 1), lid=(0.05, 0.0, 0.0)),
    "lid_3d": dict(walls=(0, 1, 1), lid=(0.04, -0.02, 0.0)),
}
SHAPES = [(37, 11, 9), (64, 5, 3), (130, 5, 3), (129, 3, 4), (200, 9, 5), (1, 7, 6),
          (3, 2, 4), (6, 1, 5), (384, 2, 3)]


def _lat(shape, geom, storage, force, tau=0.6):
    from paper_1309_1983_gb300.lattice import Lattice
    g = GEOMS[geom]
    nx, ny, nz = shape
    return Lattice(nx, ny, nz, tau, walls=tuple(bool(w) for w in g["walls"]), lid=g["lid"],
                   storage=storage, force=force)


def _random_f(shape, seed, amp=0.2):
    nx, ny, nz = shape
    OL = O.Lattice(nx, ny, nz, 0.6)
    rho = 1.0 + W.noise(OL.shape, seed, 0.02)
    u = W.noise((3,) + OL.shape, seed + 1, 0.05)
    f = O.init_equilibrium(OL, rho, u)
    return f * (1.0 + W.noise(f.shape, seed + 2, amp))


def _run(kernel, shape, geom, storage, force, rows=None, steps=3, graph_steps=0):
    nx, ny, nz = shape
    L = _lat(shape, geom, storage, force)
    try:
        L.set_kernel(kernel)
        if rows is not None:
            L.set_pair_block(32, rows)
        L.set_graph_steps(graph_steps)
        if force:
            L.force.copy_(torch.from_numpy(W.noise((3, nz, ny, nx), 31, 1e-3)).float())
        L.set_f(_random_f(shape, 30))
        L.step(steps)
        rho, u = L.step_moments(2)
        L.sync()
        return L.get_f(), rho.cpu(), u.cpu()
    finally:
        L.close()


def _same(a, b):
    np.testing.assert_array_equal(a[0], b[0])
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("force", [False, True])
def test_tma_kernel_equals_one_node_kernel(storage, geom, shape, force):
    _same(_run("node", shape, geom, storage, force), _run("tma", shape, geom, storage, force))


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("geom", ["periodic", "cavity", "lid_3d"])
@pytest.mark.parametrize("rows", [1, 8, 3])
@pytest.mark.parametrize("shape", [(130, 13, 5), (37, 7, 3), (64, 1, 2)],
                         ids=lambda s: "x".join(map(str, s)))
def test_tma_kernel_tile_rows(storage, geom, rows, shape):
    """Tiles of 128 x 2 (pair-block rows 1) and 64 x 8 (rows 8) nodes give
    the same values as the default 64 x 4 (any other rows, 3 here)."""
    ref = _run("node", shape, geom, storage, True)
    _same(ref, _run("tma", shape, geom, storage, True, rows=rows))


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_tma_kernel_in_graph_replay(storage):
    """Launches captured in CUDA graphs (40 steps: one 32-step graph replay
    and plain launches) give the plain launches' values."""
    shape = (200, 9, 5)
    ref = _run("node", shape, "cavity", storage, True, steps=40)
    _same(ref, _run("tma", shape, "cavity", storage, True, steps=40, graph_steps=32))


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("geom", ["periodic", "cavity"])
def test_tma_kernel_matches_oracle_one_step(storage, geom):
    """One step against the FP64 oracle from the same rounded state, with a
    body force: |f_gpu - f_oracle| <= |f_oracle - w| 2^-p + 1e-7 (one
    rounding of the stored shifted value, p = 11 for FP16, 8 for BF16)."""
    shape = (130, 9, 5)
    nx, ny, nz = shape
    g = GEOMS[geom]
    F = W.noise((3, nz, ny, nx), 41, 1e-3)
    L = _lat(shape, geom, storage, True)
    try:
        L.set_kernel("tma")
        L.force.copy_(torch.from_numpy(F).float())
        L.set_f(_random_f(shape, 40))
        f0 = L.get_f()  # the state as stored (rounded)
        L.step(1)
        L.sync()
        got = L.get_f()
    finally:
        L.close()
    OL = O.Lattice(nx, ny, nz, 0.6, walls=tuple(bool(w) for w in g["walls"]),
                   lid=g["lid"] is not None, lid_u=g["lid"] or (0, 0, 0))
    ref = O.run(OL, f0, 1, force=F)
    w = O.weights()[:, None, None, None]
    bound = np.abs(ref - w) * {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}[storage] + 1e-7
    assert (np.abs(got - ref) <= bound).all()
