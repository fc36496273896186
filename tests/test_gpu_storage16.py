"""16-bit shifted storage (f_i - w_i as FP16 or BF16, FP32 arithmetic).

Element-wise parity for one step uses the tolerance of the storage type: the
GPU rounds each stored shifted value once (relative 2^-11 for FP16, 2^-8 for
BF16), so after one step |f_gpu - f_oracle| <= |d| * 2^-p plus the FP32
arithmetic error; the oracle starts from the same rounded state. Over long
runs the error is reported (the stated requirement), with loose sanity bounds
that a broken conversion or a wrong shift would exceed by orders of magnitude.
"""

import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1309_1983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROUND = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_1983_gb300 import build as B
    B.build()


def _lat(n, tau, storage, walls=(True, True, True), lid=(0.05, 0.0, 0.0)):
    from paper_1309_1983_gb300.lattice import Lattice
    return Lattice(n, n, n, tau, walls=walls, lid=lid, storage=storage)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("shape", [(37, 11, 9), (16, 16, 16)], ids=lambda s: "x".join(map(str, s)))
def test_one_step_within_storage_rounding(storage, shape):
    from paper_1309_1983_gb300.lattice import Lattice
    nx, ny, nz = shape
    tau = 0.6
    L = Lattice(nx, ny, nz, tau, walls=(True, True, True), lid=(0.05, 0, 0), storage=storage)
    OL = O.Lattice(nx, ny, nz, tau, walls=(True, True, True), lid=True, lid_u=(0.05, 0, 0))
    rho = 1.0 + W.noise(OL.shape, 1, 0.02)
    u = W.noise((3,) + OL.shape, 2, 0.05)
    L.set_f(O.init_equilibrium(OL, rho, u) * (1 + W.noise((19,) + OL.shape, 3, 0.1)))
    f0 = L.get_f()  # the rounded state the GPU holds
    L.step(1)
    ref = O.run(OL, f0, 1)
    w = O.weights()[:, None, None, None]
    bound = np.abs(ref - w) * ROUND[storage] + 1e-7
    assert (np.abs(L.get_f() - ref) <= bound).all()


def test_sixteen_bit_error_vs_oracle_64_after_5000_steps(tmp_path):
    """Cavity 64^3 (tau = 0.55, lid 0.05) after 5000 steps with FP32, FP16
    and BF16 storage against the FP64 oracle: the error of each is recorded
    (max and relative L2 of rho and u); FP32 must meet the stated 1e-5 of
    the velocity field maximum (measured 6.4e-7), FP16 1e-2, and BF16 must
    stay bounded (no blow-up)."""
    n, tau, steps = 64, 0.55, 5000
    OL = O.Lattice(n, n, n, tau, walls=(True, True, True), lid=True, lid_u=(0.05, 0, 0))
    rr, ur = O.moments(OL, O.run(OL, O.init_equilibrium(OL), steps))
    report = {}
    for storage in ("f32", "f16", "bf16"):
        L = _lat(n, tau, storage)
        L.init_equilibrium()
        L.step(steps)
        rho, u = L.moments()
        rho, u = rho.double().cpu().numpy(), u.double().cpu().numpy()
        report[storage] = {
            "rho_max": float(np.abs(rho - rr).max()),
            "u_max_rel": float(np.abs(u - ur).max() / np.abs(ur).max()),
            "u_l2_rel": float(np.linalg.norm(u - ur) / np.linalg.norm(ur)),
        }
    out = os.environ.get("LBM_REPORT_DIR")
    if out:
        with open(os.path.join(out, "storage16_error_64cube_5000.json"), "w") as fh:
            json.dump(report, fh, indent=1)
    print(json.dumps(report))
    assert report["f32"]["u_max_rel"] < 1e-5, report
    assert report["f16"]["u_max_rel"] < 1e-2, report
    assert report["bf16"]["u_max_rel"] < 0.5 and np.isfinite(report["bf16"]["rho_max"]), report


PAIR_SHAPES = [(37, 11, 9), (64, 5, 3), (1, 7, 6), (3, 4, 5), (33, 6, 4), (130, 3, 2), (66, 9, 3)]
PAIR_GEOMS = {
    "periodic": dict(walls=(False, False, False), lid=None),
    "cavity": dict(walls=(True, True, True), lid=(0.05, 0.0, 0.0)),
    "walls_x": dict(walls=(True, False, False), lid=None),
    "lid_yz": dict(walls=(False, True, True), lid=(0.04, -0.02, 0.0)),
}


@pytest.mark.parametrize("variant,mode", [("pair", "auto"), ("x2", "select"), ("x2", "branch")])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("geom", sorted(PAIR_GEOMS))
@pytest.mark.parametrize("shape", PAIR_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("force", [False, True])
def test_pair_kernel_is_bit_identical_to_node_kernel(storage, geom, shape, force, variant, mode):
    """The two-nodes-per-thread kernels ("pair": packed 32-bit pulls and warp
    shuffles for the x-shifted directions; "x2": packed loads for e_x = 0,
    16-bit loads otherwise, no exchange between threads, in both wall forms)
    compute the same bits as the one-node kernel, including odd and short
    rows, every wall combination, the lid, a body force and the fused moment
    output."""
    from paper_1309_1983_gb300.lattice import Lattice
    nx, ny, nz = shape
    g = PAIR_GEOMS[geom]
    OL = O.Lattice(nx, ny, nz, 0.6)
    f0 = O.init_equilibrium(OL, 1.0 + W.noise(OL.shape, 1, 0.02),
                            W.noise((3,) + OL.shape, 2, 0.05))
    f0 = f0 * (1 + W.noise(f0.shape, 3, 0.1))
    F = torch.from_numpy(W.noise((3,) + OL.shape, 4, 1e-3)).float()
    outs = []
    for kern in ("node", variant):
        L = Lattice(nx, ny, nz, 0.6, walls=g["walls"], lid=g["lid"], storage=storage,
                    force=force)
        L.set_kernel(kern)
        L.set_wall_mode(mode)
        if force:
            L.force.copy_(F)
        L.set_f(f0)
        L.step(3)
        rho, u = L.step_moments(2)
        outs.append((L.get_f(), rho.cpu(), u.cpu()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1]) and torch.equal(outs[0][2], outs[1][2])


@pytest.mark.parametrize("variant", ["pair", "x2"])
@pytest.mark.parametrize("block", [(32, 1), (32, 8), (64, 4), (128, 2), (256, 1)])
def test_pair_block_shapes_agree(block, variant):
    from paper_1309_1983_gb300.lattice import Lattice
    L = Lattice(150, 13, 5, 0.7, walls=(True, True, True), lid=(0.05, 0, 0), storage="f16")
    L.set_kernel(variant)
    L.init_equilibrium()
    L.step(4)
    ref = L.get_f()
    L.set_pair_block(*block)
    L.init_equilibrium()
    L.step(4)
    np.testing.assert_array_equal(L.get_f(), ref)
