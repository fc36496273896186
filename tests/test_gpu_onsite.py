"""On-site velocity walls (LBM_WALLS_ONSITE, Hecht & Harting's conditions of
the paper's cavity, Sec. 5) on the GPU against the FP64 oracle.

Tolerances as for the halfway walls (test_gpu_forward.py): element-wise f
within 1e-6 after 1 and 10 steps (FP32 storage); rho and u within 1e-5 of
the field maximum after 1000 steps of the 32^3 cavity; 16-bit storage within
one storage rounding of a step from the rounded state.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1309_1983_gb300 import capi
from paper_1309_1983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ATOL_F = 1e-6
ROUND = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_1983_gb300 import build as B
    B.build()


def _lat(shape, tau, walls, lid=None, storage="f32", force=False):
    from paper_1309_1983_gb300.lattice import Lattice
    nx, ny, nz = shape
    return Lattice(nx, ny, nz, tau, walls=walls, lid=lid, storage=storage, force=force,
                   onsite=True)


def _olat(shape, tau, walls, lid=None):
    nx, ny, nz = shape
    return O.Lattice(nx, ny, nz, tau, walls=walls, lid=lid is not None,
                     lid_u=tuple(lid) if lid is not None else (0, 0, 0), onsite=True)


def _random_state(OL, seed, amp=0.2):
    rho = 1.0 + W.noise(OL.shape, seed, 0.02)
    u = W.noise((3,) + OL.shape, seed + 1, 0.05)
    f = O.init_equilibrium(OL, rho, u)
    return f * (1.0 + W.noise(f.shape, seed + 2, amp))


GEOMS = {
    "cavity": ((True, True, True), (0.05, 0.0, 0.0)),
    "closed_box": ((True, True, True), None),
    "couette_z": ((False, False, True), (0.04, -0.02, 0.0)),
    "walls_y": ((False, True, False), None),
    "edges_y": ((True, False, True), (0.03, 0.0, 0.01)),
    "edges_z": ((True, True, False), None),
}
SHAPES = [(37, 11, 9), (64, 5, 3), (3, 7, 6), (33, 4, 5)]


@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("kernel", ["x2", "node"])
def test_onsite_steps_match_oracle_elementwise(geom, shape, force, kernel):
    walls, lid = GEOMS[geom]
    tau = 0.66
    L = _lat(shape, tau, walls, lid, force=force)
    L.set_kernel(kernel)
    OL = _olat(shape, tau, walls, lid)
    f0 = _random_state(OL, 20 + shape[0])
    F = W.noise((3,) + OL.shape, 98, 2e-3) if force else None
    if force:
        L.force.copy_(torch.from_numpy(F).float())
    L.set_f(f0)
    ref = f0
    for nsteps in (1, 9):
        L.step(nsteps)
        ref = O.run(OL, ref, nsteps, F)
        err = np.abs(L.get_f() - ref).max()
        assert err <= ATOL_F, (geom, shape, nsteps, err)


def test_onsite_cavity_32_1000_steps():
    """Lid-driven cavity 32^3 with on-site walls (tau 0.6, lid 0.05) from
    rest: rho and u within 1e-5 of the oracle after 1000 steps."""
    n, tau, lid = 32, 0.6, (0.05, 0.0, 0.0)
    walls = (True, True, True)
    L = _lat((n, n, n), tau, walls, lid)
    L.init_equilibrium()
    L.step(1000)
    rho, u = L.moments()
    OL = _olat((n, n, n), tau, walls, lid)
    rr, ur = O.moments(OL, O.run(OL, O.init_equilibrium(OL), 1000))
    rho, u = rho.double().cpu().numpy(), u.double().cpu().numpy()
    er = np.abs(rho - rr).max() / np.abs(rr).max()
    eu = np.abs(u - ur).max() / np.abs(ur).max()
    assert er <= 1e-5 and eu <= 1e-5, (er, eu)
    # the lid's interior nodes move with the lid, the other walls rest
    assert np.abs(u[0, -1, 1:-1, 1:-1] - 0.05).max() < 1e-6
    assert np.abs(u[:, 0]).max() < 1e-6


def test_onsite_poiseuille_matches_closed_form():
    """Force-driven channel between on-site walls (z = 0 and z = H): the
    GPU's steady profile is the exact parabola F/(2 nu) z (H - z) up to FP32
    rounding."""
    nz, tau, Fx = 17, 0.9, 1e-5
    L = _lat((8, 4, nz), tau, (False, False, True), force=True)
    L.force[0].fill_(Fx)
    L.init_equilibrium()
    nu = (tau - 0.5) / 3.0
    L.step(int(30 * nz * nz / nu))
    _, u = L.moments()
    z = np.arange(nz)
    exact = Fx / (2.0 * nu) * z * (nz - 1 - z)
    got = u[0].double().mean(dim=(1, 2)).cpu().numpy()
    assert np.abs(got - exact).max() / exact.max() < 1e-4


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_onsite_sixteen_bit_one_step_within_storage_rounding(storage):
    shape, tau = (37, 11, 9), 0.6
    walls, lid = GEOMS["cavity"]
    L = _lat(shape, tau, walls, lid, storage=storage)
    OL = _olat(shape, tau, walls, lid)
    L.set_f(_random_state(OL, 5, 0.1))
    f0 = L.get_f()
    L.step(1)
    ref = O.run(OL, f0, 1)
    w = O.weights()[:, None, None, None]
    bound = np.abs(ref - w) * ROUND[storage] + 1e-7
    assert (np.abs(L.get_f() - ref) <= bound).all()


def test_onsite_kernels_and_host_path_agree():
    """Two-node and one-node kernels, graph replay and the end-to-end host
    call give the same bits."""
    shape = (29, 10, 7)
    walls, lid = GEOMS["cavity"]
    nx, ny, nz = shape
    u0 = torch.from_numpy(W.fourier_modes(nx, ny, nz, seed=4, kmax=2.0, amp=0.02)).float()
    outs = []
    for kernel, graph in (("x2", 0), ("node", 0), ("x2", 4)):
        L = _lat(shape, 0.7, walls, lid)
        L.set_kernel(kernel)
        L.set_graph_steps(graph)
        L.init_equilibrium(u=u0.cuda())
        L.step(12)
        outs.append(L.get_f())
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    L = _lat(shape, 0.7, walls, lid)
    rho_h = torch.empty((nz, ny, nx)).pin_memory()
    u_h = torch.empty((3, nz, ny, nx)).pin_memory()
    L.run_host(u0.pin_memory(), 12, rho_h, u_h)
    np.testing.assert_array_equal(L.get_f(), outs[0])


def test_onsite_rejects_unsupported_paths():
    L = _lat((8, 8, 8), 0.7, (True, True, True))
    for k in ("bulk", "bulk1"):
        with pytest.raises(RuntimeError):
            L.set_kernel(k)
    cur, other = L.current_buffers()
    with pytest.raises(RuntimeError):
        L.streaming(cur, other, "pull")
    with pytest.raises(RuntimeError):
        L.step_push(cur, other)
    lam = torch.zeros(L.layout.lambda_bytes, dtype=torch.uint8, device="cuda")
    lam2 = torch.zeros_like(lam)
    with pytest.raises(RuntimeError):
        capi.call("lbm_adjoint_step", L.handle, capi.ctypes.c_void_p(cur.data_ptr()),
                  capi.ctypes.c_void_p(lam.data_ptr()), capi.ctypes.c_void_p(lam2.data_ptr()),
                  None)
