"""Parity of the CUDA adjoint (through the C ABI) with the FP64 oracle's
adjoint, which is itself pinned to central finite differences.

Tolerances: single kernels are compared element by element at 2e-6 of the
largest magnitude of the compared field (FP32 arithmetic on O(1) cotangents
with O(20) dependent operations per value); whole gradients after T steps at
1e-4 relative L2 (the stated criterion), and against the oracle's finite
differences at 1e-4 relative.
"""

import ctypes

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


GEOMS = {
    "periodic": dict(walls=(0, 0, 0), lid=None),
    "cavity": dict(walls=(1, 1, 1), lid=(0.05, 0.0, 0.0)),
    "channel_y": dict(walls=(0, 1, 0), lid=None),
    "walls_xz_lid": dict(walls=(1, 0, 1), lid=(0.03, 0.01, 0.0)),
}


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _lat(shape, tau, g, force=True):
    from paper_1309_1983_gb300.lattice import Lattice
    nx, ny, nz = shape
    return Lattice(nx, ny, nz, tau, walls=tuple(bool(w) for w in g["walls"]), lid=g["lid"],
                   force=force)


def _olat(shape, tau, g):
    nx, ny, nz = shape
    lid = g["lid"]
    return O.Lattice(nx, ny, nz, tau, walls=tuple(bool(w) for w in g["walls"]),
                     lid=lid is not None, lid_u=tuple(lid) if lid else (0, 0, 0))


def _to_dev_f(L, f):
    """FP64 (19, nz, ny, nx) plain f -> a device f buffer in L's layout."""
    L.set_f(f)
    cur, _ = L.current_buffers()
    return cur.clone()


def _lam_to_dev(L, lam):
    lay = L.layout
    buf = torch.zeros(lay.lambda_bytes // 4, dtype=torch.float32, device="cuda")
    v = buf.view(19, L.nz, L.ny, lay.pitch)
    v[..., :L.nx] = torch.from_numpy(lam).float().cuda()
    return buf


def _lam_from_dev(L, buf):
    lay = L.layout
    return buf.view(19, L.nz, L.ny, lay.pitch)[..., :L.nx].double().cpu().numpy()


def _random_f(OL, seed):
    rho = 1.0 + W.noise(OL.shape, seed, 0.02)
    u = W.noise((3,) + OL.shape, seed + 1, 0.05)
    f = O.init_equilibrium(OL, rho, u)
    return f * (1.0 + W.noise(f.shape, seed + 2, 0.1))


@pytest.mark.parametrize("mode", ["auto", "branch", "select"])
@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("shape", [(37, 6, 5), (8, 8, 8), (1, 5, 7)], ids=lambda s: "x".join(map(str, s)))
def test_adjoint_step_matches_oracle(geom, shape, mode):
    """One reverse step against the oracle's dense-Jacobian adjoint, with the
    bounce-back applied by address selection, by the wall-node branch, and
    by the automatic choice."""
    from paper_1309_1983_gb300 import capi
    g = GEOMS[geom]
    tau = 0.7
    L = _lat(shape, tau, g)
    L.set_wall_mode(mode)
    OL = _olat(shape, tau, g)
    f = _random_f(OL, 40)
    F = W.noise((3,) + OL.shape, 41, 2e-3)
    lam = W.noise(f.shape, 42, 1.0)
    gF0 = W.noise((3,) + OL.shape, 43, 0.5)
    L.force.copy_(torch.from_numpy(F).float())
    fd = _to_dev_f(L, f)
    lam_in = _lam_to_dev(L, lam)
    lam_out = torch.full_like(lam_in, float("nan"))
    gF = torch.from_numpy(gF0).float().cuda()
    capi.call("lbm_adjoint_step", L.handle, _p(fd), _p(lam_in), _p(lam_out), _p(gF))
    torch.cuda.synchronize()
    gF_ref = gF0.copy()
    ref = O.adjoint_step(OL, f, lam, F, gF_ref)
    got = _lam_from_dev(L, lam_out)
    assert np.isfinite(got).all(), "some lambda^n element was not written"
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 2e-6 * scale
    gsc = np.abs(gF_ref).max()
    assert np.abs(gF.double().cpu().numpy() - gF_ref).max() <= 2e-6 * gsc


@pytest.mark.parametrize("geom", ["periodic", "cavity"])
def test_seed_and_u0_gradient_match_oracle(geom):
    from paper_1309_1983_gb300 import capi
    g = GEOMS[geom]
    shape = (21, 9, 6)
    L = _lat(shape, 0.8, g)
    OL = _olat(shape, 0.8, g)
    f = _random_f(OL, 50)
    F = W.noise((3,) + OL.shape, 51, 2e-3)
    ut = W.noise((3,) + OL.shape, 52, 0.05)
    L.force.copy_(torch.from_numpy(F).float())
    fd = _to_dev_f(L, f)
    lam = torch.empty(L.layout.lambda_bytes // 4, dtype=torch.float32, device="cuda")
    gF = torch.empty((3,) + OL.shape, dtype=torch.float32, device="cuda")
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    utd = torch.from_numpy(ut).float().cuda()
    capi.call("lbm_adjoint_seed", L.handle, _p(fd), _p(utd), _p(lam), _p(gF), _p(loss))
    lref, lam_ref, gF_ref = O.adjoint_seed(OL, f, ut.astype(np.float32).astype(np.float64), F)
    assert abs(loss.item() - lref) <= 1e-5 * lref
    np.testing.assert_allclose(_lam_from_dev(L, lam), lam_ref, rtol=0,
                               atol=2e-6 * np.abs(lam_ref).max())
    np.testing.assert_allclose(gF.double().cpu().numpy(), gF_ref, rtol=0,
                               atol=2e-6 * np.abs(gF_ref).max())
    # grad wrt u0 for f^0 = f^eq(1, u0)
    u0 = W.noise((3,) + OL.shape, 53, 0.05)
    lam0 = W.noise(f.shape, 54, 1.0)
    gu = torch.empty((3,) + OL.shape, dtype=torch.float32, device="cuda")
    # named device tensors: a temporary passed only as a raw pointer could be
    # freed (and its memory reused) before the kernel reads it
    lam0_d = _lam_to_dev(L, lam0)
    u0_d = torch.from_numpy(u0).float().cuda()
    capi.call("lbm_adjoint_u0", L.handle, _p(lam0_d), _p(u0_d), _p(gu))
    ref = O.adjoint_u0(OL, lam0, u0)
    np.testing.assert_allclose(gu.double().cpu().numpy(), ref, rtol=0,
                               atol=2e-6 * np.abs(ref).max())


@pytest.mark.parametrize("mode", ["branch", "select"])
@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("shape", [(37, 6, 5), (70, 9, 4)], ids=lambda s: "x".join(map(str, s)))
def test_moments_form_is_bit_identical(geom, shape, mode):
    """The reverse step from the forward collision's stored rho, u
    (lbm_step_to_moments + lbm_adjoint_step_moments) gives the same bits as
    the step that re-gathers f^n (lbm_adjoint_step)."""
    from paper_1309_1983_gb300 import capi
    g = GEOMS[geom]
    L = _lat(shape, 0.7, g)
    L.set_wall_mode(mode)
    OL = _olat(shape, 0.7, g)
    f = _random_f(OL, 70)
    L.force.copy_(torch.from_numpy(W.noise((3,) + OL.shape, 71, 2e-3)).float())
    fd = _to_dev_f(L, f)
    fout = torch.empty_like(fd)
    rho = torch.empty(OL.shape, device="cuda")
    u = torch.empty((3,) + OL.shape, device="cuda")
    capi.call("lbm_step_to_moments", L.handle, _p(fd), _p(fout), _p(rho), _p(u))
    lam_in = _lam_to_dev(L, W.noise(f.shape, 72, 1.0))
    outs = []
    for fn in ("state", "moments"):
        lam_out = torch.full_like(lam_in, float("nan"))
        gF = torch.from_numpy(W.noise((3,) + OL.shape, 73, 0.5)).float().cuda()
        if fn == "state":
            capi.call("lbm_adjoint_step", L.handle, _p(fd), _p(lam_in), _p(lam_out), _p(gF))
        else:
            capi.call("lbm_adjoint_step_moments", L.handle, _p(rho), _p(u), _p(lam_in),
                      _p(lam_out), _p(gF))
        torch.cuda.synchronize()
        outs.append((_lam_from_dev(L, lam_out), gF.cpu().numpy()))
    assert np.isfinite(outs[1][0]).all()
    np.testing.assert_array_equal(outs[1][0], outs[0][0])
    np.testing.assert_array_equal(outs[1][1], outs[0][1])


def test_checkpoint_forms_agree():
    """The checkpointed driver gives the same bits with segment moments
    (default) and with re-gathered segment states."""
    from paper_1309_1983_gb300.adjoint import AdjointProblem
    nx, ny, nz = 14, 9, 7
    u0 = torch.from_numpy(W.fourier_modes(nx, ny, nz, 3, 2.0, 0.02)).float().cuda()
    ut = torch.from_numpy(W.fourier_modes(nx, ny, nz, 4, 2.0, 0.02)).float().cuda()
    F = torch.from_numpy(W.noise((3, nz, ny, nx), 5, 1e-4)).float().cuda()
    res = []
    for moments in (True, False):
        P = AdjointProblem(nx, ny, nz, 0.7, T=23, K=7, walls=(True, True, True),
                           lid=(0.05, 0.0, 0.0), moments=moments)
        res.append([t.cpu().numpy() for t in P.loss_and_grad(u0, F, ut)])
    for a, b in zip(*res):
        np.testing.assert_array_equal(a, b)


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("geom,T,K", [("periodic", 20, 6), ("cavity", 24, 8),
                                      ("channel_y", 15, 15), ("walls_xz_lid", 9, 4)])
def test_checkpointed_gradients_match_oracle(geom, T, K):
    from paper_1309_1983_gb300.adjoint import AdjointProblem
    g = GEOMS[geom]
    shape = (12, 10, 8)
    nx, ny, nz = shape
    tau = 0.7
    P = AdjointProblem(nx, ny, nz, tau, T=T, K=K, walls=tuple(bool(w) for w in g["walls"]),
                       lid=g["lid"])
    OL = _olat(shape, tau, g)
    u0 = W.fourier_modes(nx, ny, nz, seed=1, kmax=2.0, amp=0.02)
    ut = W.fourier_modes(nx, ny, nz, seed=2, kmax=2.0, amp=0.02)
    F = W.noise((3,) + OL.shape, 60, 1e-4)
    u0d, utd, Fd = (torch.from_numpy(a).float().cuda() for a in (u0, ut, F))
    loss, gu0, gF = P.loss_and_grad(u0d, Fd, utd)
    # the oracle sees the same FP32-rounded inputs
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    lref, gu0_ref, gF_ref = O.loss_and_gradients(OL, r32(u0), r32(ut), T, r32(F))
    assert abs(loss.item() - lref) <= 1e-4 * lref
    assert _rel_l2(gu0.double().cpu().numpy(), gu0_ref) <= 1e-4
    assert _rel_l2(gF.double().cpu().numpy(), gF_ref) <= 1e-4


def test_gradient_matches_oracle_finite_differences():
    """Directional derivatives of the GPU gradient against central FD of the
    FP64 oracle's forward loss (h small, FP64), 1e-4 relative."""
    from paper_1309_1983_gb300.adjoint import AdjointProblem
    g = GEOMS["cavity"]
    nx, ny, nz, tau, T = 10, 8, 6, 0.65, 12
    P = AdjointProblem(nx, ny, nz, tau, T=T, K=5, walls=(True, True, True), lid=g["lid"])
    OL = _olat((nx, ny, nz), tau, g)
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    u0 = r32(W.fourier_modes(nx, ny, nz, seed=5, kmax=2.0, amp=0.02))
    ut = r32(W.fourier_modes(nx, ny, nz, seed=6, kmax=2.0, amp=0.02))
    F = r32(W.noise((3, nz, ny, nx), 7, 1e-4))
    _, gu0, gF = P.loss_and_grad(*(torch.from_numpy(a).float().cuda() for a in (u0, F, ut)))
    gu0 = gu0.double().cpu().numpy()
    gF = gF.double().cpu().numpy()
    for k in range(3):
        d = W.noise(u0.shape, 100 + k, 1.0)
        h = 1e-5
        lp = O.loss_and_gradients(OL, u0 + h * d, ut, T, F, want_grad=False)[0]
        lm = O.loss_and_gradients(OL, u0 - h * d, ut, T, F, want_grad=False)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - (gu0 * d).sum()) <= 1e-4 * abs(fd), (k, fd, (gu0 * d).sum())
        lp = O.loss_and_gradients(OL, u0, ut, T, F + h * d, want_grad=False)[0]
        lm = O.loss_and_gradients(OL, u0, ut, T, F - h * d, want_grad=False)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - (gF * d).sum()) <= 1e-4 * abs(fd), (k, fd, (gF * d).sum())


def test_autograd_function():
    from paper_1309_1983_gb300.adjoint import AdjointProblem, VelocityMismatch
    nx, ny, nz = 8, 8, 8
    P = AdjointProblem(nx, ny, nz, 0.7, T=10, K=4)
    u0 = torch.from_numpy(W.fourier_modes(nx, ny, nz, 1, 2.0, 0.02)).float().cuda()
    ut = torch.from_numpy(W.fourier_modes(nx, ny, nz, 2, 2.0, 0.02)).float().cuda()
    u0.requires_grad_(True)
    F = torch.zeros((3, nz, ny, nx), device="cuda", requires_grad=True)
    loss = VelocityMismatch.apply(u0, F, ut, P)
    (2.0 * loss).backward()
    _, gu0, gF = P.loss_and_grad(u0.detach(), F.detach(), ut)
    torch.testing.assert_close(u0.grad, 2.0 * gu0)
    torch.testing.assert_close(F.grad, 2.0 * gF)


def test_adjoint_rejects_16bit_storage():
    from paper_1309_1983_gb300 import capi
    from paper_1309_1983_gb300.lattice import Lattice
    L = Lattice(8, 8, 8, 0.7, storage="f16")
    buf = torch.zeros(L.layout.lambda_bytes // 4, device="cuda")
    cur, _ = L.current_buffers()
    rc = capi.load().lbm_adjoint_step(L.handle, _p(cur), _p(buf), _p(buf.clone()), None)
    assert rc == capi.LBM_EINVAL
