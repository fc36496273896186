"""Pins of the oracle's discrete adjoint against central finite differences
of the oracle's own forward map (FP64), and the transpose (dot-product) test
of single steps."""

import numpy as np
import pytest

import oracle as O
from paper_1309_1983_gb300 import workloads as W

CASES = {
    "periodic": dict(L=O.Lattice(4, 5, 3, 0.7), T=5, force=False),
    "cavity_force": dict(L=O.Lattice(4, 3, 5, 0.62, walls=(True, True, True), lid=True,
                                     lid_u=(0.05, 0.0, 0.0)), T=6, force=True),
    "channel_force": dict(L=O.Lattice(3, 4, 4, 0.9, walls=(False, True, False)), T=4, force=True),
}


def _setup(case):
    L = CASES[case]["L"]
    u0 = W.fourier_modes(L.nx, L.ny, L.nz, seed=1, kmax=2.0, amp=0.03)
    ut = W.fourier_modes(L.nx, L.ny, L.nz, seed=2, kmax=2.0, amp=0.03)
    F = W.noise((3,) + L.shape, 77, 1e-3) if CASES[case]["force"] else None
    return L, u0, ut, F


@pytest.mark.parametrize("case", sorted(CASES))
def test_adjoint_matches_central_differences(case):
    L, u0, ut, F = _setup(case)
    T = CASES[case]["T"]
    loss, gu0, gF = O.loss_and_gradients(L, u0, ut, T, F)
    Fz = F if F is not None else np.zeros((3,) + L.shape)
    for k in range(4):
        d = W.noise(u0.shape, 500 + k, 1.0)
        h = 1e-4 * np.abs(u0).max()
        lp = O.loss_and_gradients(L, u0 + h * d, ut, T, F, want_grad=False)[0]
        lm = O.loss_and_gradients(L, u0 - h * d, ut, T, F, want_grad=False)[0]
        fd = (lp - lm) / (2 * h)
        an = float((gu0 * d).sum())
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-14, (k, fd, an)
        dF = W.noise(u0.shape, 600 + k, 1.0)
        hF = 1e-6
        lp = O.loss_and_gradients(L, u0, ut, T, Fz + hF * dF, want_grad=False)[0]
        lm = O.loss_and_gradients(L, u0, ut, T, Fz - hF * dF, want_grad=False)[0]
        fd = (lp - lm) / (2 * hF)
        an = float((gF * dF).sum())
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-14, (k, fd, an)


@pytest.mark.parametrize("case", sorted(CASES))
def test_adjoint_step_is_transpose_of_linearised_step(case):
    """<J v, w> = <v, J^T w> for one step, J v by central differences of the
    forward step."""
    L, u0, _, F = _setup(case)
    f = O.run(L, O.init_equilibrium(L, None, u0), 2, F)
    for k in range(3):
        v = W.noise(f.shape, 700 + k, 1e-2)
        w = W.noise(f.shape, 800 + k, 1.0)
        h = 1e-4
        Jv = (O.run(L, f + h * v, 1, F) - O.run(L, f - h * v, 1, F)) / (2 * h)
        JTw = O.adjoint_step(L, f, w, F)
        a, b = float((Jv * w).sum()), float((v * JTw).sum())
        assert abs(a - b) <= 1e-9 * max(abs(a), abs(b)), (a, b)


def test_seed_is_gradient_of_loss():
    L, u0, ut, F = _setup("cavity_force")
    f = O.run(L, O.init_equilibrium(L, None, u0), 3, F)
    loss, lam, gF = O.adjoint_seed(L, f, ut, F)
    _, u = O.moments(L, f, F)
    assert abs(loss - 0.5 * ((u - ut) ** 2).sum()) < 1e-15
    d = W.noise(f.shape, 901, 1.0)
    h = 1e-7  # the loss is strongly curved along d; truncation error ~ h^2
    fd = (O.adjoint_seed(L, f + h * d, ut, F)[0] - O.adjoint_seed(L, f - h * d, ut, F)[0]) / (2 * h)
    assert abs(fd - float((lam * d).sum())) < 1e-6 * abs(fd)
