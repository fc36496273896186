"""Lid-driven cavity validation by self-convergence (Sec. 5).

The paper validated its solver on the cubic lid-driven cavity at
Re = 100, 400 and 1000 and observed that the centre-line velocity profiles
converge as the lattice is refined. Re = 100 is checked here (the higher
Reynolds numbers need lattices of 200+ nodes per edge and minutes of run
time to settle). The external reference data it compared
against is not available here, so this test checks the convergence itself:
cavities of N = 24, 48 and 96 nodes per edge at the same Reynolds number
(Eq. 8 with L = N: tau = 1/2 + 3 N U / Re), run to a steady state, and the
profile u_x(z)/U on the vertical centre line x = y = (N-1)/2 compared on the
coarse lattice's node positions. Halfway bounce-back makes the scheme second
order, so the difference between successive resolutions must shrink by a
factor near 4 (accepted: > 2.5).
"""

import numpy as np
import pytest

from paper_1309_1983_gb300 import perfmodel as PM

pytestmark = pytest.mark.gpu

U = 0.05


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_1983_gb300 import build as B
    B.build()


def _centre_profile(N, Re):
    from paper_1309_1983_gb300.lattice import Lattice
    tau = 0.5 + 3.0 * N * U / Re
    assert abs(PM.reynolds(U, tau, N) - Re) < 1e-9
    L = Lattice(N, N, N, tau, walls=(True, True, True), lid=(U, 0.0, 0.0))
    L.init_equilibrium()
    chunk = max(1000, int(5 * N / U))
    prev = None
    for _ in range(100):
        L.step(chunk)
        _, u = L.moments()
        # centre line: average the two (or one) central columns in x and y
        c = [N // 2 - 1, N // 2] if N % 2 == 0 else [N // 2]
        prof = u[0][:, c][:, :, c].double().mean(dim=(1, 2)).cpu().numpy() / U
        if prev is not None and np.abs(prof - prev).max() < 2e-5:
            break
        prev = prof
    else:
        pytest.fail(f"N={N} did not reach a steady state")
    z = (np.arange(N) + 0.5) / N  # node centres between the halfway walls
    return z, prof


@pytest.mark.parametrize("Re", [100])
def test_cavity_centre_line_converges_at_second_order(Re):
    profs = [_centre_profile(N, Re) for N in (24, 48, 96)]
    zc = profs[0][0]
    on_coarse = [np.interp(zc, z, p) for z, p in profs]
    d1 = np.abs(on_coarse[1] - on_coarse[0]).max()
    d2 = np.abs(on_coarse[2] - on_coarse[1]).max()
    assert np.isfinite(on_coarse).all()
    assert d1 / d2 > 2.5, (d1, d2)
    # the flow under the lid follows it and recirculates below
    assert on_coarse[2][-1] > 0.3 and on_coarse[2].min() < -0.1
