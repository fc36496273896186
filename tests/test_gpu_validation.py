"""Lid-driven cavity validation (Sec. 5, Eq. 8).

The paper validated its solver on the cubic lid-driven cavity at Re = 100,
400 and 1000 by comparing centre-line velocity profiles with published data,
which is not available here. These tests check instead:
* the steady centre-line profile u_x(z)/U of the GPU against the FP64 oracle
  run for the same number of steps from rest (Re = 100, N = 24 halfway walls
  at U = 0.05 and N = 25 on-site walls at U = 0.1), within 1e-5 of U;
* self-convergence under refinement (``paper_1309_1983_gb300.validation``):
  cavities of N, 2N and 4N nodes per edge at fixed Re (Eq. 8), each run to a
  steady state, the profiles compared on the coarse lattice's nodes. The
  differences between successive resolutions must shrink by more than 1.5
  per doubling (about first order: the lid's velocity jump at the side walls
  is a singularity that slows the convergence of the whole flow), and the
  primary vortex strength u_min must converge monotonically.
The on-site walls are run at U = 0.1, which keeps tau >= 0.57: with BGK
their rule amplifies tangential disturbances below tau ~ 0.56 (seen in the
FP64 oracle as well: a plain channel between on-site walls started from
noise grows at tau = 0.55 and decays at 0.56), while halfway bounce-back
stays stable down to the tau = 0.536 of the N = 24, U = 0.05 case.
Re = 1000 needs lattices of 256 nodes per edge and minutes per run; it is
run with the module's command line, not here.
"""

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_1983_gb300 import build as B
    B.build()


def _oracle_profile(N, tau, U, steps, onsite, chunk):
    """The oracle's centre-line profile after `steps` steps from rest, and
    its change over the last chunk (in units of U)."""
    from paper_1309_1983_gb300.validation import centre_columns
    OL = O.Lattice(N, N, N, tau, walls=(True, True, True), lid=True, lid_u=(U, 0.0, 0.0),
                   onsite=onsite)
    c = centre_columns(N)

    def prof(f):
        _, u = O.moments(OL, f)
        return u[0][:, c][:, :, c].mean(axis=(1, 2)) / U

    f = O.run(OL, O.init_equilibrium(OL), steps - chunk)
    before = prof(f)
    after = prof(O.run(OL, f, chunk))
    return after, float(np.abs(after - before).max())


@pytest.mark.parametrize("N,onsite,U", [(24, False, 0.05), (25, True, 0.1)])
def test_cavity_steady_profile_matches_oracle(N, onsite, U):
    from paper_1309_1983_gb300.validation import centre_profile, tau_for
    Re, tol = 100.0, 2e-5
    z, prof, steps, converged = centre_profile(N, Re, U, tol=tol, onsite=onsite)
    assert converged, steps
    chunk = max(1000, int(5 * N / U))
    ref, last_change = _oracle_profile(N, tau_for(N, U, Re, onsite), U, steps, onsite, chunk)
    assert last_change < tol, last_change  # the oracle is at the steady state too
    err = float(np.abs(prof - ref).max())
    print(f"\nRe=100 N={N} {'on-site' if onsite else 'halfway'}: {steps} steps, "
          f"max |GPU - oracle| {err:.2e} U, u_min/U {ref.min():.4f}")
    assert err <= 1e-5, err
    assert ref[-1] > 0.3 and ref.min() < -0.1


def _check_refinement(r, min_ratio=1.5):
    d1, d2 = r["diffs"]
    prof = np.array(r["profiles_on_coarse"])
    assert all(r["converged"]), r["steps"]
    assert np.isfinite(prof).all()
    assert d1 / d2 > min_ratio, (d1, d2)
    m = r["u_min"]
    assert m[0] > m[1] > m[2] and (m[0] - m[1]) > (m[1] - m[2]), m
    # the flow under the lid follows it and recirculates below
    assert prof[2][-1] > 0.3 and prof[2].min() < -0.1
    return d1, d2, prof


@pytest.mark.parametrize("Re,sizes,U,onsite", [
    (100, (24, 48, 96), 0.05, False),
    (400, (48, 96, 192), 0.1, False),
    (100, (25, 49, 97), 0.1, True),
])
def test_cavity_centre_line_converges_under_refinement(Re, sizes, U, onsite):
    from paper_1309_1983_gb300.validation import self_convergence
    r = self_convergence(Re, sizes, U=U, onsite=onsite)
    d1, d2, prof = _check_refinement(r)
    print(f"\nRe={Re} {r['walls']}: max centre-line change {d1:.3e}, {d2:.3e}, "
          f"ratio {d1 / d2:.2f}, u_min/U {r['u_min']}, steps {r['steps']}")
