"""Lid-driven cavity validation by self-convergence (Sec. 5).

The paper validated its solver on the cubic lid-driven cavity at
Re = 100, 400 and 1000 and observed that the centre-line velocity profiles
converge as the lattice is refined. The external reference data it compared
against is not available here, so this test checks the convergence itself
(``paper_1309_1983_gb300.validation``): cavities of N = 24, 48 and 96 nodes
per edge at Re = 100 (Eq. 8 with L = N: tau = 1/2 + 3 N U / Re), run to a
steady state, and the profile u_x(z)/U on the vertical centre line compared
on the coarse lattice's node positions. The differences between successive
resolutions must shrink (by more than 1.5 per doubling here: the lid's
velocity jump at the side walls makes the classical cavity converge at
about first order, measured 2.7 for this case and 1.6-1.9 at Re = 400 and
1000), and the primary vortex strength u_min must converge monotonically
(successive changes of one sign, shrinking).
Re = 400 and 1000 need lattices of 100-250 nodes per edge and a minute or
more each; they are run with the module's command line, not here.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_1983_gb300 import build as B
    B.build()


@pytest.mark.parametrize("Re", [100])
def test_cavity_centre_line_converges_at_second_order(Re):
    from paper_1309_1983_gb300.validation import self_convergence
    r = self_convergence(Re, (24, 48, 96), U=0.05)
    d1, d2 = r["diffs"]
    prof = np.array(r["profiles_on_coarse"])
    print(f"\nRe={Re}: max centre-line change 24->48 {d1:.3e}, 48->96 {d2:.3e}, "
          f"ratio {d1 / d2:.2f}, u_x/U min {prof[2].min():.4f}, steps {r['steps']}")
    assert all(r["converged"]), r["steps"]
    assert np.isfinite(prof).all()
    assert d1 / d2 > 1.5, (d1, d2)
    m = r["u_min"]
    assert m[0] > m[1] > m[2] and (m[0] - m[1]) > (m[1] - m[2]), m
    # the flow under the lid follows it and recirculates below
    assert prof[2][-1] > 0.3 and prof[2].min() < -0.1
