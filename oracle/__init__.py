"""FP64 CPU oracle for the D3Q19 BGK lattice Boltzmann hot path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product path (``paper_1309_1983_gb300``) never imports it and shares no code
with it.

Every function follows the plain definition of the method (Sec. 3, Eqs. 3-7,
pull order of Alg. 3) and is pinned by the ``-m "not gpu"`` tests against
facts fixed independently of it: the velocity table printed as Eq. 4, the
lattice isotropy identities, mass and momentum conservation, the equilibrium
fixed point, the closed-form shear-wave decay, the force-driven Poiseuille
parabola between halfway walls, and central finite differences of its own
forward map for the adjoint.
"""

from .oracle import (  # noqa: F401
    Lattice,
    build,
    library,
    velocity_set,
    weights,
    opposites,
    init_equilibrium,
    stream,
    collide,
    run,
    run_aos,
    to_aos,
    moments,
    adjoint_seed,
    adjoint_step,
    adjoint_u0,
    loss_and_gradients,
    max_threads,
    set_threads,
)
