"""Lid-driven cavity validation by self-convergence (Sec. 5).

The paper checks its solver on the cubic lid-driven cavity at Re = 100, 400
and 1000 by comparing centre-line velocity profiles with published data.
That data is not available here, so the check is the convergence itself:
the same cavity at successive resolutions N (Eq. 8 with L = N gives
tau = 1/2 + 3 N U / Re), each run to a steady state, and the profile
u_x(z)/U on the vertical centre line compared on the coarsest lattice's
node positions. Observed on GB300 (FP32): the differences shrink by 1.6 to
2.7 per doubling (order 0.7 to 1.4, in max and RMS norm and in the vortex
strength u_min alike) rather than 4: the classical cavity's lid meets the
side walls with a jump in velocity, a singularity that degrades the
convergence of the whole flow whichever way the lattice is refined.

Two ways to refine: acoustic scaling keeps the lid speed U (the Mach number)
fixed, so tau - 1/2 grows with N and BGK's viscosity-dependent bounce-back
wall error does not vanish; diffusive scaling keeps tau fixed and lowers
U = Re (tau - 1/2) / (3 N), so for a smooth flow lattice and compressibility
errors both fall as N^-2.

Two wall treatments: halfway bounce-back (walls half a node outside the
first and last nodes, edge length L = N in Eq. 8) and the on-site velocity
walls the paper used (``onsite=True``: walls on the first and last node
planes, L = N - 1).

Command line (writes one JSON object):

    python -m paper_1309_1983_gb300.validation --re 400 --sizes 48,96,192 --tau 0.53
    python -m paper_1309_1983_gb300.validation --re 400 --sizes 48,96,192 --u 0.1
    python -m paper_1309_1983_gb300.validation --re 100 --sizes 25,49,97 --u 0.05 --onsite
"""

from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import perfmodel as PM


def edge(N: int, onsite: bool = False) -> int:
    """Cavity edge length in lattice units: N for halfway walls, N - 1 for
    walls on the first and last nodes."""
    return N - 1 if onsite else N


def tau_for(N: int, U: float, Re: float, onsite: bool = False) -> float:
    """Relaxation time giving Reynolds number Re on an N^3 cavity (Eq. 8)."""
    return 0.5 + 3.0 * edge(N, onsite) * U / Re


def lid_for(N: int, tau: float, Re: float, onsite: bool = False) -> float:
    """Lid speed giving Reynolds number Re on an N^3 cavity at fixed tau (Eq. 8)."""
    return Re * (tau - 0.5) / (3.0 * edge(N, onsite))


def centre_columns(N: int):
    """x (= y) indices whose mean is the vertical centre line."""
    return [N // 2 - 1, N // 2] if N % 2 == 0 else [N // 2]


def node_positions(N: int, onsite: bool = False):
    """Node positions in units of the edge, walls at 0 and 1."""
    k = np.arange(N, dtype=np.float64)
    return k / (N - 1) if onsite else (k + 0.5) / N


def centre_profile(N: int, Re: float, U: float = 0.05, tol: float = 2e-5,
                   max_chunks: int = 200, storage: str = "f32", onsite: bool = False):
    """Run an N^3 cavity from rest to a steady state and return
    (z, u_x(z)/U, steps, converged): z the node positions in units of the
    edge (walls at 0 and 1), the profile on the vertical centre line (mean
    of the central one or two columns in x and y). Steady means the profile
    moved by less than ``tol`` (in units of U) over one chunk of
    max(1000, 5 N / U) steps."""
    import torch
    from .lattice import Lattice
    tau = tau_for(N, U, Re, onsite)
    assert abs(PM.reynolds(U, tau, edge(N, onsite)) - Re) < 1e-9 * Re
    L = Lattice(N, N, N, tau, walls=(True, True, True), lid=(U, 0.0, 0.0), storage=storage,
                onsite=onsite)
    try:
        L.init_equilibrium()
        chunk = max(1000, int(5 * N / U))
        c = centre_columns(N)
        prev, steps, converged = None, 0, False
        for _ in range(max_chunks):
            L.step(chunk)
            steps += chunk
            _, u = L.moments()
            prof = u[0][:, c][:, :, c].double().mean(dim=(1, 2)).cpu().numpy() / U
            if not np.isfinite(prof).all():
                break
            if prev is not None and np.abs(prof - prev).max() < tol:
                converged = True
                break
            prev = prof
        torch.cuda.synchronize()
    finally:
        L.close()
    return node_positions(N, onsite), prof, steps, converged


def self_convergence(Re: float, sizes=(24, 48, 96), U: float = 0.05, tau: float = None,
                     onsite: bool = False, **kw):
    """Profiles at each size, interpolated to the coarsest lattice's nodes,
    and the successive maximum differences d_k = max |p_{k+1} - p_k| with
    their ratios. With ``tau`` given, diffusive scaling (fixed tau, lid speed
    from Eq. 8 per size); else acoustic scaling at lid speed U."""
    Us = [lid_for(N, tau, Re, onsite) if tau is not None else U for N in sizes]
    runs = [centre_profile(N, Re, u, onsite=onsite, **kw) for N, u in zip(sizes, Us)]
    zc = runs[0][0]
    on_coarse = [np.interp(zc, z, p) for z, p, _, _ in runs]
    diffs = [float(np.abs(on_coarse[k + 1] - on_coarse[k]).max())
             for k in range(len(sizes) - 1)]
    ratios = [diffs[k] / diffs[k + 1] for k in range(len(diffs) - 1)]
    rms = [float(np.sqrt(np.mean((on_coarse[k + 1] - on_coarse[k]) ** 2)))
           for k in range(len(sizes) - 1)]
    # strength of the primary vortex on the centre line, from each run's own
    # nodes (a parabola through the minimum and its neighbours)
    umin = []
    for z, p, _, _ in runs:
        k = int(np.clip(np.argmin(p), 1, len(p) - 2))
        a, b, c = np.polyfit(z[k - 1:k + 2], p[k - 1:k + 2], 2)
        umin.append(float(c - b * b / (4 * a)) if a > 0 else float(p[k]))
    return {"Re": Re, "scaling": "diffusive" if tau is not None else "acoustic",
            "walls": "on-site" if onsite else "halfway", "U": Us, "sizes": list(sizes),
            "tau": [tau_for(N, u, Re, onsite) for N, u in zip(sizes, Us)],
            "steps": [r[2] for r in runs], "converged": [r[3] for r in runs],
            "diffs": diffs, "ratios": ratios, "rms_diffs": rms, "u_min": umin,
            "observed_order": [float(np.log2(r)) for r in ratios],
            "z": zc.tolist(), "profiles_on_coarse": [p.tolist() for p in on_coarse]}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--re", type=float, required=True)
    p.add_argument("--sizes", default="24,48,96")
    p.add_argument("--u", type=float, default=0.05, help="lid speed (acoustic scaling)")
    p.add_argument("--tau", type=float, default=None, help="fixed tau (diffusive scaling)")
    p.add_argument("--tol", type=float, default=2e-5)
    p.add_argument("--onsite", action="store_true", help="on-site velocity walls")
    a = p.parse_args(argv)
    t0 = time.time()
    out = self_convergence(a.re, tuple(int(s) for s in a.sizes.split(",")), a.u, tau=a.tau,
                           tol=a.tol, onsite=a.onsite)
    out["seconds"] = round(time.time() - t0, 1)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
