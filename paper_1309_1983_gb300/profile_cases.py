"""Small, self-contained runs of one kernel each, for profiler captures.

Each case builds its own state on the GPU, launches the kernel of interest a
few times (so a capture can skip the warm-up launches) and exits; sizes stay
at a few GB of device memory so that a full ``ncu`` capture, which saves and
restores device memory around its passes, ends in about a minute.

    python -m paper_1309_1983_gb300.profile_cases step --geometry cavity --storage f16 --n 256
        init + 4 plain step launches (k_step_x2 by default; --kernel x4 / node;
        --onsite: on-site velocity walls instead of halfway bounce-back)
    python -m paper_1309_1983_gb300.profile_cases batch-adjoint --steps 4
        the 64-cavity batch: one forward sequence with moments, then two
        reverse-sequence launches (k_batch_adj_seq) of `steps` steps each
"""

from __future__ import annotations

import argparse
import ctypes
import sys


def step(geometry: str = "cavity", storage: str = "f16", n: int = 256, launches: int = 4,
         tau: float = 0.55, kernel: str = "x2", onsite: bool = False, rows: int = 0) -> None:
    import torch
    from .lattice import Lattice
    walls = (geometry == "cavity",) * 3
    L = Lattice(n, n, n, tau, walls=walls, lid=(0.05, 0.0, 0.0) if geometry == "cavity" else None,
                storage=storage, onsite=onsite)
    L.set_graph_steps(0)
    L.set_kernel(kernel)
    if rows:
        L.set_pair_block(32, rows)
    L.init_equilibrium()
    for _ in range(launches):
        L.step(1)
    torch.cuda.synchronize()
    L.close()


def batch_adjoint(steps: int = 4, launches: int = 2) -> None:
    import torch
    from . import capi, workloads as W
    from .batch import Batch
    G = W.batch_geometry(64, seed=3)
    B = Batch(G.dims, G.tau, G.lid_u)
    B.init_rest()
    B.step(10)
    cells = B.cells

    def ptrs(ts):
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    f0, f1 = B.current_buffers()
    rho = [torch.empty(cells, device=B.device) for _ in range(steps)]
    u = [torch.empty(3 * cells, device=B.device) for _ in range(steps)]
    fins = [f0 if k % 2 == 0 else f1 for k in range(steps)]
    fouts = [f1 if k % 2 == 0 else f0 for k in range(steps)]
    capi.call("lbm_batch_run", B.handle, steps, ptrs(fins), ptrs(fouts), ptrs(rho), ptrs(u))
    lam = [torch.full((B.f_bytes // 4,), 1e-3, device=B.device) for _ in range(2)]
    gF = torch.zeros(3 * cells, device=B.device)
    for _ in range(launches):
        capi.call("lbm_batch_adjoint_run", B.handle, steps, ptrs(rho[::-1]), ptrs(u[::-1]),
                  ctypes.c_void_p(lam[0].data_ptr()), ctypes.c_void_p(lam[1].data_ptr()),
                  ctypes.c_void_p(gF.data_ptr()))
    torch.cuda.synchronize()
    B.close()


def main(argv=None) -> int:
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = p.add_subparsers(dest="case", required=True)
    s = sub.add_parser("step")
    s.add_argument("--geometry", default="cavity", choices=["cavity", "periodic"])
    s.add_argument("--storage", default="f16", choices=["f32", "f16", "bf16"])
    s.add_argument("--n", type=int, default=256)
    s.add_argument("--launches", type=int, default=4)
    s.add_argument("--kernel", default="x2", choices=["x2", "x4", "node", "tma"])
    s.add_argument("--rows", type=int, default=0,
                   help="tile rows of the tma kernel (pair-block rows; 0: the default)")
    s.add_argument("--onsite", action="store_true")
    s.add_argument("--tau", type=float, default=0.55)
    b = sub.add_parser("batch-adjoint")
    b.add_argument("--steps", type=int, default=4)
    b.add_argument("--launches", type=int, default=2)
    a = p.parse_args(argv)
    if a.case == "step":
        step(a.geometry, a.storage, a.n, a.launches, tau=a.tau, kernel=a.kernel, onsite=a.onsite,
             rows=a.rows)
    else:
        batch_adjoint(a.steps, a.launches)
    print("ok")
    return 0


if __name__ == "__main__":
    sys.exit(main())
