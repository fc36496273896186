"""Workloads for the checked debug build (LBM_CHECK, csrc/check.cuh).

Runs every kernel family of the library once on small ragged lattices and
writes, per workload, the number of accesses the check build refused and a
SHA-256 digest of every output (so that the normal and the checked build can
be compared bit for bit). Run in a process of its own, with the library to
test named by LBM_LIBRARY:

    LBM_LIBRARY=.../liblbm_check.so python tests/check_workloads.py out.json
    python tests/check_workloads.py out.json                # the normal build
    LBM_LIBRARY=... python tests/check_workloads.py out.json --narrow 64

--narrow B ends every range of every launch table B bytes early
(lbm_check_narrow) for one plain step of a periodic FP32 lattice, and
records the first refused access and the tails of the buffers it could lie
in; --narrow-tma B does the same for one step of the tensor-copy staged
kernel (FP16) and records the error code of the lbm_sync after it. --large runs the benchmark's sizes instead (one step of 384^3 periodic
FP32, 384^3 cavity FP16 with halfway and with on-site walls, the 1024^3
FP32 cavity (163 GB of f), and the 64-cavity batch: persistent steps, a
step sequence with moments and a reverse sequence) and records only the
refusals. Inputs are seeded; nothing here is compared with the oracle (the parity
tests do that for the normal build).
"""

from __future__ import annotations

import hashlib
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1309_1983_gb300 import capi  # noqa: E402
from paper_1309_1983_gb300.adjoint import AdjointProblem, BatchAdjointProblem  # noqa: E402
from paper_1309_1983_gb300.batch import Batch  # noqa: E402
from paper_1309_1983_gb300.lattice import Lattice  # noqa: E402

SHAPE = (37, 23, 19)  # odd rows: padding nodes, ragged tiles and pair ends
CHECKED = os.path.basename(capi.LIB_PATH) == "liblbm_check.so"


def digest(ts):
    h = hashlib.sha256()
    for t in ts:
        if isinstance(t, torch.Tensor):
            h.update(t.detach().contiguous().cpu().numpy().tobytes())
        else:
            h.update(np.ascontiguousarray(t).tobytes())
    return h.hexdigest()


def refused():
    """Refused accesses since the last reset (0 in the normal build), then reset."""
    torch.cuda.synchronize()
    if not CHECKED:
        return 0
    n = capi.check_status()[0]
    capi.call("lbm_check_reset")
    return n


def rand_field(shape, seed, scale):
    g = torch.Generator().manual_seed(seed)
    return (scale * (2 * torch.rand(shape, generator=g) - 1)).float().cuda()


def lattice(geom, storage, force=False, onsite=False):
    nx, ny, nz = SHAPE
    walls = {"periodic": (False,) * 3, "cavity": (True,) * 3, "channel": (False, True, True)}[geom]
    lid = (0.05, 0.01, 0.0) if geom == "cavity" else None
    L = Lattice(nx, ny, nz, 0.62, walls=walls, lid=lid, storage=storage, force=force,
                onsite=onsite)
    L.set_graph_steps(0)
    if force:
        L.force.copy_(rand_field((3, nz, ny, nx), 7, 1e-5))
    return L


def forward(geom, storage, kernel, force=False, onsite=False, wall_mode=None, graph=0):
    L = lattice(geom, storage, force, onsite)
    try:
        L.set_kernel(kernel)
        if wall_mode:
            L.set_wall_mode(wall_mode)
        nx, ny, nz = SHAPE
        L.init_equilibrium(u=rand_field((3, nz, ny, nx), 3, 0.02))
        if graph:
            L.set_graph_steps(graph)
            L.step(2 * graph)
        else:
            L.step(3)
        rho1, u1 = L.step_moments(1)
        rho, u, m = L.moments(mass=True)
        cur, _ = L.current_buffers()
        return [cur, rho1, u1, rho, u, np.float64(m)]
    finally:
        L.close()


def streams_and_push(storage):
    L = lattice("cavity", storage)
    try:
        nx, ny, nz = SHAPE
        L.init_equilibrium(u=rand_field((3, nz, ny, nx), 5, 0.02))
        a, b = L.current_buffers()
        out = []
        for form in ("pull", "push", "copy", "pull_l2"):
            L.streaming(a, b, form)
            out.append(b.clone())
        L.step_push(a, b)
        out.append(b.clone())
        L.step_to(a, b)
        out.append(b.clone())
        rho = torch.empty((nz, ny, nx), device="cuda")
        u = torch.empty((3, nz, ny, nx), device="cuda")
        L.step_to_moments(a, b, rho, u)
        out += [b.clone(), rho, u]
        return out
    finally:
        L.close()


def noalloc(storage):
    L = lattice("periodic", storage, force=True)
    try:
        nx, ny, nz = SHAPE
        L.init_equilibrium(u=rand_field((3, nz, ny, nx), 9, 0.02))
        L.step(2)
        cur, _ = L.current_buffers()
        rho = torch.empty((nz, ny, nx), device="cuda")
        u = torch.empty((3, nz, ny, nx), device="cuda")
        mass = torch.zeros((), dtype=torch.float64, device="cuda")
        flags = L.flags & ~(capi.LBM_WALL_X | capi.LBM_WALL_Y | capi.LBM_WALL_Z | capi.LBM_LID)
        capi.call("lbm_moments_noalloc", capi._vp(cur.data_ptr()), nx, ny, nz, flags,
                  capi._vp(L.force.data_ptr()), capi._vp(rho.data_ptr()),
                  capi._vp(u.data_ptr()), capi._vp(mass.data_ptr()),
                  capi._vp(torch.cuda.current_stream().cuda_stream))
        return [rho, u, mass]
    finally:
        L.close()


def run_host():
    L = lattice("cavity", "f32")
    try:
        nx, ny, nz = SHAPE
        u0 = rand_field((3, nz, ny, nx), 11, 0.02).cpu().pin_memory()
        rho = torch.empty((nz, ny, nx)).pin_memory()
        u = torch.empty((3, nz, ny, nx)).pin_memory()
        L.run_host(u0, 3, rho, u)
        return [rho, u]
    finally:
        L.close()


def adjoint(geom, moments, wall_mode=None):
    nx, ny, nz = SHAPE
    walls = (True,) * 3 if geom == "cavity" else (False,) * 3
    P = AdjointProblem(nx, ny, nz, 0.7, T=7, K=3, walls=walls,
                       lid=(0.03, 0.0, 0.0) if geom == "cavity" else None, moments=moments)
    try:
        if wall_mode:
            P.lat.set_wall_mode(wall_mode)
        u0 = rand_field((3, nz, ny, nx), 13, 0.02)
        F = rand_field((3, nz, ny, nx), 17, 1e-5)
        ut = rand_field((3, nz, ny, nx), 19, 0.02)
        return list(P.loss_and_grad(u0, F, ut))
    finally:
        P.lat.close()


def batch_dims():
    return np.array([[9, 7, 5], [16, 11, 13], [21, 6, 10], [5, 5, 5]], dtype=np.int32)


def batch_forward():
    dims = batch_dims()
    B = Batch(dims, np.array([0.6, 0.7, 0.55, 0.9], dtype=np.float32),
              lid_ux=np.array([0.05, 0.02, 0.04, 0.0], dtype=np.float32))
    try:
        g = torch.Generator().manual_seed(23)
        u0 = (0.02 * (2 * torch.rand(3 * B.cells, generator=g) - 1)).float().cuda()
        B.init_equilibrium(u0)
        B.step(4)                 # persistent launch with grid barriers
        B.step_launches(3)        # one launch per step
        rho, u = B.moments()
        cur, other = B.current_buffers()
        out = [cur, rho, u]
        # the step sequence of lbm_batch_run with moments
        fins, fouts = [cur, other, cur], [other, cur, other]
        rs = [torch.empty(B.cells, device="cuda") for _ in range(3)]
        us = [torch.empty(3 * B.cells, device="cuda") for _ in range(3)]
        ptrs = BatchAdjointProblem._ptrs
        capi.call("lbm_batch_run", B.handle, 3, ptrs(fins), ptrs(fouts), ptrs(rs), ptrs(us))
        B.init_rest()
        return out + [other] + rs + us
    finally:
        B.close()


def batch_adjoint(moments):
    dims = batch_dims()
    B = Batch(dims, np.array([0.6, 0.7, 0.55, 0.9], dtype=np.float32),
              lid_ux=np.array([0.05, 0.02, 0.04, 0.0], dtype=np.float32))
    try:
        P = BatchAdjointProblem(B, T=7, K=3, moments=moments)
        g = torch.Generator().manual_seed(29)
        u0 = (0.02 * (2 * torch.rand(3 * B.cells, generator=g) - 1)).float().cuda()
        ut = (0.02 * (2 * torch.rand(3 * B.cells, generator=g) - 1)).float().cuda()
        F = torch.zeros(3 * B.cells, device="cuda")
        return list(P.loss_and_grad(u0, F, ut))
    finally:
        B.close()


def workloads():
    w = {}
    for storage in ("f32", "f16", "bf16"):
        for geom in ("periodic", "cavity", "channel"):
            kernels = ["x2", "node", "bulk", "bulk1"] + (["x4", "pair", "tma"] if storage != "f32"
                                                         else [])
            for k in kernels:
                w[f"fwd_{geom}_{storage}_{k}"] = (forward, (geom, storage, k))
        w[f"fwd_cavity_{storage}_x2_force"] = (forward, ("cavity", storage, "x2", True))
        w[f"fwd_cavity_{storage}_node_branch"] = (forward, ("cavity", storage, "node", True, False,
                                                            "branch"))
        w[f"fwd_cavity_{storage}_x2_select"] = (forward, ("cavity", storage, "x2", False, False,
                                                          "select"))
        w[f"onsite_{storage}_x2"] = (forward, ("cavity", storage, "x2", True, True))
        w[f"onsite_{storage}_node"] = (forward, ("cavity", storage, "node", True, True))
        w[f"graph_cavity_{storage}"] = (forward, ("cavity", storage, "x2", False, False, None, 2))
        if storage != "f32":
            w[f"graph_cavity_{storage}_tma"] = (forward, ("cavity", storage, "tma", True, False,
                                                          None, 2))
        w[f"streams_push_{storage}"] = (streams_and_push, (storage,))
        w[f"noalloc_{storage}"] = (noalloc, (storage,))
    w["run_host"] = (run_host, ())
    for geom in ("periodic", "cavity"):
        w[f"adjoint_{geom}_regather"] = (adjoint, (geom, False))
        w[f"adjoint_{geom}_moments"] = (adjoint, (geom, True))
    w["adjoint_cavity_branch"] = (adjoint, ("cavity", True, "branch"))
    w["batch_forward"] = (batch_forward, ())
    w["batch_adjoint_regather"] = (batch_adjoint, (False,))
    w["batch_adjoint_moments"] = (batch_adjoint, (True,))
    return w


def narrow(nbytes):
    """One plain x2 step of a periodic FP32 lattice with every table range
    ended nbytes early: the refusals and the buffer tails they may lie in."""
    L = lattice("periodic", "f32")
    try:
        nx, ny, nz = SHAPE
        L.init_equilibrium(u=rand_field((3, nz, ny, nx), 31, 0.02))
        refused()
        capi.call("lbm_check_narrow", nbytes)
        try:
            L.step(1)
            torch.cuda.synchronize()
            n, addr, size, kind = capi.check_status()
        finally:
            capi.call("lbm_check_narrow", 0)
        capi.call("lbm_check_reset")
        fb = L.layout.f_bytes
        tails = [[t.data_ptr() + fb - nbytes, t.data_ptr() + fb] for t in (L.f_a, L.f_b)]
        return {"refused": n, "first": addr, "bytes": size, "kind": kind, "tails": tails}
    finally:
        L.close()


def narrow_tma(nbytes):
    """One step of the tensor-copy staged kernel (periodic FP16) with every
    table range ended nbytes early: the copies reading a tail are not issued,
    so their stages never complete and the bounded waits end the launch with
    a timeout instead of a hang. Returns the refusals, the buffer tails and
    the error code of the following lbm_sync."""
    L = lattice("periodic", "f16")
    try:
        nx, ny, nz = SHAPE
        L.set_kernel("tma")
        L.init_equilibrium(u=rand_field((3, nz, ny, nx), 33, 0.02))
        refused()
        capi.call("lbm_check_narrow", nbytes)
        try:
            L.step(1)
            torch.cuda.synchronize()
            n, addr, size, kind = capi.check_status()
        finally:
            capi.call("lbm_check_narrow", 0)
        code = 0
        try:
            L.sync()
        except capi.LBMError as e:
            code = e.code
        capi.call("lbm_check_reset")
        fb = L.layout.f_bytes
        tails = [[t.data_ptr() + fb - nbytes, t.data_ptr() + fb] for t in (L.f_a, L.f_b)]
        return {"refused": n, "first": addr, "bytes": size, "kind": kind, "tails": tails,
                "sync": code}
    finally:
        L.close()


def large():
    from paper_1309_1983_gb300 import workloads as W
    res = {}

    def one(name, n, geom, storage, onsite=False):
        walls = (geom == "cavity",) * 3
        L = Lattice(n, n, n, 0.6, walls=walls, lid=(0.05, 0.0, 0.0) if walls[0] else None,
                    storage=storage, onsite=onsite)
        try:
            L.set_graph_steps(0)
            L.init_equilibrium()
            L.step(1)
            m = L.mass()
            res[name] = {"refused": refused(), "mass": m}
        finally:
            L.close()
            torch.cuda.empty_cache()

    one("periodic_384_f32", 384, "periodic", "f32")
    one("cavity_384_f16", 384, "cavity", "f16")
    one("onsite_384_f16", 384, "cavity", "f16", onsite=True)
    one("cavity_1024_f32", 1024, "cavity", "f32")
    G = W.batch_geometry(64, seed=3)
    B = Batch(G.dims, G.tau, G.lid_u)
    try:
        B.init_rest()
        B.step(4)
        f0, f1 = B.current_buffers()
        k = 8
        rho = [torch.empty(B.cells, device="cuda") for _ in range(k)]
        u = [torch.empty(3 * B.cells, device="cuda") for _ in range(k)]
        ptrs = BatchAdjointProblem._ptrs
        fins = [f0 if j % 2 == 0 else f1 for j in range(k)]
        fouts = [f1 if j % 2 == 0 else f0 for j in range(k)]
        capi.call("lbm_batch_run", B.handle, k, ptrs(fins), ptrs(fouts), ptrs(rho), ptrs(u))
        lam = [torch.full((B.f_bytes // 4,), 1e-3, device="cuda") for _ in range(2)]
        gF = torch.zeros(3 * B.cells, device="cuda")
        capi.call("lbm_batch_adjoint_run", B.handle, k, ptrs(rho[::-1]), ptrs(u[::-1]),
                  capi._vp(lam[0].data_ptr()), capi._vp(lam[1].data_ptr()),
                  capi._vp(gF.data_ptr()))
        res["batch_64_cavities"] = {"refused": refused(), "cells": int(B.cells)}
    finally:
        B.close()
    return res


def main(argv):
    out_path = argv[0]
    res = {"library": os.path.basename(capi.LIB_PATH), "checked": CHECKED}
    if "--narrow" in argv:
        res["narrow"] = narrow(int(argv[argv.index("--narrow") + 1]))
    elif "--narrow-tma" in argv:
        res["narrow_tma"] = narrow_tma(int(argv[argv.index("--narrow-tma") + 1]))
    elif "--large" in argv:
        if CHECKED:
            refused()
        res["large"] = large()
    else:
        capi.load()
        if CHECKED:
            refused()
        for name, (fn, args) in workloads().items():
            outs = fn(*args)
            res[name] = {"refused": refused(), "digest": digest(outs)}
    with open(out_path, "w") as fh:
        json.dump(res, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
