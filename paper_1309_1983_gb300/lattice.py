"""Python handle over one lattice of liblbm (thin binding).

PyTorch provides the device memory (the two f buffers, the force field and
the moment outputs) and the stream; every operation on the data runs in the
library's CUDA kernels through :mod:`paper_1309_1983_gb300.capi`.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi

_STORAGE = {"f32": capi.LBM_STORE_F32, "f16": capi.LBM_STORE_F16, "bf16": capi.LBM_STORE_BF16}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Lattice:
    """A D3Q19 lattice of ``nx * ny * nz`` nodes bound to two device f
    buffers.

    ``walls``: (x, y, z) booleans for halfway bounce-back walls (else
    periodic). ``lid``: lid velocity (ux, uy, uz) of the moving plane
    z = nz (needs a z wall), or None. ``storage``: "f32", "f16" or "bf16".
    ``force``: True to allocate a per-cell body force field
    (:attr:`force`, shape (3, nz, ny, nx), zero-initialised).
    ``onsite``: True for on-site velocity walls (LBM_WALLS_ONSITE) instead
    of halfway bounce-back.
    """

    def __init__(self, nx, ny, nz, tau, walls=(False, False, False), lid=None,
                 storage="f32", force=False, device="cuda", stream=None, onsite=False):
        flags = 0
        if walls[0]:
            flags |= capi.LBM_WALL_X
        if walls[1]:
            flags |= capi.LBM_WALL_Y
        if walls[2]:
            flags |= capi.LBM_WALL_Z
        if lid is not None:
            flags |= capi.LBM_LID
        flags |= _STORAGE[storage]
        if force:
            flags |= capi.LBM_FORCE
        if onsite:
            flags |= capi.LBM_WALLS_ONSITE
        self.nx, self.ny, self.nz = nx, ny, nz
        self.tau = float(tau)
        self.storage = storage
        self.flags = flags
        self.device = torch.device(device)
        self._h = capi.create(nx, ny, nz, tau, flags)
        try:
            self.layout = capi.layout(self._h)
            nb = self.layout.f_bytes
            self.f_a = torch.empty(nb, dtype=torch.uint8, device=self.device)
            self.f_b = torch.empty(nb, dtype=torch.uint8, device=self.device)
            self.force = (torch.zeros((3, nz, ny, nx), dtype=torch.float32, device=self.device)
                          if force else None)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._bind()
            if lid is not None:
                capi.call("lbm_set_lid", self._h, *[float(v) for v in lid])
        except Exception:
            capi.load().lbm_destroy(self._h)
            self._h = None
            raise

    # -- handle plumbing ------------------------------------------------------
    def _bind(self):
        capi.call("lbm_bind", self._h, _ptr(self.f_a), _ptr(self.f_b), _ptr(self.force),
                  ctypes.c_void_p(self.stream.cuda_stream))

    def close(self):
        if getattr(self, "_h", None):
            capi.load().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    def current_buffers(self):
        """(current, other) as the torch byte tensors bound to the handle."""
        cur, _ = capi.current(self._h)
        if cur == self.f_a.data_ptr():
            return self.f_a, self.f_b
        return self.f_b, self.f_a

    def set_lid(self, ux, uy=0.0, uz=0.0):
        capi.call("lbm_set_lid", self._h, float(ux), float(uy), float(uz))

    def set_tau(self, tau):
        capi.call("lbm_set_tau", self._h, float(tau))
        self.tau = float(tau)

    def set_block(self, bx, by):
        capi.call("lbm_set_block", self._h, int(bx), int(by))

    def set_kernel(self, variant):
        """"node" (one node per thread), "x2" (two nodes per thread, the
        default), "x4" (four nodes per thread), "pair" (16-bit storage
        only, two nodes per thread with warp shuffles), or "bulk" / "bulk1"
        (rows staged in shared memory by bulk copies)."""
        v = {"node": capi.LBM_KERNEL_NODE, "pair": capi.LBM_KERNEL_PAIR,
             "bulk": capi.LBM_KERNEL_BULK, "bulk1": capi.LBM_KERNEL_BULK1,
             "x2": capi.LBM_KERNEL_X2, "x4": capi.LBM_KERNEL_X4,
             "tma": capi.LBM_KERNEL_TMA}[variant]
        capi.call("lbm_set_kernel", self._h, v)

    def set_graph_steps(self, steps):
        """Steps per replayed CUDA graph in multi-step calls (0 = plain
        launches; see lbm_set_graph_steps)."""
        capi.call("lbm_set_graph_steps", self._h, int(steps))

    def set_wall_mode(self, mode):
        """"auto", "branch" or "select" (see lbm_set_wall_mode)."""
        v = {"auto": capi.LBM_WALLS_AUTO, "branch": capi.LBM_WALLS_BRANCH,
             "select": capi.LBM_WALLS_SELECT}[mode]
        capi.call("lbm_set_wall_mode", self._h, v)

    def set_pair_block(self, bxp, by):
        capi.call("lbm_set_pair_block", self._h, int(bxp), int(by))

    # -- operations -------------------------------------------------------------
    def _field(self, a, comps):
        if a is None:
            return None
        t = torch.as_tensor(a, dtype=torch.float32, device=self.device).contiguous()
        exp = (comps,) + self.shape if comps > 1 else self.shape
        if tuple(t.shape) != exp:
            raise ValueError(f"field shape {tuple(t.shape)} != {exp}")
        return t

    def init_equilibrium(self, rho=None, u=None):
        r = self._field(rho, 1)
        v = self._field(u, 3)
        capi.call("lbm_init_equilibrium", self._h, _ptr(r), _ptr(v))
        self._keep = (r, v)  # alive until the kernel has read them

    def step(self, n=1):
        capi.call("lbm_step", self._h, int(n))

    def step_moments(self, n=1):
        rho = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        u = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)
        capi.call("lbm_step_moments", self._h, int(n), _ptr(rho), _ptr(u))
        return rho, u

    def step_to(self, f_in, f_out):
        capi.call("lbm_step_to", self._h, _ptr(f_in), _ptr(f_out))

    def step_to_moments(self, f_in, f_out, rho, u):
        """One step f_in -> f_out also writing the rho, u its collision used
        (the inputs of the adjoint's stored-moments reverse step)."""
        capi.call("lbm_step_to_moments", self._h, _ptr(f_in), _ptr(f_out), _ptr(rho), _ptr(u))

    def buffer_bytes(self, which):
        """Bytes of one caller-owned buffer: "f", "force", "rho", "u",
        "lambda" or "gradf" (lbm_buffer_bytes)."""
        k = {"f": capi.LBM_BUF_F, "force": capi.LBM_BUF_FORCE, "rho": capi.LBM_BUF_RHO,
             "u": capi.LBM_BUF_U, "lambda": capi.LBM_BUF_LAMBDA,
             "gradf": capi.LBM_BUF_GRADF}[which]
        b = ctypes.c_size_t()
        capi.call("lbm_buffer_bytes", self._h, k, ctypes.byref(b))
        return b.value

    def step_push(self, g_in, g_out):
        """One push step (Alg. 2) on post-streaming states."""
        capi.call("lbm_step_push", self._h, _ptr(g_in), _ptr(g_out))

    def streaming(self, f_in, f_out, form="pull"):
        """f_out = P f_in; form "pull", "push", "pull_l2" (the gather through
        L2 only) or "copy" (unshifted)."""
        v = {"pull": capi.LBM_STREAM_PULL, "push": capi.LBM_STREAM_PUSH,
             "copy": capi.LBM_STREAM_COPY, "pull_l2": capi.LBM_STREAM_PULL_L2}[form]
        capi.call("lbm_stream", self._h, _ptr(f_in), _ptr(f_out), v)

    def buffer_to_numpy(self, buf):
        """Any device f buffer of this lattice as FP64 (19, nz, ny, nx) plain
        values (as get_f for the current state)."""
        out = np.empty((19,) + self.shape, dtype=np.float64)
        capi.call("lbm_get_buffer", self._h, _ptr(buf), out.ctypes.data_as(ctypes.c_void_p))
        return out

    def moments(self, mass=False):
        """(rho, u) of the current state as device tensors; with mass=True
        also the FP64 total mass (synchronises)."""
        rho = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        u = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)
        m = capi.moments(self._h, _ptr(rho), _ptr(u), mass)
        return (rho, u, m) if mass else (rho, u)

    def mass(self):
        return capi.moments(self._h, None, None, True)

    def sync(self):
        capi.call("lbm_sync", self._h)

    def get_f(self) -> np.ndarray:
        """Current state as FP64 (19, nz, ny, nx), plain f_i (w_i added)."""
        out = np.empty((19,) + self.shape, dtype=np.float64)
        capi.call("lbm_get_f", self._h, out.ctypes.data_as(ctypes.c_void_p))
        return out

    def set_f(self, f) -> None:
        a = np.ascontiguousarray(f, dtype=np.float64)
        if a.shape != (19,) + self.shape:
            raise ValueError(f"f shape {a.shape} != {(19,) + self.shape}")
        capi.call("lbm_set_f", self._h, a.ctypes.data_as(ctypes.c_void_p))

    def run_host(self, u0_host, n, rho_host, u_host):
        """End-to-end call on host tensors (pinned recommended)."""
        for t in (u0_host, rho_host, u_host):
            if t is not None and (t.device.type != "cpu" or not t.is_contiguous()
                                  or t.dtype != torch.float32):
                raise ValueError("host buffers must be contiguous float32 CPU tensors")
        capi.call("lbm_run_host", self._h, _ptr(u0_host), int(n), _ptr(rho_host), _ptr(u_host))
