"""Python handle over a batch of independent lattices (thin binding of the
lbm_batch_* entry points): uneven cavities, each with its own tau and lid
speed, advanced in one persistent, graph-captured cooperative launch."""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Batch:
    def __init__(self, dims, tau, lid_ux=None, walls=(True, True, True), lid=True,
                 device="cuda", stream=None):
        dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
        tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float32).reshape(-1))
        self.ndom = dims.shape[0]
        if tau.shape[0] != self.ndom:
            raise ValueError("one tau per domain")
        lid_arr = None
        if lid_ux is not None:
            lid_arr = np.ascontiguousarray(np.asarray(lid_ux, dtype=np.float32).reshape(-1))
        flags = 0
        if walls[0]:
            flags |= capi.LBM_WALL_X
        if walls[1]:
            flags |= capi.LBM_WALL_Y
        if walls[2]:
            flags |= capi.LBM_WALL_Z
        if lid:
            flags |= capi.LBM_LID
        self.dims = dims
        self.tau = tau
        self.lid_ux = lid_arr
        self.device = torch.device(device)
        h = ctypes.c_void_p()
        capi.call("lbm_batch_create", self.ndom, dims.ctypes.data_as(ctypes.c_void_p),
                  tau.ctypes.data_as(ctypes.c_void_p),
                  None if lid_arr is None else lid_arr.ctypes.data_as(ctypes.c_void_p),
                  flags, ctypes.byref(h))
        self._h = h.value
        try:
            fb, cells = ctypes.c_size_t(), ctypes.c_size_t()
            self.f_offsets = np.zeros(self.ndom, dtype=np.uint64)
            self.cell_offsets = np.zeros(self.ndom, dtype=np.uint64)
            capi.call("lbm_batch_layout", self._h, ctypes.byref(fb), ctypes.byref(cells),
                      self.f_offsets.ctypes.data_as(ctypes.c_void_p),
                      self.cell_offsets.ctypes.data_as(ctypes.c_void_p))
            self.f_bytes, self.cells = fb.value, cells.value
            self.f_a = torch.empty(self.f_bytes, dtype=torch.uint8, device=self.device)
            self.f_b = torch.empty(self.f_bytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            capi.call("lbm_batch_bind", self._h, _p(self.f_a), _p(self.f_b),
                      ctypes.c_void_p(self.stream.cuda_stream))
        except Exception:
            capi.load().lbm_batch_destroy(self._h)
            self._h = None
            raise

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            capi.load().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tiling(self, threads, blocks_per_sm=0):
        capi.call("lbm_batch_set_tiling", self._h, int(threads), int(blocks_per_sm))

    def set_timeout(self, seconds):
        capi.call("lbm_batch_set_timeout", self._h, float(seconds))

    def inject_barrier_fault(self, extra):
        capi.call("lbm_batch_inject_barrier_fault", self._h, int(extra))

    def use_graph(self, on):
        capi.call("lbm_batch_use_graph", self._h, int(bool(on)))

    def info(self):
        g, t, n, gr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        capi.call("lbm_batch_info", self._h, ctypes.byref(g), ctypes.byref(t), ctypes.byref(n),
                  ctypes.byref(gr))
        return {"grid": g.value, "threads": t.value, "tiles": n.value, "graph": bool(gr.value)}

    def init_rest(self):
        capi.call("lbm_batch_init_rest", self._h)

    def init_equilibrium(self, u0=None):
        """f = f^eq(1, u0) in every domain; u0 in the packed field layout."""
        capi.call("lbm_batch_init_equilibrium", self._h, _p(u0))
        self._keep = u0

    def current_buffers(self):
        cur, other = ctypes.c_void_p(), ctypes.c_void_p()
        capi.call("lbm_batch_current", self._h, ctypes.byref(cur), ctypes.byref(other))
        if cur.value == self.f_a.data_ptr():
            return self.f_a, self.f_b
        return self.f_b, self.f_a

    def pack_vectors(self, fields):
        """Per-domain (3, nz, ny, nx) arrays -> one device tensor in the
        packed layout u[3 * cell_offset[d] + comp * cells_d + node]."""
        out = torch.empty(3 * self.cells, dtype=torch.float32, device=self.device)
        for d, a in enumerate(fields):
            c0 = int(self.cell_offsets[d])
            t = torch.as_tensor(a, dtype=torch.float32).reshape(-1)
            out[3 * c0:3 * c0 + t.numel()] = t.to(self.device)
        return out

    def unpack_vectors(self, t):
        """Inverse of pack_vectors: list of (3, nz, ny, nx) host arrays."""
        host = t.detach().double().cpu().numpy()
        res = []
        for d in range(self.ndom):
            nx, ny, nz = (int(v) for v in self.dims[d])
            c0 = int(self.cell_offsets[d])
            res.append(host[3 * c0:3 * c0 + 3 * nx * ny * nz].reshape(3, nz, ny, nx))
        return res

    def step(self, n):
        """n steps in one persistent launch (synchronises)."""
        capi.call("lbm_batch_step", self._h, int(n))

    def step_launches(self, n):
        capi.call("lbm_batch_step_launches", self._h, int(n))

    def moments(self):
        rho = torch.empty(self.cells, dtype=torch.float32, device=self.device)
        u = torch.empty(3 * self.cells, dtype=torch.float32, device=self.device)
        capi.call("lbm_batch_moments", self._h, _p(rho), _p(u))
        return rho, u

    def domain_fields(self, rho, u, d):
        """Views of domain d in the dense field outputs: (nz, ny, nx) and
        (3, nz, ny, nx)."""
        nx, ny, nz = (int(v) for v in self.dims[d])
        c0 = int(self.cell_offsets[d])
        cells = nx * ny * nz
        return (rho[c0:c0 + cells].view(nz, ny, nx),
                u[3 * c0:3 * c0 + 3 * cells].view(3, nz, ny, nx))

    def get_f(self, d):
        nx, ny, nz = (int(v) for v in self.dims[d])
        out = np.empty((19, nz, ny, nx), dtype=np.float64)
        capi.call("lbm_batch_get_f", self._h, int(d), out.ctypes.data_as(ctypes.c_void_p))
        return out

    def set_f(self, d, f):
        nx, ny, nz = (int(v) for v in self.dims[d])
        a = np.ascontiguousarray(f, dtype=np.float64)
        if a.shape != (19, nz, ny, nx):
            raise ValueError("bad shape")
        capi.call("lbm_batch_set_f", self._h, int(d), a.ctypes.data_as(ctypes.c_void_p))
