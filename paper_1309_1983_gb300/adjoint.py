"""Checkpointed discrete adjoint behind ``torch.autograd``.

Problem: the initial state is f^0 = f^eq(1, u0) (Eq. 5), T fused steps
follow with a per-node body force F held fixed, and the loss is
L = 1/2 sum_x |u(x, T) - u_target(x)|^2. Gradients with respect to u0 and F
come from the library's adjoint kernels (lbm_adjoint_seed, lbm_adjoint_step,
lbm_adjoint_u0). The forward keeps the states f^0, f^K, f^2K, ...; the
backward recomputes each segment of K states from its checkpoint
(lbm_step_to) and then runs the reverse steps over it, so memory holds
ceil(T/K) checkpoints plus K - 1 segment states.

Every array operation runs in the library's kernels; this module only owns
the torch buffers and orders the calls.
"""

from __future__ import annotations

import ctypes

import torch

from . import capi
from .lattice import Lattice


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class AdjointProblem:
    """Geometry, tau, horizon T and checkpoint interval K of a
    velocity-mismatch problem (FP32 storage)."""

    def __init__(self, nx, ny, nz, tau, T, K=50, walls=(False, False, False), lid=None,
                 device="cuda"):
        if T < 1 or K < 1:
            raise ValueError("T and K must be >= 1")
        self.T, self.K = int(T), int(K)
        self.lat = Lattice(nx, ny, nz, tau, walls=walls, lid=lid, storage="f32", force=True,
                           device=device)
        self.shape = self.lat.shape
        self.device = self.lat.device
        lay = self.lat.layout
        self.f_bytes = lay.f_bytes
        self.lam_elems = lay.lambda_bytes // 4
        self._scratch = [self._fbuf(), self._fbuf()]
        self._segment = []
        self._ckpt_pool = []

    def _fbuf(self):
        return torch.empty(self.f_bytes, dtype=torch.uint8, device=self.device)

    @property
    def launches_forward(self):
        return 1 + self.T

    def forward(self, u0, F):
        """f^0 = f^eq(1, u0), then T steps keeping every K-th state.
        Returns (f_T, checkpoints); the buffers stay valid until the next
        call of forward()."""
        L = self.lat
        L.force.copy_(F)
        L.init_equilibrium(u=u0)
        f0, _ = L.current_buffers()  # init writes the current buffer in place
        ckpts = [f0]
        prev = f0
        for n in range(1, self.T + 1):
            if n % self.K == 0 and n < self.T:
                c = len(ckpts) - 1  # checkpoint buffers are reused across calls
                if c == len(self._ckpt_pool):
                    self._ckpt_pool.append(self._fbuf())
                dst = self._ckpt_pool[c]
                ckpts.append(dst)
            else:
                dst = self._scratch[n % 2]
            L.step_to(prev, dst)
            prev = dst
        return prev, ckpts

    def backward(self, f_T, ckpts, u0, ut):
        """Reverse sweep: (loss, grad_u0, grad_F) as device tensors."""
        L = self.lat
        h = L.handle
        lam_a = torch.empty(self.lam_elems, dtype=torch.float32, device=self.device)
        lam_b = torch.empty_like(lam_a)
        gF = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)
        loss = torch.zeros((), dtype=torch.float64, device=self.device)
        capi.call("lbm_adjoint_seed", h, _p(f_T), _p(ut), _p(lam_a), _p(gF), _p(loss))
        need = min(self.K, self.T) - 1
        while len(self._segment) < need:
            self._segment.append(self._fbuf())
        for s in range(len(ckpts) - 1, -1, -1):
            start = s * self.K
            stop = min(start + self.K, self.T)
            states = [ckpts[s]]
            for k in range(1, stop - start):
                L.step_to(states[-1], self._segment[k - 1])
                states.append(self._segment[k - 1])
            for n in range(stop - 1, start - 1, -1):
                capi.call("lbm_adjoint_step", h, _p(states[n - start]), _p(lam_a), _p(lam_b),
                          _p(gF))
                lam_a, lam_b = lam_b, lam_a
        gu0 = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)
        capi.call("lbm_adjoint_u0", h, _p(lam_a), _p(u0), _p(gu0))
        return loss, gu0, gF

    def loss_and_grad(self, u0, F, u_target):
        u0 = u0.detach().float().contiguous()
        F = F.detach().float().contiguous()
        ut = u_target.detach().float().contiguous()
        f_T, ckpts = self.forward(u0, F)
        return self.backward(f_T, ckpts, u0, ut)

    def loss(self, u0, F, u_target):
        """Forward loss only (FP64 reduction on the device)."""
        f_T, _ = self.forward(u0.detach().float().contiguous(), F.detach().float().contiguous())
        lam = torch.empty(self.lam_elems, dtype=torch.float32, device=self.device)
        out = torch.zeros((), dtype=torch.float64, device=self.device)
        capi.call("lbm_adjoint_seed", self.lat.handle, _p(f_T),
                  _p(u_target.detach().float().contiguous()), _p(lam), None, _p(out))
        return out


class VelocityMismatch(torch.autograd.Function):
    """loss = VelocityMismatch.apply(u0, F, u_target, problem): FP64 scalar
    loss; backward runs the checkpointed adjoint of ``problem``. The saved
    checkpoints live in ``problem``'s buffers, so call backward before the
    next forward on the same problem."""

    @staticmethod
    def forward(ctx, u0, F, u_target, problem: AdjointProblem):
        u0c = u0.detach().float().contiguous()
        Fc = F.detach().float().contiguous()
        utc = u_target.detach().float().contiguous()
        f_T, ckpts = problem.forward(u0c, Fc)
        lam = torch.empty(problem.lam_elems, dtype=torch.float32, device=problem.device)
        loss = torch.zeros((), dtype=torch.float64, device=problem.device)
        capi.call("lbm_adjoint_seed", problem.lat.handle, _p(f_T), _p(utc), _p(lam), None,
                  _p(loss))
        ctx.problem = problem
        ctx.state = (f_T, ckpts, u0c, utc)
        ctx.dtypes = (u0.dtype, F.dtype)
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        f_T, ckpts, u0c, utc = ctx.state
        _, gu0, gF = ctx.problem.backward(f_T, ckpts, u0c, utc)
        g = grad_out.to(torch.float32)
        return (g * gu0).to(ctx.dtypes[0]), (g * gF).to(ctx.dtypes[1]), None, None
