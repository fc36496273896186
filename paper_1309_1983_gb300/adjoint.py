"""Checkpointed discrete adjoint behind ``torch.autograd``.

Problem: the initial state is f^0 = f^eq(1, u0) (Eq. 5), T fused steps
follow with a per-node body force F held fixed, and the loss is
L = 1/2 sum_x |u(x, T) - u_target(x)|^2. Gradients with respect to u0 and F
come from the library's adjoint kernels (lbm_adjoint_seed, lbm_adjoint_step,
lbm_adjoint_u0, or their lbm_batch_* counterparts for a batch of lattices).
The forward keeps the states f^0, f^K, f^2K, ...; the backward recomputes
each segment from its checkpoint and then runs the reverse steps over it.
By default (``moments=True``) the recompute stores, per step, only the
density and velocity its collision used (lbm_step_to_moments, 16 bytes per
node): the collision Jacobian depends on the pulled state only through
them, so the reverse step (lbm_adjoint_step_moments) reads those instead of
re-gathering f^n, and a segment needs 16 instead of 76 bytes per node and
step. ``moments=False`` keeps the K - 1 segment states and re-gathers them
(lbm_adjoint_step); both give the same bits.

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


class _Checkpointed:
    """Checkpoint / recompute driver; subclasses supply the kernels."""

    def __init__(self, T, K, moments=True):
        if T < 1 or K < 1:
            raise ValueError("T and K must be >= 1")
        self.T, self.K = int(T), int(K)
        self.moments = bool(moments)
        self._scratch = None
        self._segment = []
        self._mom_seg = []
        self._ckpt_pool = []
        self._tail_moments = False  # the last segment's moments are in _mom_seg

    # -- supplied by subclasses ------------------------------------------------
    def _fbuf(self):
        raise NotImplementedError

    def _init(self, u0, F):  # returns the buffer holding f^0
        raise NotImplementedError

    def _step_to(self, fin, fout):
        raise NotImplementedError

    def _seed(self, fT, ut, lam, gF, loss):
        raise NotImplementedError

    def _adj_step(self, fn, lam_in, lam_out, gF):
        raise NotImplementedError

    def _step_mom(self, fin, fout, rho, u):
        raise NotImplementedError

    def _adj_step_mom(self, rho, u, lam_in, lam_out, gF):
        raise NotImplementedError

    def _mom(self):  # (rho, u) buffers for one step
        raise NotImplementedError

    def _u0grad(self, lam0, u0, gu0):
        raise NotImplementedError

    def _lam(self):
        raise NotImplementedError

    def _field(self):
        raise NotImplementedError

    # -- step sequences: one call per step unless a subclass runs them in bulk --
    def _run(self, fins, fouts):
        for fin, fout in zip(fins, fouts):
            self._step_to(fin, fout)

    def _run_mom(self, fins, fouts, moms):
        for fin, fout, (rho, u) in zip(fins, fouts, moms):
            self._step_mom(fin, fout, rho, u)

    def _reverse(self, moms, lam_a, lam_b, gF):
        """Reverse steps over moms (last forward step first), lambda^{n+1} in
        lam_a; returns (lambda^n, the other buffer)."""
        for rho, u in moms:
            self._adj_step_mom(rho, u, lam_a, lam_b, gF)
            lam_a, lam_b = lam_b, lam_a
        return lam_a, lam_b

    # -- driver -------------------------------------------------------------------
    def _moment_buffers(self, m):
        while len(self._mom_seg) < m:
            self._mom_seg.append(self._mom())
        return self._mom_seg[:m]

    def forward(self, u0, F, keep_tail=False):
        """f^0 = f^eq(1, u0), then T steps keeping every K-th state.
        Returns (f_T, checkpoints); the buffers stay valid until the next
        call of forward(). keep_tail (with moments=True): the last segment's
        steps also write the rho, u their collisions used, so that the next
        backward() need not recompute that segment."""
        if self._scratch is None:
            self._scratch = [self._fbuf(), self._fbuf()]
        self._tail_moments = False
        f0 = self._init(u0, F)
        ckpts = [f0]
        prev = f0
        fins, fouts = [], []
        for n in range(1, self.T + 1):
            if n % self.K == 0 and n < self.T:
                c = len(ckpts) - 1  # checkpoint buffers are reused across calls
                if c == len(self._ckpt_pool):
                    self._ckpt_pool.append(self._fbuf())
                dst = self._ckpt_pool[c]
                ckpts.append(dst)
            else:
                dst = self._scratch[n % 2]
            fins.append(prev)
            fouts.append(dst)
            prev = dst
            if n % self.K == 0 or n == self.T:  # one segment per call
                if n == self.T and keep_tail and self.moments:
                    self._run_mom(fins, fouts, self._moment_buffers(len(fins)))
                    self._tail_moments = True
                else:
                    self._run(fins, fouts)
                fins, fouts = [], []
        return prev, ckpts

    def backward(self, f_T, ckpts, u0, ut):
        """Reverse sweep: (loss, grad_u0, grad_F) as device tensors."""
        lam_a, lam_b = self._lam(), self._lam()
        gF = self._field()
        loss = torch.zeros((), dtype=torch.float64, device=gF.device)
        self._seed(f_T, ut, lam_a, gF, loss)
        if self.moments:
            self._moment_buffers(min(self.K, self.T))
        else:
            need = min(self.K, self.T) - 1
            while len(self._segment) < need:
                self._segment.append(self._fbuf())
        for s in range(len(ckpts) - 1, -1, -1):
            start = s * self.K
            stop = min(start + self.K, self.T)
            if self.moments:
                # f_T (a scratch buffer) is no longer needed after the seed
                m = stop - start
                if not (self._tail_moments and s == len(ckpts) - 1):
                    fins = [ckpts[s]] + [self._scratch[k % 2] for k in range(m - 1)]
                    fouts = [self._scratch[k % 2] for k in range(m)]
                    self._run_mom(fins, fouts, self._mom_seg[:m])
                lam_a, lam_b = self._reverse(self._mom_seg[:m][::-1], lam_a, lam_b, gF)
                continue
            states = [ckpts[s]]
            for k in range(1, stop - start):
                self._step_to(states[-1], self._segment[k - 1])
                states.append(self._segment[k - 1])
            for n in range(stop - 1, start - 1, -1):
                self._adj_step(states[n - start], lam_a, lam_b, gF)
                lam_a, lam_b = lam_b, lam_a
        gu0 = self._field()
        self._u0grad(lam_a, u0, gu0)
        self._tail_moments = False  # the segment buffers now hold the first segment's
        return loss, gu0, gF

    def loss_and_grad(self, u0, F, u_target):
        u0 = u0.detach().float().contiguous()
        F = F.detach().float().contiguous()
        ut = u_target.detach().float().contiguous()
        f_T, ckpts = self.forward(u0, F, keep_tail=True)
        return self.backward(f_T, ckpts, u0, ut)

    def loss(self, u0, F, u_target):
        """Forward loss only (FP64 reduction on the device)."""
        f_T, _ = self.forward(u0.detach().float().contiguous(), F.detach().float().contiguous())
        lam = self._lam()
        out = torch.zeros((), dtype=torch.float64, device=lam.device)
        self._seed(f_T, u_target.detach().float().contiguous(), lam, None, out)
        return out


class AdjointProblem(_Checkpointed):
    """Geometry, tau, horizon T and checkpoint interval K of a
    velocity-mismatch problem on one lattice (FP32 storage)."""

    def __init__(self, nx, ny, nz, tau, T, K=50, walls=(False, False, False), lid=None,
                 device="cuda", moments=True):
        super().__init__(T, K, moments)
        self.lat = Lattice(nx, ny, nz, tau, walls=walls, lid=lid, storage="f32", force=True,
                           device=device)
        self.shape = self.lat.shape
        self.device = self.lat.device
        lay = self.lat.layout
        self.f_bytes = lay.f_bytes
        self.lam_elems = lay.lambda_bytes // 4

    @property
    def launches_forward(self):
        return 1 + self.T

    def _fbuf(self):
        return torch.empty(self.f_bytes, dtype=torch.uint8, device=self.device)

    def _init(self, u0, F):
        self.lat.force.copy_(F)
        self.lat.init_equilibrium(u=u0)
        f0, _ = self.lat.current_buffers()  # init writes the current buffer in place
        return f0

    def _step_to(self, fin, fout):
        self.lat.step_to(fin, fout)

    def _seed(self, fT, ut, lam, gF, loss):
        capi.call("lbm_adjoint_seed", self.lat.handle, _p(fT), _p(ut), _p(lam), _p(gF),
                  _p(loss))

    def _adj_step(self, fn, lam_in, lam_out, gF):
        capi.call("lbm_adjoint_step", self.lat.handle, _p(fn), _p(lam_in), _p(lam_out), _p(gF))

    def _step_mom(self, fin, fout, rho, u):
        capi.call("lbm_step_to_moments", self.lat.handle, _p(fin), _p(fout), _p(rho), _p(u))

    def _adj_step_mom(self, rho, u, lam_in, lam_out, gF):
        capi.call("lbm_adjoint_step_moments", self.lat.handle, _p(rho), _p(u), _p(lam_in),
                  _p(lam_out), _p(gF))

    def _mom(self):
        return (torch.empty(self.shape, dtype=torch.float32, device=self.device),
                torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device))

    def _u0grad(self, lam0, u0, gu0):
        capi.call("lbm_adjoint_u0", self.lat.handle, _p(lam0), _p(u0), _p(gu0))

    def _lam(self):
        return torch.empty(self.lam_elems, dtype=torch.float32, device=self.device)

    def _field(self):
        return torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)


class BatchAdjointProblem(_Checkpointed):
    """The same problem for every domain of a :class:`~.batch.Batch` at once
    (F = 0; the force gradient is taken at F = 0). Fields (u0, u_target and
    the gradients) use the batch's dense per-domain layout, see
    :meth:`~.batch.Batch.pack_vectors`."""

    def __init__(self, batch, T, K=50, moments=True):
        super().__init__(T, K, moments)
        self.b = batch
        self.device = batch.device

    def _fbuf(self):
        return torch.empty(self.b.f_bytes, dtype=torch.uint8, device=self.device)

    def _init(self, u0, F):
        capi.call("lbm_batch_init_equilibrium", self.b.handle, _p(u0))
        f0, _ = self.b.current_buffers()
        return f0

    def _step_to(self, fin, fout):
        capi.call("lbm_batch_step_to", self.b.handle, _p(fin), _p(fout))

    def _seed(self, fT, ut, lam, gF, loss):
        capi.call("lbm_batch_adjoint_seed", self.b.handle, _p(fT), _p(ut), _p(lam), _p(gF),
                  _p(loss))

    def _adj_step(self, fn, lam_in, lam_out, gF):
        capi.call("lbm_batch_adjoint_step", self.b.handle, _p(fn), _p(lam_in), _p(lam_out),
                  _p(gF))

    def _step_mom(self, fin, fout, rho, u):
        capi.call("lbm_batch_step_to_moments", self.b.handle, _p(fin), _p(fout), _p(rho), _p(u))

    def _adj_step_mom(self, rho, u, lam_in, lam_out, gF):
        capi.call("lbm_batch_adjoint_step_moments", self.b.handle, _p(rho), _p(u), _p(lam_in),
                  _p(lam_out), _p(gF))

    def _mom(self):
        return (torch.empty(self.b.cells, dtype=torch.float32, device=self.device),
                torch.empty(3 * self.b.cells, dtype=torch.float32, device=self.device))

    def _u0grad(self, lam0, u0, gu0):
        capi.call("lbm_batch_adjoint_u0", self.b.handle, _p(lam0), _p(u0), _p(gu0))

    def _lam(self):
        return torch.empty(self.b.f_bytes // 4, dtype=torch.float32, device=self.device)

    def _field(self):
        return torch.empty(3 * self.b.cells, dtype=torch.float32, device=self.device)

    # segments, recompute and reverse sweeps as persistent launches of up to
    # 64 steps each (lbm_batch_run, lbm_batch_adjoint_run)
    _CHUNK = 64

    @staticmethod
    def _ptrs(ts):
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def _run(self, fins, fouts):
        for k in range(0, len(fins), self._CHUNK):
            fi, fo = fins[k:k + self._CHUNK], fouts[k:k + self._CHUNK]
            capi.call("lbm_batch_run", self.b.handle, len(fi), self._ptrs(fi), self._ptrs(fo),
                      None, None)

    def _run_mom(self, fins, fouts, moms):
        for k in range(0, len(fins), self._CHUNK):
            fi, fo, mm = fins[k:k + self._CHUNK], fouts[k:k + self._CHUNK], moms[k:k + self._CHUNK]
            capi.call("lbm_batch_run", self.b.handle, len(fi), self._ptrs(fi), self._ptrs(fo),
                      self._ptrs([r for r, _ in mm]), self._ptrs([u for _, u in mm]))

    def _reverse(self, moms, lam_a, lam_b, gF):
        for k in range(0, len(moms), self._CHUNK):
            mm = moms[k:k + self._CHUNK]
            capi.call("lbm_batch_adjoint_run", self.b.handle, len(mm),
                      self._ptrs([r for r, _ in mm]), self._ptrs([u for _, u in mm]),
                      _p(lam_a), _p(lam_b), _p(gF))
            if len(mm) % 2:
                lam_a, lam_b = lam_b, lam_a
        return lam_a, lam_b


class VelocityMismatch(torch.autograd.Function):
    """loss = VelocityMismatch.apply(u0, F, u_target, problem): FP64 scalar
    loss; backward runs the checkpointed adjoint of ``problem``. The saved
    checkpoints live in ``problem``'s buffers, so call backward before the
    next forward on the same problem."""

    @staticmethod
    def forward(ctx, u0, F, u_target, problem):
        u0c = u0.detach().float().contiguous()
        Fc = F.detach().float().contiguous()
        utc = u_target.detach().float().contiguous()
        f_T, ckpts = problem.forward(u0c, Fc, keep_tail=True)
        lam = problem._lam()
        loss = torch.zeros((), dtype=torch.float64, device=u0c.device)
        problem._seed(f_T, utc, lam, None, loss)
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
