"""ctypes wrapper around ``lbm_oracle.c`` (FP64 CPU oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Python-side array conventions, chosen to match the CUDA library's host
exchange format so tests can compare element by element:

* distributions ``f``: float64 array of shape ``(19, nz, ny, nx)``, the plain
  (unshifted) f_i;
* scalar fields (``rho``): shape ``(nz, ny, nx)``;
* vector fields (velocity, force, their gradients): shape ``(3, nz, ny, nx)``.

The C code itself stores f as Array of Structures; the transposes below are
plain numpy layout changes, not arithmetic of the method.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")

Q = 19


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) if the shared object is missing
    or older than its source. Returns the path of the shared object."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _CLattice(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_x", ctypes.c_int), ("wall_y", ctypes.c_int), ("wall_z", ctypes.c_int),
        ("lid", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("lid_u", ctypes.c_double * 3),
        ("onsite", ctypes.c_int),
    ]


_lib = None


def library():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(_CLattice)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_velocity.argtypes = [ctypes.c_int, ip, ip, ip]
        lib.oracle_weight.argtypes = [ctypes.c_int]
        lib.oracle_weight.restype = ctypes.c_double
        lib.oracle_opposite.argtypes = [ctypes.c_int]
        lib.oracle_max_threads.argtypes = []
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        lib.oracle_init_equilibrium.argtypes = [lp, dp, dp, dp]
        lib.oracle_stream.argtypes = [lp, dp, dp]
        lib.oracle_stream_forced.argtypes = [lp, dp, dp, dp]
        lib.oracle_collide.argtypes = [lp, dp, dp, dp]
        lib.oracle_run.argtypes = [lp, dp, dp, ctypes.c_int, dp]
        lib.oracle_moments.argtypes = [lp, dp, dp, dp, dp]
        lib.oracle_adjoint_step.argtypes = [lp, dp, dp, dp, dp, dp]
        lib.oracle_adjoint_seed.argtypes = [lp, dp, dp, dp, dp, dp, dp]
        lib.oracle_adjoint_u0.argtypes = [lp, dp, dp, dp]
        _lib = lib
    return _lib


@dataclass
class Lattice:
    """Geometry and parameters of one lattice (mirrors ``oracle_lattice``).

    ``walls`` is a triple of booleans (x, y, z): a walled axis has halfway
    bounce-back walls at -1/2 and n-1/2, any other axis is periodic.
    ``lid`` (requires a walled z axis) makes the plane z = nz move with
    velocity ``lid_u``. ``onsite`` selects the on-site velocity walls
    instead: the walls lie on the first and last node planes of each walled
    axis (at least 3 nodes long), and the lid is the node plane z = nz - 1
    without its edges.
    """

    nx: int
    ny: int
    nz: int
    tau: float
    walls: tuple = (False, False, False)
    lid: bool = False
    lid_u: tuple = (0.0, 0.0, 0.0)
    onsite: bool = False
    _c: _CLattice = field(default=None, repr=False, compare=False)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz

    def c(self):
        s = _CLattice()
        s.nx, s.ny, s.nz = self.nx, self.ny, self.nz
        s.wall_x, s.wall_y, s.wall_z = (int(bool(w)) for w in self.walls)
        s.lid = int(bool(self.lid))
        s.tau = float(self.tau)
        for a in range(3):
            s.lid_u[a] = float(self.lid_u[a])
        s.onsite = int(bool(self.onsite))
        return s


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _aos(f_soa):
    """(19, nz, ny, nx) -> contiguous AoS (nz, ny, nx, 19)."""
    return np.ascontiguousarray(np.moveaxis(np.asarray(f_soa, dtype=np.float64), 0, -1))


def _soa(f_aos):
    return np.ascontiguousarray(np.moveaxis(f_aos, -1, 0))


def _vec(v, L):
    if v is None:
        return None
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.shape == (3,) + L.shape, v.shape
    return v


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"oracle {name} failed with code {rc}")


def velocity_set() -> np.ndarray:
    """The oracle's e_i table, shape (19, 3)."""
    lib = library()
    out = np.zeros((Q, 3), dtype=int)
    for i in range(Q):
        ex, ey, ez = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.oracle_velocity(i, ctypes.byref(ex), ctypes.byref(ey), ctypes.byref(ez)), "velocity")
        out[i] = (ex.value, ey.value, ez.value)
    return out


def weights() -> np.ndarray:
    lib = library()
    return np.array([lib.oracle_weight(i) for i in range(Q)])


def opposites() -> np.ndarray:
    lib = library()
    return np.array([lib.oracle_opposite(i) for i in range(Q)])


def max_threads() -> int:
    return int(library().oracle_max_threads())


def set_threads(n: int) -> None:
    library().oracle_set_threads(int(n))


def init_equilibrium(L: Lattice, rho=None, u=None) -> np.ndarray:
    """f = f^eq(rho0, u0) (Eq. 5); rho None -> 1, u None -> 0."""
    lib = library()
    c = L.c()
    r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    uu = _vec(u, L)
    f = np.empty(L.shape + (Q,), dtype=np.float64)
    _check(lib.oracle_init_equilibrium(ctypes.byref(c), _dp(r), _dp(uu), _dp(f)), "init")
    return _soa(f)


def stream(L: Lattice, f, force=None) -> np.ndarray:
    """Streaming pass with the boundary rule: g_i(x) = f_i(x - e_i) or its
    bounce-back replacement, or for on-site walls the rebuilt unknown
    populations (whose target momentum rho u_w - F/2 uses the force)."""
    lib = library()
    c = L.c()
    fa = _aos(f)
    g = np.empty_like(fa)
    _check(lib.oracle_stream_forced(ctypes.byref(c), _dp(fa), _dp(_vec(force, L)), _dp(g)),
           "stream")
    return _soa(g)


def collide(L: Lattice, g, force=None) -> np.ndarray:
    """Collision pass (Eqs. 3, 5-7 with the Guo force term)."""
    lib = library()
    c = L.c()
    ga = _aos(g)
    out = np.empty_like(ga)
    _check(lib.oracle_collide(ctypes.byref(c), _dp(ga), _dp(_vec(force, L)), _dp(out)), "collide")
    return _soa(out)


def run(L: Lattice, f, nsteps: int, force=None) -> np.ndarray:
    """``nsteps`` full time steps (stream pass then collide pass each)."""
    lib = library()
    c = L.c()
    fa = _aos(f)
    out = np.empty_like(fa)
    _check(lib.oracle_run(ctypes.byref(c), _dp(fa), _dp(_vec(force, L)), int(nsteps), _dp(out)), "run")
    return _soa(out)


def to_aos(f):
    """(19, nz, ny, nx) -> the oracle's native (nz, ny, nx, 19) layout."""
    return _aos(f)


def run_aos(L: Lattice, f_aos, nsteps: int, force=None) -> np.ndarray:
    """``run`` on an array already in the oracle's native layout (no layout
    changes around the C call; used to time the oracle itself)."""
    lib = library()
    c = L.c()
    assert f_aos.dtype == np.float64 and f_aos.flags["C_CONTIGUOUS"]
    out = np.empty_like(f_aos)
    _check(lib.oracle_run(ctypes.byref(c), _dp(f_aos), _dp(_vec(force, L)), int(nsteps),
                          _dp(out)), "run")
    return out


def moments(L: Lattice, f, force=None):
    """(rho, u) of a stored post-collision state."""
    lib = library()
    c = L.c()
    fa = _aos(f)
    rho = np.empty(L.shape, dtype=np.float64)
    u = np.empty((3,) + L.shape, dtype=np.float64)
    _check(lib.oracle_moments(ctypes.byref(c), _dp(fa), _dp(_vec(force, L)), _dp(rho), _dp(u)), "moments")
    return rho, u


def adjoint_seed(L: Lattice, f_T, u_target, force=None):
    """Returns (loss, lambda_T, direct term dL/dF = -(u - u_t)/(2 rho))."""
    lib = library()
    c = L.c()
    fa = _aos(f_T)
    lam = np.empty_like(fa)
    gF = np.zeros((3,) + L.shape, dtype=np.float64)
    loss = ctypes.c_double()
    _check(lib.oracle_adjoint_seed(ctypes.byref(c), _dp(fa), _dp(_vec(force, L)),
                                   _dp(_vec(u_target, L)), _dp(lam), _dp(gF),
                                   ctypes.byref(loss)), "adjoint_seed")
    return loss.value, _soa(lam), gF


def adjoint_step(L: Lattice, f_n, lam_next, force=None, grad_force=None):
    """lambda^n from lambda^{n+1}; adds the force term into ``grad_force``
    (shape (3, nz, ny, nx), modified in place) when given."""
    lib = library()
    c = L.c()
    fa = _aos(f_n)
    la = _aos(lam_next)
    out = np.empty_like(la)
    gf = None
    if grad_force is not None:
        assert grad_force.dtype == np.float64 and grad_force.flags["C_CONTIGUOUS"]
        gf = grad_force
    _check(lib.oracle_adjoint_step(ctypes.byref(c), _dp(fa), _dp(_vec(force, L)), _dp(la),
                                   _dp(out), _dp(gf)), "adjoint_step")
    return _soa(out)


def adjoint_u0(L: Lattice, lam0, u0):
    lib = library()
    c = L.c()
    la = _aos(lam0)
    g = np.empty((3,) + L.shape, dtype=np.float64)
    _check(lib.oracle_adjoint_u0(ctypes.byref(c), _dp(la), _dp(_vec(u0, L)), _dp(g)), "adjoint_u0")
    return g


def loss_and_gradients(L: Lattice, u0, u_target, nsteps: int, force=None, want_grad=True):
    """Forward f^0 = f^eq(1, u0), ``nsteps`` steps, loss on u(T); then the
    full reverse sweep keeping every state in memory (small lattices only).

    Returns (loss, grad_u0, grad_force)."""
    f = init_equilibrium(L, None, u0)
    states = [f]
    for _ in range(nsteps):
        f = run(L, f, 1, force)
        states.append(f)
    loss, lam, gF = adjoint_seed(L, states[-1], u_target, force)
    if not want_grad:
        return loss, None, None
    for n in range(nsteps - 1, -1, -1):
        lam = adjoint_step(L, states[n], lam, force, gF)
    gu0 = adjoint_u0(L, lam, u0)
    return loss, gu0, gF
