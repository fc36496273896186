"""lbm_moments_noalloc: the allocation-free moments + mass entry point, for
callers that cannot allocate device memory (memory owned by another
allocator, or loops where cudaMalloc/cudaFree would synchronise the device).

It is checked through the C ABI against lbm_moments, the handle-based entry
point (itself checked against the FP64 oracle in test_gpu_forward.py):
* two calls in a row, a larger FP32 lattice with a body force and then a
  smaller FP16 lattice, so the second call runs on scratch that still holds
  the first call's partial sums;
* every storage type (FP32, FP16, BF16);
* the optional outputs left out one at a time (no mass: no reduction and no
  scratch use; no u; no rho).
Tolerances are those of the moment tests: 1e-6 on rho and u, 1e-9 relative
on the FP64 mass. This file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_1309_1983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_1983_gb300 import build as B
    B.build()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _random_state(nx, ny, nz, tau, seed):
    OL = O.Lattice(nx, ny, nz, tau)
    rho = 1.0 + W.noise(OL.shape, seed, 0.02)
    u = W.noise((3,) + OL.shape, seed + 1, 0.05)
    f = O.init_equilibrium(OL, rho, u)
    return f * (1.0 + W.noise(f.shape, seed + 2, 0.1))


def _compare(L, force, want_rho=True, want_u=True, want_mass=True):
    from paper_1309_1983_gb300 import capi
    lib = capi.load()
    rho_ref, u_ref, mass_ref = L.moments(mass=True)
    cur, _ = L.current_buffers()
    rho = torch.full_like(rho_ref, float("nan"))
    u = torch.full_like(u_ref, float("nan"))
    mass = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.lbm_moments_noalloc(_p(cur), L.nx, L.ny, L.nz, L.flags,
                                 None if force is None else _p(force),
                                 _p(rho) if want_rho else None, _p(u) if want_u else None,
                                 _p(mass) if want_mass else None,
                                 ctypes.c_void_p(L.stream.cuda_stream))
    assert rc == capi.LBM_OK, capi.last_error()
    L.stream.synchronize()
    if want_rho:
        torch.testing.assert_close(rho, rho_ref, rtol=0, atol=1e-6)
    else:
        assert torch.isnan(rho).all()  # left untouched
    if want_u:
        torch.testing.assert_close(u, u_ref, rtol=0, atol=1e-6)
    else:
        assert torch.isnan(u).all()
    if want_mass:
        assert abs(mass.item() - mass_ref) <= 1e-9 * abs(mass_ref)
    else:
        assert np.isnan(mass.item())


def test_noalloc_moments_match_handle_moments_twice():
    from paper_1309_1983_gb300.lattice import Lattice
    # first call: larger FP32 lattice with a body force
    L1 = Lattice(50, 30, 20, 0.7, force=True)
    L1.force.copy_(torch.from_numpy(W.noise((3, 20, 30, 50), 7, 1e-3)).float())
    L1.set_f(_random_state(50, 30, 20, 0.7, 1))
    L1.step(3)
    _compare(L1, L1.force)
    # second call in a row: smaller FP16 lattice, no force
    L2 = Lattice(17, 9, 5, 0.6, walls=(True, True, True), lid=(0.05, 0.0, 0.0), storage="f16")
    L2.set_f(_random_state(17, 9, 5, 0.6, 11))
    L2.step(2)
    _compare(L2, None)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("outputs", ["all", "no_mass", "no_u", "no_rho"])
def test_noalloc_storage_types_and_optional_outputs(storage, outputs):
    from paper_1309_1983_gb300.lattice import Lattice
    nx, ny, nz = 37, 12, 7
    L = Lattice(nx, ny, nz, 0.65, walls=(True, False, True), lid=(0.04, 0.0, 0.0),
                storage=storage)
    L.set_f(_random_state(nx, ny, nz, 0.65, 21))
    L.step(2)
    _compare(L, None, want_rho=outputs != "no_rho", want_u=outputs != "no_u",
             want_mass=outputs != "no_mass")


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_1309_1983_gb300 import capi
    from paper_1309_1983_gb300.lattice import Lattice
    L = Lattice(8, 8, 8, 0.7)
    cur, _ = L.current_buffers()
    mass = torch.zeros((), dtype=torch.float64, device="cuda")
    rc = capi.load().lbm_moments_noalloc(_p(cur), 2048, 2048, 1024, 0, None, None, None,
                                         _p(mass), None)
    assert rc == capi.LBM_ERANGE
    assert "2^31" in capi.last_error()
