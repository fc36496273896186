"""Guard-band canaries: no kernel writes outside the buffers it is given.

A memory checker cannot be run on these GPUs, so out-of-bounds WRITES are
looked for directly. Every buffer a kernel writes (f, lambda, rho, u,
gradients, the FP64 loss) is allocated with a trailing guard region of
4 KiB, and the whole allocation (guard, x-row padding of the f and lambda
layouts, gaps between the 256-byte aligned domain regions of a batch) is
filled with the byte 0xFF, a NaN in FP32, FP16 and BF16 alike. States are set
by initialisation kernels that write node elements only; after each group
of kernels every byte outside the node elements must still be 0xFF.

The documented exceptions: the two-node step kernels (LBM_KERNEL_X2, the
default, and LBM_KERNEL_PAIR) load and store the padding element that
follows the last node of an odd-length row, together with that node, and
the four-node kernel (LBM_KERNEL_X4) the padding elements up to the next
multiple of four.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_1309_1983_gb300 import capi
from paper_1309_1983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 4096


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_1983_gb300 import build as B
    B.build()


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _guarded(nbytes):
    """0xFF-filled allocation of nbytes + GUARD; the buffer is its head."""
    return torch.full((nbytes + GUARD,), 0xFF, dtype=torch.uint8, device="cuda")


def _guard_intact(full, nbytes):
    return bool((full[nbytes:] == 0xFF).all())


def _f_outside_intact(full, nbytes, elem_bytes, pitch, nx, ny, nz, pad_written=False,
                      group=2):
    """Guard and row padding of an f-layout buffer [19][nz][ny][pitch];
    with pad_written, the padding up to the next multiple of `group` nodes
    (the multi-node kernels' last group) may have been written."""
    if not _guard_intact(full, nbytes):
        return "guard"
    v = full[:nbytes].view(19, nz, ny, pitch * elem_bytes)
    first = -(-nx // group) * group if pad_written else nx
    pad = v[..., first * elem_bytes:]
    if pad.numel() and not bool((pad == 0xFF).all()):
        return "row padding"
    return None


def _field(shape_or_n):
    n = int(np.prod(shape_or_n))
    full = _guarded(4 * n)
    return full, full[:4 * n].view(torch.float32)


SHAPES = [(37, 6, 5), (20, 3, 4), (33, 1, 3)]
GEOMS = {"periodic": ((False, False, False), None),
         "cavity": ((True, True, True), (0.05, 0.0, 0.0)),
         "walls_y": ((False, True, False), None)}


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("shape", SHAPES)
def test_forward_kernels_write_only_node_elements(storage, geom, shape):
    from paper_1309_1983_gb300.lattice import Lattice
    nx, ny, nz = shape
    walls, lid = GEOMS[geom]
    force = storage == "f32" and geom != "cavity"
    L = Lattice(nx, ny, nz, 0.7, walls=walls, lid=lid, storage=storage, force=force)
    if force:
        L.force.copy_(torch.from_numpy(W.noise((3, nz, ny, nx), 3, 1e-3)).float())
    lay = L.layout
    fb, eb, pitch = lay.f_bytes, lay.elem_bytes, lay.pitch
    A, B = _guarded(fb), _guarded(fb)
    L.f_a, L.f_b = A[:fb], B[:fb]
    L._bind()
    h = L.handle

    group = [2]

    def check(tag, pad_written):
        torch.cuda.synchronize()
        for name, full in (("A", A), ("B", B)):
            bad = _f_outside_intact(full, fb, eb, pitch, nx, ny, nz, pad_written, group[0])
            assert bad is None, (tag, name, bad)

    u0 = torch.from_numpy(W.noise((3, nz, ny, nx), 1, 0.03)).float().cuda()
    L.init_equilibrium(u=u0)
    check("init", False)
    L.step(3)  # default two-node kernel
    check("x2", True)
    kernels = ["node", "bulk", "bulk1"] + (["pair", "tma", "x4"] if storage != "f32" else [])
    for k in kernels:
        L.set_kernel(k)
        if k == "x4":
            group[0] = 4
        L.step(2)
        L.sync()
        check(k, True)
    L.set_kernel("x2")
    L.set_graph_steps(4)
    L.step(9)  # graph replay of 4-launch graphs plus plain launches
    check("graph", True)

    cells = nx * ny * nz
    rf, rho = _field(cells)
    uf, u = _field(3 * cells)
    capi.call("lbm_step_moments", h, 2, _p(rho), _p(u))
    check("step_moments", True)
    capi.call("lbm_moments", h, _p(rho), _p(u), None)
    torch.cuda.synchronize()
    assert _guard_intact(rf, 4 * cells) and _guard_intact(uf, 12 * cells), "moments"
    mass = torch.zeros((), dtype=torch.float64, device="cuda")
    capi.call("lbm_moments", h, _p(rho), _p(u), ctypes.byref(ctypes.c_double()))
    capi.call("lbm_moments_noalloc", _p(L.current_buffers()[0]), nx, ny, nz, L.flags,
              _p(L.force), _p(rho), _p(u), _p(mass), ctypes.c_void_p(L.stream.cuda_stream))
    torch.cuda.synchronize()
    assert _guard_intact(rf, 4 * cells) and _guard_intact(uf, 12 * cells), "noalloc"

    cur, other = L.current_buffers()
    for form in ("pull", "push", "copy", "pull_l2"):
        L.streaming(cur, other, form)
        check("stream " + form, True)
    L.step_push(cur, other)
    check("push", True)
    L.step_to(cur, other)
    check("step_to", True)
    L.step_to_moments(cur, other, rho, u)
    check("step_to_moments", True)
    torch.cuda.synchronize()
    assert _guard_intact(rf, 4 * cells) and _guard_intact(uf, 12 * cells), "step_to_moments"
    assert torch.isfinite(rho).all() and torch.isfinite(u).all()


@pytest.mark.parametrize("geom", ["periodic", "cavity"])
@pytest.mark.parametrize("shape", SHAPES[:2])
def test_adjoint_kernels_write_only_node_elements(geom, shape):
    from paper_1309_1983_gb300.lattice import Lattice
    nx, ny, nz = shape
    walls, lid = GEOMS[geom]
    force = geom == "periodic"
    L = Lattice(nx, ny, nz, 0.7, walls=walls, lid=lid, force=force)
    if force:
        L.force.copy_(torch.from_numpy(W.noise((3, nz, ny, nx), 3, 1e-3)).float())
    lay = L.layout
    fb, lb, pitch = lay.f_bytes, lay.lambda_bytes, lay.pitch
    cells = nx * ny * nz
    A, B = _guarded(fb), _guarded(fb)
    L.f_a, L.f_b = A[:fb], B[:fb]
    L._bind()
    h = L.handle
    L.init_equilibrium(u=torch.from_numpy(W.noise((3, nz, ny, nx), 2, 0.03)).float().cuda())
    L.step(4)
    fn, fT = L.current_buffers()
    L.step_to(fn, fT)  # f^T = one step from f^n

    lam = [_guarded(lb), _guarded(lb)]
    gFf, gF = _field(3 * cells)
    gF.zero_()
    rf, rho = _field(cells)
    uf, u = _field(3 * cells)
    guf, gu0 = _field(3 * cells)
    lossf = _guarded(8)
    ut = torch.from_numpy(W.noise((3, nz, ny, nx), 4, 0.01)).float().cuda()
    u0 = torch.from_numpy(W.noise((3, nz, ny, nx), 5, 0.01)).float().cuda()

    def check(tag):
        torch.cuda.synchronize()
        for k, full in enumerate(lam):
            bad = _f_outside_intact(full, lb, 4, pitch, nx, ny, nz)
            assert bad is None, (tag, "lambda", k, bad)
        for name, full, n in (("gF", gFf, 12 * cells), ("rho", rf, 4 * cells),
                              ("u", uf, 12 * cells), ("gu0", guf, 12 * cells),
                              ("loss", lossf, 8)):
            assert _guard_intact(full, n), (tag, name)
        for name, full in (("A", A), ("B", B)):
            bad = _f_outside_intact(full, fb, 4, pitch, nx, ny, nz, pad_written=True)
            assert bad is None, (tag, name, bad)

    capi.call("lbm_adjoint_seed", h, _p(fT), _p(ut), _p(lam[0]), _p(gF), _p(lossf))
    check("seed")
    for mode in ("select", "branch"):
        L.set_wall_mode(mode)
        capi.call("lbm_adjoint_step", h, _p(fn), _p(lam[0]), _p(lam[1]), _p(gF))
        check("adjoint_step")
        capi.call("lbm_step_to_moments", h, _p(fn), _p(fT), _p(rho), _p(u))
        capi.call("lbm_adjoint_step_moments", h, _p(rho), _p(u), _p(lam[1]), _p(lam[0]), _p(gF))
        check("adjoint_step_moments")
    capi.call("lbm_adjoint_u0", h, _p(lam[0]), _p(u0), _p(gu0))
    check("u0")
    assert torch.isfinite(gu0).all() and torch.isfinite(gF).all()


def test_batch_kernels_write_only_node_elements():
    """Ragged domains whose f regions leave gaps before the next 256-byte
    aligned region; persistent launch, plain launches, moments and the
    adjoint kernels keep every gap and the trailing guard intact."""
    from paper_1309_1983_gb300.batch import Batch
    dims = [(17, 5, 9), (33, 16, 4), (1, 6, 7), (40, 3, 3), (9, 7, 5)]
    tau = [0.55, 0.7, 0.9, 1.0, 0.62]
    lid = [0.02, 0.05, 0.08, 0.03, 0.06]
    Bt = Batch(dims, tau, lid)
    fb, cells = Bt.f_bytes, Bt.cells
    A, B = _guarded(fb), _guarded(fb)
    Bt.f_a, Bt.f_b = A[:fb], B[:fb]
    capi.call("lbm_batch_bind", Bt.handle, _p(Bt.f_a), _p(Bt.f_b),
              ctypes.c_void_p(Bt.stream.cuda_stream))
    # node elements of every domain region (FP32, unpadded rows)
    node = torch.zeros(fb // 4, dtype=torch.bool, device="cuda")
    for d, (nx, ny, nz) in enumerate(dims):
        o = int(Bt.f_offsets[d])
        node[o:o + 19 * nx * ny * nz] = True
    assert int((~node).sum()) > 0, "no gaps between domain regions to watch"

    def outside_intact(full, nbytes):
        if not _guard_intact(full, nbytes):
            return "guard"
        words = full[:nbytes].view(torch.int32)
        if not bool((words[~node] == -1).all()):
            return "gap between domains"
        return None

    lam = [_guarded(fb), _guarded(fb)]
    fields = {k: _field(n) for k, n in (("rho", cells), ("u", 3 * cells), ("gF", 3 * cells),
                                        ("gu0", 3 * cells))}
    lossf = _guarded(8)

    def check(tag):
        torch.cuda.synchronize()
        for name, full in (("A", A), ("B", B), ("lam0", lam[0]), ("lam1", lam[1])):
            bad = outside_intact(full, fb)
            assert bad is None, (tag, name, bad)
        for name, (full, t) in fields.items():
            assert _guard_intact(full, 4 * t.numel()), (tag, name)
        assert _guard_intact(lossf, 8), (tag, "loss")

    u0 = Bt.pack_vectors([W.noise((3, nz, ny, nx), 7 + d, 0.02)
                          for d, (nx, ny, nz) in enumerate(dims)])
    Bt.init_equilibrium(u0)
    check("init_eq")
    Bt.init_rest()
    check("init_rest")
    Bt.init_equilibrium(u0)
    Bt.step(5)
    check("persistent")
    Bt.step_launches(3)
    check("launches")
    rho, u = fields["rho"][1], fields["u"][1]
    capi.call("lbm_batch_moments", Bt.handle, _p(rho), _p(u))
    check("moments")
    fn, fT = Bt.current_buffers()
    capi.call("lbm_batch_step_to", Bt.handle, _p(fn), _p(fT))
    check("step_to")
    gF, gu0 = fields["gF"][1], fields["gu0"][1]
    gF.zero_()
    ut = torch.zeros(3 * cells, dtype=torch.float32, device="cuda")
    capi.call("lbm_batch_adjoint_seed", Bt.handle, _p(fT), _p(ut), _p(lam[0]), _p(gF), _p(lossf))
    check("seed")
    capi.call("lbm_batch_adjoint_step", Bt.handle, _p(fn), _p(lam[0]), _p(lam[1]), _p(gF))
    check("adjoint_step")
    capi.call("lbm_batch_step_to_moments", Bt.handle, _p(fn), _p(fT), _p(rho), _p(u))
    capi.call("lbm_batch_adjoint_step_moments", Bt.handle, _p(rho), _p(u), _p(lam[1]),
              _p(lam[0]), _p(gF))
    check("adjoint_step_moments")
    capi.call("lbm_batch_adjoint_u0", Bt.handle, _p(lam[0]), _p(u0), _p(gu0))
    check("u0")
    assert torch.isfinite(gu0).all() and torch.isfinite(gF).all()
