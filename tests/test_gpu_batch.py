"""The batched persistent path against the FP64 oracle, per domain."""

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


def _olat(dims, tau, lid):
    nx, ny, nz = (int(v) for v in dims)
    return O.Lattice(nx, ny, nz, float(np.float32(tau)), walls=(True, True, True), lid=True,
                     lid_u=(float(np.float32(lid)), 0.0, 0.0))


SMALL_DIMS = [(17, 5, 9), (33, 16, 4), (1, 6, 7), (40, 3, 3), (8, 8, 8)]


def _small_batch():
    from paper_1309_1983_gb300.batch import Batch
    tau = [0.55, 0.7, 0.9, 1.0, 0.62]
    lid = [0.02, 0.05, 0.08, 0.03, 0.06]
    return Batch(SMALL_DIMS, tau, lid), tau, lid


def _random_f(OL, seed):
    rho = 1.0 + W.noise(OL.shape, seed, 0.02)
    u = W.noise((3,) + OL.shape, seed + 1, 0.05)
    f = O.init_equilibrium(OL, rho, u)
    return f * (1.0 + W.noise(f.shape, seed + 2, 0.1))


def test_persistent_steps_match_oracle_per_domain():
    B, tau, lid = _small_batch()
    refs = []
    for d, dims in enumerate(SMALL_DIMS):
        OL = _olat(dims, tau[d], lid[d])
        f0 = _random_f(OL, 10 * d + 1)
        B.set_f(d, f0)
        refs.append((OL, f0))
    B.step(7)
    assert B.info()["graph"], "the persistent launch was not replayed from a CUDA graph"
    for d, (OL, f0) in enumerate(refs):
        ref = O.run(OL, f0, 7)
        assert np.abs(B.get_f(d) - ref).max() <= 1e-6, d


@pytest.mark.parametrize("threads,bps", [(256, 0), (128, 0), (64, 2), (32, 1)])
def test_tilings_and_launch_modes_agree(threads, bps):
    B, _, _ = _small_batch()
    B.init_rest()
    B.step_launches(6)
    ref = [B.get_f(d) for d in range(B.ndom)]
    B.set_tiling(threads, bps)
    B.init_rest()
    B.step(6)
    for d in range(B.ndom):
        np.testing.assert_array_equal(B.get_f(d), ref[d])
    B.use_graph(False)
    B.init_rest()
    B.step(6)
    for d in range(B.ndom):
        np.testing.assert_array_equal(B.get_f(d), ref[d])


def test_batch_moments_layout():
    B, tau, lid = _small_batch()
    B.init_rest()
    B.step(30)
    rho, u = B.moments()
    for d, dims in enumerate(SMALL_DIMS):
        OL = _olat(dims, tau[d], lid[d])
        rr, ur = O.moments(OL, B.get_f(d))
        r, v = B.domain_fields(rho, u, d)
        np.testing.assert_allclose(r.double().cpu().numpy(), rr, rtol=0, atol=1e-6)
        np.testing.assert_allclose(v.double().cpu().numpy(), ur, rtol=0, atol=1e-6)


def test_sixty_four_cavities_2000_steps():
    """The seeded 64-cavity workload (edges 16..96, tau in [0.55, 1], lid in
    [0.02, 0.08]): 2000 steps in one persistent launch; the three smallest
    domains against the oracle (rho, u within 1e-5 of the field maximum),
    every domain's mass conserved."""
    from paper_1309_1983_gb300.batch import Batch
    G = W.batch_geometry(64, seed=3)
    B = Batch(G.dims, G.tau, G.lid_u)
    B.init_rest()
    B.step(2000)
    rho, u = B.moments()
    cells = G.dims.prod(axis=1)
    for d in range(64):
        r, _ = B.domain_fields(rho, u, d)
        assert abs(r.double().sum().item() / cells[d] - 1.0) < 1e-6, d
    for d in np.argsort(cells)[:3]:
        OL = _olat(G.dims[d], G.tau[d], G.lid_u[d])
        fr = O.run(OL, O.init_equilibrium(OL), 2000)
        rr, ur = O.moments(OL, fr)
        r, v = B.domain_fields(rho, u, d)
        er = np.abs(r.double().cpu().numpy() - rr).max()
        eu = np.abs(v.double().cpu().numpy() - ur).max() / np.abs(ur).max()
        assert er <= 1e-5 and eu <= 1e-5, (d, er, eu)


def test_barrier_timeout_is_reported_and_context_survives():
    """Host-side fault injection: the grid barrier expects one block more than
    the launch has. Every wait gives up after 50 ms, the kernel returns, the
    call reports LBM_ETIMEOUT, and the next launch on the same context works."""
    from paper_1309_1983_gb300 import capi
    B, _, _ = _small_batch()
    B.init_rest()
    B.set_timeout(0.05)
    B.inject_barrier_fault(1)
    with pytest.raises(capi.LBMError) as e:
        B.step(3)
    assert e.value.code == capi.LBM_ETIMEOUT
    B.inject_barrier_fault(0)
    B.set_timeout(1.0)
    B.init_rest()
    B.step(4)
    B.step_launches(0)
    ref = B.get_f(0)
    assert np.isfinite(ref).all()
    torch.cuda.synchronize()


def test_batched_adjoint_matches_oracle_per_domain():
    """Checkpointed adjoint over a batch of uneven cavities: the loss is the
    sum of the per-domain losses and every domain's gradients (with respect
    to its initial velocity and, at F = 0, its body force) match the FP64
    oracle's adjoint of that domain (1e-4 relative L2)."""
    from paper_1309_1983_gb300.adjoint import BatchAdjointProblem
    from paper_1309_1983_gb300.batch import Batch
    dims = [(12, 9, 7), (7, 10, 11), (16, 5, 6)]
    tau = [0.6, 0.75, 0.9]
    lid = [0.05, 0.03, 0.04]
    B = Batch(dims, tau, lid)
    T, K = 10, 4
    P = BatchAdjointProblem(B, T, K)
    u0s = [W.fourier_modes(*d, seed=10 + k, kmax=2.0, amp=0.02) for k, d in enumerate(dims)]
    uts = [W.fourier_modes(*d, seed=20 + k, kmax=2.0, amp=0.02) for k, d in enumerate(dims)]
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    u0 = B.pack_vectors([r32(a) for a in u0s])
    ut = B.pack_vectors([r32(a) for a in uts])
    F = torch.zeros_like(u0)
    loss, gu0, gF = P.loss_and_grad(u0, F, ut)
    gu0s, gFs = B.unpack_vectors(gu0), B.unpack_vectors(gF)
    total = 0.0
    for k, d in enumerate(dims):
        OL = _olat(d, tau[k], lid[k])
        l, g_u0, g_F = O.loss_and_gradients(OL, r32(u0s[k]), r32(uts[k]), T, None)
        total += l
        for got, ref in ((gu0s[k], g_u0), (gFs[k], g_F)):
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel <= 1e-4, (k, rel)
    assert abs(loss.item() - total) <= 1e-4 * total


def test_batched_adjoint_forms_agree():
    """Batched checkpointed adjoint: segment moments (default) and
    re-gathered segment states give the same bits."""
    from paper_1309_1983_gb300.adjoint import BatchAdjointProblem
    from paper_1309_1983_gb300.batch import Batch
    dims = [(12, 9, 7), (7, 10, 11), (16, 5, 6)]
    res = []
    for moments in (True, False):
        B = Batch(dims, [0.6, 0.75, 0.9], [0.05, 0.03, 0.04])
        P = BatchAdjointProblem(B, 11, 4, moments=moments)
        u0 = B.pack_vectors([W.fourier_modes(*d, seed=30 + k, kmax=2.0, amp=0.02)
                             for k, d in enumerate(dims)])
        ut = B.pack_vectors([W.fourier_modes(*d, seed=40 + k, kmax=2.0, amp=0.02)
                             for k, d in enumerate(dims)])
        res.append([t.cpu().numpy() for t in P.loss_and_grad(u0, torch.zeros_like(u0), ut)])
    for a, b in zip(*res):
        np.testing.assert_array_equal(a, b)


def _axis_block(n, c):
    """Indices of the oracle block along one walled axis, and the node's
    position in it: the node and its neighbours, cut at the walls."""
    lo, hi = max(c - 1, 0), min(c + 1, n - 1)
    return list(range(lo, hi + 1)), c - lo


def _large_domain_samples(nx, ny, nz, threads, rng, count=48):
    """Corners, face centres, and nodes on both sides of tile boundaries
    (tiles are `threads` consecutive nodes in dense order), including tiles
    that cross from one z plane into the next; then random nodes."""
    def node(dc):
        return (dc % nx, (dc // nx) % ny, dc // (nx * ny))
    pts = {(x, y, z) for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)}
    pts |= {(nx // 2, ny // 2, 0), (nx // 2, ny // 2, nz - 1), (0, ny // 2, nz // 2),
            (nx - 1, ny // 2, nz // 2), (nx // 2, 0, nz // 2), (nx // 2, ny - 1, nz // 2)}
    plane, cells = nx * ny, nx * ny * nz
    crossing = [k for k in range(1, nz) if (k * plane) % threads != 0]
    for k in crossing[:4] + crossing[-2:]:  # z-plane seam inside a tile
        pts |= {node(k * plane - 1), node(k * plane)}
    for t in (1, 2, cells // threads // 2, cells // threads - 1):  # tile seams
        if 0 < t * threads < cells:
            pts |= {node(t * threads - 1), node(t * threads)}
    while len(pts) < count:
        pts.add((int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))))
    return sorted(pts)


@pytest.mark.parametrize("tiling", [None, (128, 0)])
def test_sixty_four_cavities_large_domains_sampled_parity(tiling):
    """One persistent step of the seeded 64-cavity workload from random
    non-equilibrium states in its five largest domains; on >= 48 sampled
    nodes per domain (corners, faces, both sides of tile seams and of tiles
    that cross a z plane, random nodes) f^{n+1} matches one oracle step on
    the node's neighbourhood block within 1e-6. These domains (up to 96^3
    nodes) reach tile indices and node decodes the small-domain tests do
    not."""
    from paper_1309_1983_gb300.batch import Batch
    G = W.batch_geometry(64, seed=3)
    B = Batch(G.dims, G.tau, G.lid_u)
    if tiling:
        B.set_tiling(*tiling)
    threads = B.info()["threads"]
    B.init_rest()
    cells = G.dims.prod(axis=1)
    large = [int(d) for d in np.argsort(cells)[-5:]]
    rng = np.random.default_rng(5)
    blocks = {}
    for d in large:
        OL = _olat(G.dims[d], G.tau[d], G.lid_u[d])
        f0 = _random_f(OL, 100 + d)
        B.set_f(d, f0)
        nx, ny, nz = OL.nx, OL.ny, OL.nz
        samples = _large_domain_samples(nx, ny, nz, threads, rng)
        assert len(samples) >= 48
        blocks[d] = []
        for (x, y, z) in samples:
            xi, cx = _axis_block(nx, x)
            yi, cy = _axis_block(ny, y)
            zi, cz = _axis_block(nz, z)
            sub = np.ascontiguousarray(f0[:, zi][:, :, yi][:, :, :, xi])
            # the block is walled (or lid-covered) only where it touches the
            # lattice's own faces; a cut inside the lattice would be wrong for
            # the node's neighbours but not for the node itself, whose pulls
            # all come from inside the block
            OB = O.Lattice(len(xi), len(yi), len(zi), OL.tau, walls=(True, True, True),
                           lid=zi[-1] == nz - 1, lid_u=OL.lid_u)
            blocks[d].append(((x, y, z), sub, OB, (cx, cy, cz)))
    B.step(1)
    assert B.info()["graph"]
    for d in large:
        f1 = B.get_f(d)
        worst = 0.0
        for (x, y, z), sub, OB, (cx, cy, cz) in blocks[d]:
            ref = O.run(OB, sub, 1)[:, cz, cy, cx]
            worst = max(worst, float(np.abs(f1[:, z, y, x] - ref).max()))
        assert worst <= 1e-6, (d, tuple(G.dims[d]), worst)


def _ptrs(ts):
    import ctypes
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def test_step_sequences_equal_single_launches():
    """lbm_batch_run (forward steps with moments) and lbm_batch_adjoint_run
    (reverse steps from those moments), each one persistent launch, give
    the bits of the same steps launched one by one."""
    import ctypes
    from paper_1309_1983_gb300 import capi
    B, tau, lid = _small_batch()
    for d, dims in enumerate(SMALL_DIMS):
        B.set_f(d, _random_f(_olat(dims, tau[d], lid[d]), 50 + d))
    f0, _ = B.current_buffers()
    n = 5
    buf = lambda: torch.empty(B.f_bytes, dtype=torch.uint8, device="cuda")
    field = lambda c: torch.empty(c * B.cells, dtype=torch.float32, device="cuda")
    outs = [[buf() for _ in range(n)] for _ in range(2)]
    moms = [[(field(1), field(3)) for _ in range(n)] for _ in range(2)]
    # one by one
    prev = f0
    for k in range(n):
        capi.call("lbm_batch_step_to_moments", B.handle, ctypes.c_void_p(prev.data_ptr()),
                  ctypes.c_void_p(outs[0][k].data_ptr()), ctypes.c_void_p(moms[0][k][0].data_ptr()),
                  ctypes.c_void_p(moms[0][k][1].data_ptr()))
        prev = outs[0][k]
    # one persistent launch
    fins = [f0] + outs[1][:-1]
    capi.call("lbm_batch_run", B.handle, n, _ptrs(fins), _ptrs(outs[1]),
              _ptrs([m[0] for m in moms[1]]), _ptrs([m[1] for m in moms[1]]))
    torch.cuda.synchronize()
    regions = [(int(B.f_offsets[d]), 19 * nx * ny * nz) for d, (nx, ny, nz) in enumerate(SMALL_DIMS)]
    for k in range(n):
        a, b = outs[0][k].view(torch.float32), outs[1][k].view(torch.float32)
        for o, m in regions:  # node elements (the gaps between regions are not state)
            assert torch.equal(a[o:o + m], b[o:o + m]), k
        assert torch.equal(moms[0][k][0], moms[1][k][0]) and torch.equal(moms[0][k][1], moms[1][k][1])
    # reverse: lambda seeded with noise, force gradient accumulated
    lam0 = torch.from_numpy(W.noise(B.f_bytes // 4, 7, 1e-2)).float().cuda()
    res = []
    for mode in ("single", "run"):
        la, lb = lam0.clone(), torch.zeros_like(lam0)
        gF = torch.zeros(3 * B.cells, dtype=torch.float32, device="cuda")
        rev = moms[0][::-1]
        if mode == "single":
            for r, u in rev:
                capi.call("lbm_batch_adjoint_step_moments", B.handle, ctypes.c_void_p(r.data_ptr()),
                          ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(la.data_ptr()),
                          ctypes.c_void_p(lb.data_ptr()), ctypes.c_void_p(gF.data_ptr()))
                la, lb = lb, la
        else:
            capi.call("lbm_batch_adjoint_run", B.handle, n, _ptrs([r for r, _ in rev]),
                      _ptrs([u for _, u in rev]), ctypes.c_void_p(la.data_ptr()),
                      ctypes.c_void_p(lb.data_ptr()), ctypes.c_void_p(gF.data_ptr()))
            la, lb = (lb, la) if n % 2 else (la, lb)
        res.append((la, gF))
    torch.cuda.synchronize()
    for o, m in regions:
        assert torch.equal(res[0][0][o:o + m], res[1][0][o:o + m])
    assert torch.equal(res[0][1], res[1][1])


def test_sequence_barrier_timeout_is_reported():
    """The step-sequence launches stop at a barrier that cannot complete
    (host-side fault injection) and report LBM_ETIMEOUT; the context keeps
    working."""
    import ctypes
    from paper_1309_1983_gb300 import capi
    B, _, _ = _small_batch()
    B.init_rest()
    f0, f1 = B.current_buffers()
    field = lambda c: torch.zeros(c * B.cells, dtype=torch.float32, device="cuda")
    lam = [torch.zeros(B.f_bytes // 4, dtype=torch.float32, device="cuda") for _ in range(2)]
    r, u = field(1) + 1.0, field(3)
    B.set_timeout(0.05)
    B.inject_barrier_fault(1)
    lib = capi.load()
    rc = lib.lbm_batch_run(B.handle, 3, _ptrs([f0, f1, f0]), _ptrs([f1, f0, f1]), None, None)
    assert rc == capi.LBM_ETIMEOUT
    rc = lib.lbm_batch_adjoint_run(B.handle, 3, _ptrs([r] * 3), _ptrs([u] * 3),
                                   ctypes.c_void_p(lam[0].data_ptr()),
                                   ctypes.c_void_p(lam[1].data_ptr()), None)
    assert rc == capi.LBM_ETIMEOUT
    B.inject_barrier_fault(0)
    B.set_timeout(1.0)
    B.init_rest()
    rc = lib.lbm_batch_run(B.handle, 3, _ptrs([f0, f1, f0]), _ptrs([f1, f0, f1]), None, None)
    assert rc == capi.LBM_OK
    torch.cuda.synchronize()


def test_batched_adjoint_long_segments_are_chunked():
    """Segments longer than one sequence launch (K = 70 > 64) run as
    several launches and still give the bits of the re-gathering form."""
    from paper_1309_1983_gb300.adjoint import BatchAdjointProblem
    from paper_1309_1983_gb300.batch import Batch
    dims = [(9, 8, 7), (6, 10, 5)]
    res = []
    for moments in (True, False):
        B = Batch(dims, [0.7, 0.8], [0.04, 0.03])
        P = BatchAdjointProblem(B, 75, 70, moments=moments)
        u0 = B.pack_vectors([W.fourier_modes(*d, seed=60 + k, kmax=2.0, amp=0.02)
                             for k, d in enumerate(dims)])
        ut = B.pack_vectors([W.fourier_modes(*d, seed=70 + k, kmax=2.0, amp=0.02)
                             for k, d in enumerate(dims)])
        res.append([t.cpu().numpy() for t in P.loss_and_grad(u0, torch.zeros_like(u0), ut)])
    for a, b in zip(*res):
        np.testing.assert_array_equal(a, b)
