"""Host-side checks of liblbm.so that need no GPU: the library loads, exports
every function declared in include/lbm.h, and rejects bad arguments before
any CUDA call."""

import ctypes

import numpy as np
import pytest

from paper_1309_1983_gb300 import build as B
from paper_1309_1983_gb300 import capi


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.load()


def test_every_declared_symbol_is_exported(lib):
    names = capi.header_symbols()
    assert "lbm_create" in names and "lbm_step" in names and "lbm_moments" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(capi.header_symbols()) <= set(capi._SIGNATURES)


def test_strerror_names_every_code(lib):
    for code in range(0, -9, -1):
        s = capi.strerror(code)
        assert s.startswith("LBM_"), s
    assert "unknown" in capi.strerror(-99)


@pytest.mark.parametrize("args,code", [
    ((0, 4, 4, 0.8, 0), capi.LBM_EINVAL),
    ((4, -1, 4, 0.8, 0), capi.LBM_EINVAL),
    ((4, 4, 4, 0.5, 0), capi.LBM_EINVAL),
    ((4, 4, 4, float("nan"), 0), capi.LBM_EINVAL),
    ((4, 4, 4, 0.8, capi.LBM_LID), capi.LBM_EINVAL),
    ((4, 4, 4, 0.8, capi.LBM_STORE_F16 | capi.LBM_STORE_BF16), capi.LBM_EINVAL),
    ((4, 4, 4, 0.8, 0x1000), capi.LBM_EINVAL),
    ((2048, 2048, 1024, 0.8, 0), capi.LBM_ERANGE),
    # on-site walls need 3 nodes along every walled axis, and no adjoint
    ((4, 2, 4, 0.8, capi.LBM_WALLS_ONSITE | capi.LBM_WALL_Y), capi.LBM_EINVAL),
    ((4, 4, 4, 0.8, capi.LBM_WALLS_ONSITE | capi.LBM_CAVITY | capi.LBM_ADJOINT),
     capi.LBM_EINVAL),
])
def test_create_rejects_bad_arguments(lib, args, code):
    h = ctypes.c_void_p()
    assert lib.lbm_create(*args, ctypes.byref(h)) == code
    assert h.value is None
    assert capi.last_error() != ""


@pytest.mark.parametrize("storage,eb,align", [
    (capi.LBM_STORE_F32, 4, 8), (capi.LBM_STORE_F16, 2, 16), (capi.LBM_STORE_BF16, 2, 16)])
def test_layout(lib, storage, eb, align):
    h = capi.create(37, 11, 9, 0.8, storage)
    try:
        L = capi.layout(h)
        assert (L.nx, L.ny, L.nz) == (37, 11, 9)
        assert L.pitch % align == 0 and L.pitch >= 37 and L.pitch < 37 + align
        assert L.plane == L.pitch * 11 * 9
        assert L.f_bytes == 19 * L.plane * eb
        assert L.elem_bytes == eb
        assert L.cells == 37 * 11 * 9
        assert (L.pitch * eb) % 32 == 0
    finally:
        lib.lbm_destroy(h)


def test_unbound_handle_is_reported(lib):
    h = capi.create(8, 8, 8, 0.8, capi.LBM_CAVITY)
    try:
        assert lib.lbm_step(h, 1) == capi.LBM_EUNBOUND
        assert lib.lbm_moments(h, None, None, None) == capi.LBM_EUNBOUND
        assert lib.lbm_sync(h) == capi.LBM_EUNBOUND
        assert lib.lbm_set_lid(h, ctypes.c_float(0.05), ctypes.c_float(0), ctypes.c_float(0)) == 0
        assert lib.lbm_set_tau(h, ctypes.c_float(0.4)) == capi.LBM_EINVAL
        assert lib.lbm_set_block(h, 48, 1) == capi.LBM_EINVAL
        assert lib.lbm_set_block(h, 128, 4) == capi.LBM_EINVAL
        assert lib.lbm_set_block(h, 64, 4) == 0
        assert lib.lbm_autotune(h, None, 5, None, None, None) == capi.LBM_EUNBOUND
    finally:
        lib.lbm_destroy(h)


def test_buffer_bytes_match_layout(lib):
    h = capi.create(37, 11, 9, 0.8, capi.LBM_STORE_F16)
    try:
        L = capi.layout(h)
        want = {capi.LBM_BUF_F: L.f_bytes, capi.LBM_BUF_FORCE: 12 * L.cells,
                capi.LBM_BUF_RHO: 4 * L.cells, capi.LBM_BUF_U: 12 * L.cells,
                capi.LBM_BUF_LAMBDA: L.lambda_bytes, capi.LBM_BUF_GRADF: 12 * L.cells}
        for which, nbytes in want.items():
            b = ctypes.c_size_t()
            assert lib.lbm_buffer_bytes(h, which, ctypes.byref(b)) == 0
            assert b.value == nbytes, which
        b = ctypes.c_size_t()
        assert lib.lbm_buffer_bytes(h, 6, ctypes.byref(b)) == capi.LBM_EINVAL
        assert lib.lbm_buffer_bytes(h, 0, None) == capi.LBM_EINVAL
    finally:
        lib.lbm_destroy(h)


def test_adjoint_flag_needs_fp32(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_create(8, 8, 8, ctypes.c_float(0.8), capi.LBM_ADJOINT | capi.LBM_STORE_BF16,
                          ctypes.byref(h)) == capi.LBM_EINVAL
    assert lib.lbm_create(8, 8, 8, ctypes.c_float(0.8), capi.LBM_ADJOINT | capi.LBM_CAVITY,
                          ctypes.byref(h)) == 0
    lib.lbm_destroy(h)


def test_graph_steps_validation(lib):
    h = capi.create(8, 8, 8, 0.8, 0)
    try:
        for bad in (-2, 3, 1026):
            assert lib.lbm_set_graph_steps(h, bad) == capi.LBM_EINVAL
        for ok in (0, 2, 64, 1024):
            assert lib.lbm_set_graph_steps(h, ok) == 0
    finally:
        lib.lbm_destroy(h)
    assert lib.lbm_set_graph_steps(None, 2) == capi.LBM_EINVAL


def test_autotune_rejects_bad_arguments(lib):
    assert lib.lbm_autotune(None, None, 5, None, None, None) == capi.LBM_EINVAL
    assert lib.lbm_batch_autotune(None, None, 5, None, None, None) == capi.LBM_EINVAL


def test_lid_needs_lid_flag(lib):
    h = capi.create(8, 8, 8, 0.8, capi.LBM_WALL_Z)
    try:
        assert lib.lbm_set_lid(h, ctypes.c_float(0.05), ctypes.c_float(0), ctypes.c_float(0)) \
            == capi.LBM_EINVAL
    finally:
        lib.lbm_destroy(h)


def test_destroy_accepts_null(lib):
    assert lib.lbm_destroy(None) == 0


def test_batch_create_validation(lib):
    def create(ndom, dims, tau, flags=capi.LBM_CAVITY):
        d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1))
        t = np.ascontiguousarray(np.asarray(tau, dtype=np.float32).reshape(-1))
        h = ctypes.c_void_p()
        rc = lib.lbm_batch_create(ndom, d.ctypes.data_as(ctypes.c_void_p),
                                  t.ctypes.data_as(ctypes.c_void_p), None, flags,
                                  ctypes.byref(h))
        if rc == 0:
            lib.lbm_batch_destroy(h)
        else:
            assert h.value is None
        return rc
    assert create(1, [8, 8, 8], [0.6]) == 0
    assert create(0, [8, 8, 8], [0.6]) == capi.LBM_EINVAL            # no domain
    assert create(2, [8, 8, 8, 0, 4, 4], [0.6, 0.7]) == capi.LBM_EINVAL  # empty domain
    assert create(1, [8, 8, 8], [0.5]) == capi.LBM_EINVAL             # tau = 1/2
    assert create(1, [8, 8, 8], [0.6], capi.LBM_STORE_F16) == capi.LBM_EINVAL
    assert create(1, [8, 8, 8], [0.6], capi.LBM_LID) == capi.LBM_EINVAL  # lid without z wall
    assert create(1, [256, 128, 129], [0.6]) == capi.LBM_ERANGE       # > 2^22 nodes
    many = 257
    assert create(many, [4, 4, 4] * many, [0.6] * many) == capi.LBM_ERANGE


def test_moments_form_entry_points_validate(lib):
    nul = ctypes.c_void_p()
    assert lib.lbm_step_to_moments(None, nul, nul, nul, nul) == capi.LBM_EINVAL
    assert lib.lbm_adjoint_step_moments(None, nul, nul, nul, nul, nul) == capi.LBM_EINVAL
    assert lib.lbm_batch_step_to_moments(None, nul, nul, nul, nul) == capi.LBM_EINVAL
    assert lib.lbm_batch_adjoint_step_moments(None, nul, nul, nul, nul, nul) == capi.LBM_EINVAL
    h = capi.create(8, 8, 8, 0.8, 0)
    try:
        assert lib.lbm_step_to_moments(h, nul, nul, nul, nul) == capi.LBM_EUNBOUND
        assert lib.lbm_adjoint_step_moments(h, nul, nul, nul, nul, nul) == capi.LBM_EUNBOUND
    finally:
        lib.lbm_destroy(h)


def test_kernel_variants_need_matching_storage(lib):
    h32 = capi.create(8, 8, 8, 0.8, capi.LBM_STORE_F32)
    h16 = capi.create(8, 8, 8, 0.8, capi.LBM_STORE_F16)
    try:
        assert lib.lbm_set_kernel(h32, capi.LBM_KERNEL_PAIR) == capi.LBM_EINVAL
        for v in (capi.LBM_KERNEL_PAIR, capi.LBM_KERNEL_X2):
            assert lib.lbm_set_kernel(h16, v) == 0
        assert lib.lbm_set_kernel(h32, capi.LBM_KERNEL_X2) == 0
        assert lib.lbm_set_kernel(h16, 7) == capi.LBM_EINVAL  # unknown variant
        assert lib.lbm_set_kernel(h32, capi.LBM_KERNEL_NODE) == 0
    finally:
        lib.lbm_destroy(h32)
        lib.lbm_destroy(h16)


def test_onsite_handles_reject_kernels_without_the_rule(lib):
    """On-site walls run on the two-node and one-node kernels only; the
    choice is checked on the host (no CUDA call)."""
    h = capi.create(8, 8, 8, 0.8, capi.LBM_WALLS_ONSITE | capi.LBM_CAVITY)
    try:
        for k in (capi.LBM_KERNEL_BULK, capi.LBM_KERNEL_BULK1):
            assert lib.lbm_set_kernel(h, k) == capi.LBM_EINVAL
        for k in (capi.LBM_KERNEL_NODE, capi.LBM_KERNEL_X2):
            assert lib.lbm_set_kernel(h, k) == capi.LBM_OK
    finally:
        lib.lbm_destroy(h)
    # without a walled axis the flag changes nothing
    h = capi.create(8, 8, 8, 0.8, capi.LBM_WALLS_ONSITE)
    try:
        assert lib.lbm_set_kernel(h, capi.LBM_KERNEL_BULK) == capi.LBM_OK
    finally:
        lib.lbm_destroy(h)


def test_four_node_kernel_needs_sixteen_bit_storage_and_halfway_walls(lib):
    h = capi.create(16, 8, 8, 0.8, capi.LBM_STORE_F32)
    try:
        assert lib.lbm_set_kernel(h, capi.LBM_KERNEL_X4) == capi.LBM_EINVAL
    finally:
        lib.lbm_destroy(h)
    h = capi.create(16, 8, 8, 0.8, capi.LBM_STORE_F16 | capi.LBM_CAVITY)
    try:
        assert lib.lbm_set_kernel(h, capi.LBM_KERNEL_X4) == capi.LBM_OK
    finally:
        lib.lbm_destroy(h)
    h = capi.create(16, 8, 8, 0.8, capi.LBM_STORE_F16 | capi.LBM_CAVITY | capi.LBM_WALLS_ONSITE)
    try:
        assert lib.lbm_set_kernel(h, capi.LBM_KERNEL_X4) == capi.LBM_EINVAL
    finally:
        lib.lbm_destroy(h)


def test_tensor_copy_kernel_needs_sixteen_bit_storage_and_halfway_walls(lib):
    h = capi.create(16, 8, 8, 0.8, capi.LBM_STORE_F32)
    try:
        assert lib.lbm_set_kernel(h, capi.LBM_KERNEL_TMA) == capi.LBM_EINVAL
    finally:
        lib.lbm_destroy(h)
    for st in (capi.LBM_STORE_F16, capi.LBM_STORE_BF16):
        h = capi.create(16, 8, 8, 0.8, st | capi.LBM_CAVITY)
        try:
            assert lib.lbm_set_kernel(h, capi.LBM_KERNEL_TMA) == capi.LBM_OK
        finally:
            lib.lbm_destroy(h)
    h = capi.create(16, 8, 8, 0.8, capi.LBM_STORE_F16 | capi.LBM_CAVITY | capi.LBM_WALLS_ONSITE)
    try:
        assert lib.lbm_set_kernel(h, capi.LBM_KERNEL_TMA) == capi.LBM_EINVAL
    finally:
        lib.lbm_destroy(h)


def test_check_calls_are_not_in_the_normal_build(lib):
    # the checked debug build is liblbm_check.so; the normal one says so
    assert lib.lbm_check_reset() == capi.LBM_ENOTSUP
    assert lib.lbm_check_narrow(0) == capi.LBM_ENOTSUP
    with pytest.raises(capi.LBMError) as e:
        capi.check_status()
    assert e.value.code == capi.LBM_ENOTSUP


def test_check_build_compiles_and_exports_every_symbol():
    path = B.build(check=True)
    assert path.endswith("liblbm_check.so")
    chk = ctypes.CDLL(path)
    missing = [n for n in capi.header_symbols() if not hasattr(chk, n)]
    assert not missing, missing


def test_misaligned_device_buffers_are_rejected_before_anything_else(lib):
    # a misaligned pointer is refused before the handle's state is looked at
    # (so an unbound handle, or a NULL batch handle, still reports it) and
    # before any CUDA call: f buffers need 256 bytes, fields and lambda 4,
    # a device FP64 result 8
    v = ctypes.c_void_p
    bad_f, bad_field, ok = v(0x10000 + 16), v(0x10000 + 2), v(0x10000)

    def refused(rc):
        return rc == capi.LBM_EINVAL and "misaligned" in capi.last_error()

    h = capi.create(8, 8, 8, 0.8, capi.LBM_CAVITY)
    try:
        assert refused(lib.lbm_init_equilibrium(h, bad_field, None))
        assert refused(lib.lbm_step_moments(h, 1, ok, bad_field))
        assert refused(lib.lbm_step_to(h, bad_f, ok))
        assert refused(lib.lbm_step_to_moments(h, ok, ok, bad_field, ok))
        assert refused(lib.lbm_step_push(h, ok, bad_f))
        assert refused(lib.lbm_stream(h, bad_f, ok, 0))
        assert refused(lib.lbm_moments(h, bad_field, None, None))
        assert refused(lib.lbm_adjoint_seed(h, ok, ok, ok, None, v(0x10000 + 4)))
        assert refused(lib.lbm_adjoint_step(h, ok, bad_field, ok, None))
        assert refused(lib.lbm_adjoint_step_moments(h, ok, ok, ok, ok, bad_field))
        assert refused(lib.lbm_adjoint_u0(h, ok, bad_field, ok))
        # aligned (or NULL) buffers get past the check to the handle's state
        assert lib.lbm_step_to(h, ok, v(0x20000)) == capi.LBM_EUNBOUND
        assert lib.lbm_moments(h, None, None, None) == capi.LBM_EUNBOUND
    finally:
        lib.lbm_destroy(h)
    nb = None
    assert refused(lib.lbm_batch_init_equilibrium(nb, bad_field))
    assert refused(lib.lbm_batch_step_to(nb, ok, bad_f))
    assert refused(lib.lbm_batch_step_to_moments(nb, ok, ok, ok, bad_field))
    assert refused(lib.lbm_batch_adjoint_seed(nb, bad_f, ok, ok, None, None))
    assert refused(lib.lbm_batch_adjoint_step(nb, ok, ok, bad_field, None))
    assert refused(lib.lbm_batch_adjoint_step_moments(nb, bad_field, ok, ok, ok, None))
    assert refused(lib.lbm_batch_adjoint_u0(nb, ok, ok, bad_field))
    assert refused(lib.lbm_batch_moments(nb, None, bad_field))
    assert lib.lbm_batch_moments(nb, None, None) == capi.LBM_EINVAL  # the NULL handle
    assert refused(lib.lbm_moments_noalloc(bad_f, 8, 8, 8, 0, None, None, None, None, None))
    assert refused(lib.lbm_moments_noalloc(ok, 8, 8, 8, 0, None, None, None,
                                           v(0x10000 + 4), None))

