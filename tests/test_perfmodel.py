"""The benchmark's byte accounting reproduces the byte model and the
throughput limits printed in Sec. 4.1 (tests/golden/byte_model.txt)."""

import os

from paper_1309_1983_gb300 import perfmodel as PM


def _golden(golden_dir):
    kv, rows = {}, []
    with open(os.path.join(golden_dir, "byte_model.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if len(parts) == 2:
                kv[parts[0]] = int(parts[1])
            else:
                rows.append((parts[0], float(parts[1]), int(parts[2]), int(parts[3])))
    return kv, rows


def test_bytes_per_update(golden_dir):
    kv, _ = _golden(golden_dir)
    assert PM.bytes_per_update(4) == kv["bytes_per_lu_fp32"]
    assert PM.bytes_per_update(4, moments=True) == kv["bytes_per_lu_fp32_moments"]
    assert PM.bytes_per_update(2) == kv["bytes_per_lu_fp32"] // 2


def test_printed_limits(golden_dir):
    kv, rows = _golden(golden_dir)
    for gpu, bw, lim, lim_m in rows:
        assert int(PM.mlups_limit(bw, kv["bytes_per_lu_fp32"], gib=True)) == lim, gpu
        assert int(PM.mlups_limit(bw, kv["bytes_per_lu_fp32_moments"], gib=True)) == lim_m, gpu


def test_reynolds_eq8():
    # Eq. 8 inverted: the 32^3 cavity at tau = 0.6 with lid 0.05 is Re = 48
    assert abs(PM.reynolds(0.05, 0.6, 32) - 48.0) < 1e-12


def test_step_time_spectrum_finds_a_planted_period():
    import numpy as np
    rng = np.random.default_rng(0)
    n, base = 2000, 1.25  # ms per step, like the 384^3 step
    t_s = np.arange(n) * base / 1e3
    step = base + 0.02 * np.sin(2 * np.pi * 11.7 * t_s) + 0.002 * rng.standard_normal(n)
    f, a, res = PM.step_time_spectrum(step)
    assert abs(f - 11.7) <= res and 0.015 < a < 0.025
    assert PM.step_time_spectrum([1.0] * 5) == (None, None, None)


def test_adjoint_byte_model():
    # gathered state: 3 x 76 B of lambda and f plus 24 B of force gradient
    assert PM.adjoint_bytes_per_update() == 252
    assert PM.adjoint_bytes_per_update(force=True) == 264
    assert PM.adjoint_bytes_per_update(force_grad=False) == 228
    # from stored moments: rho, u (16 B) replace the 76 B gather
    assert PM.adjoint_bytes_per_update(moments=True, force=True) == 204
    assert PM.adjoint_bytes_per_update(moments=True) == 192


def test_validation_scalings_follow_eq8():
    from paper_1309_1983_gb300 import validation as V
    for N, Re in ((24, 100.0), (128, 400.0), (256, 1000.0)):
        tau = V.tau_for(N, 0.05, Re)
        assert abs(PM.reynolds(0.05, tau, N) - Re) < 1e-9 * Re
        U = V.lid_for(N, 0.53, Re)
        assert abs(PM.reynolds(U, 0.53, N) - Re) < 1e-9 * Re
    # diffusive scaling: doubling N halves the lid speed at fixed tau
    assert abs(V.lid_for(64, 0.6, 100) - 2 * V.lid_for(128, 0.6, 100)) < 1e-15
