"""Byte model of the D3Q19 step (Sec. 4.1) and roofline bookkeeping.

A lattice update reads 19 distribution values and writes 19 (the stores go
to the second copy of f): 152 bytes in FP32, 76 bytes with 16-bit storage.
Writing rho and u adds four FP32 stores (16 bytes); reading a per-cell
force adds three FP32 loads (12 bytes). These are ALGORITHMIC bytes: what
the update must move if every value crosses DRAM exactly once.
"""

from __future__ import annotations

Q = 19


def bytes_per_update(elem_bytes: int = 4, moments: bool = False, force: bool = False) -> int:
    b = 2 * Q * elem_bytes
    if moments:
        b += 4 * 4
    if force:
        b += 3 * 4
    return b


def adjoint_bytes_per_update(force_grad: bool = True, moments: bool = False,
                             force: bool = False) -> int:
    """One reverse step of the adjoint kernel: read lambda^{n+1} (19 FP32),
    write lambda^n (19), and either pull f^n (19 FP32 loads) or read the
    forward collision's rho, u (4 FP32, ``moments``); plus read and write
    the three force-gradient components and read the force itself."""
    b = 2 * Q * 4 + (4 * 4 if moments else Q * 4)
    if force_grad:
        b += 2 * 3 * 4
    if force:
        b += 3 * 4
    return b


def mlups_limit(bandwidth_gbs: float, bytes_per_lu: float, gib: bool = False) -> float:
    """Throughput bound in MLUPS at a given bandwidth. ``gib`` reads GB as
    2^30 bytes (the reading under which Sec. 4.1's printed limits follow from
    Sec. 2.2's measured bandwidths)."""
    unit = 2 ** 30 if gib else 1e9
    return bandwidth_gbs * unit / bytes_per_lu / 1e6


def achieved_gbs(mlups: float, bytes_per_lu: float) -> float:
    return mlups * 1e6 * bytes_per_lu / 1e9


def reynolds(u: float, tau: float, L: float) -> float:
    """Eq. 8 solved for Re: u = (tau - 1/2) Re / (3 L)."""
    return 3.0 * L * u / (tau - 0.5)


def step_time_spectrum(step_ms):
    """Periodic variation of per-iteration times (the Fourier analysis of
    Sec. 6 / Table 5). The series is taken at the iterations' own (uneven)
    completion times, resampled to a uniform grid of the mean step length,
    detrended, and its amplitude spectrum computed with an FFT. Returns
    (peak frequency in Hz, peak amplitude in ms, frequency resolution in Hz);
    (None, None, None) for fewer than 16 iterations."""
    import numpy as np

    t = np.asarray(step_ms, dtype=np.float64)
    if t.size < 16:
        return None, None, None
    when = np.cumsum(t) / 1e3  # completion times in s
    dt = float(t.mean()) / 1e3
    grid = when[0] + dt * np.arange(t.size)
    x = np.interp(grid, when, t)
    x = x - np.polyval(np.polyfit(grid, x, 1), grid)
    amp = np.abs(np.fft.rfft(x)) * 2.0 / x.size
    freq = np.fft.rfftfreq(x.size, d=dt)
    k = int(np.argmax(amp[1:]) + 1)
    return float(freq[k]), float(amp[k]), float(freq[1])
