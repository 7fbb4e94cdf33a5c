"""Host side of the continuous-time projective protocol in libfm.so against the
oracle (CPU only: the event draws and the propagation stencils are host code).

The taps are pinned to the plane-wave row of exp(-i H~ tau) (App. A's
propagator), which the oracle pins to expm of the hopping matrix; the draws to
the oracle's Philox stream, bit for bit.
"""
import ctypes

import numpy as np
import pytest
from scipy import special

from oracle import lattice, philox


@pytest.fixture(scope="module")
def lib():
    from paper_2508_18468_gb300 import build
    build.build()
    from paper_2508_18468_gb300 import fm as mod
    L = mod.lib
    L.fmx_poisson_draw.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_longlong, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double)]
    L.fmx_poisson_taps.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_double)]
    L.fmx_poisson_width.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    return L


def draw(lib, seed, traj, e, L):
    out = (ctypes.c_double * 3)()
    assert lib.fmx_poisson_draw(seed, traj, e, L, out) == 0
    return out[0], int(out[1]), out[2]


def taps(lib, n, w, J, tau):
    k = n if w < 0 else 2 * w + 1
    out = np.zeros(2 * k)
    assert lib.fmx_poisson_taps(n, w, J, tau, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 0
    return out[0::2] + 1j * out[1::2]


@pytest.mark.parametrize("seed,traj", [(1, 0), (2**40 + 17, 5), (99, 2**33 + 7)])
def test_event_draws_bit_identical(lib, seed, traj):
    for e in list(range(40)) + [2**32 - 1, 2**32, 2**35 + 3]:
        got = draw(lib, seed, traj, e, 1000)
        assert got == philox.poisson_event(seed, traj, e, 1000), e


@pytest.mark.parametrize("J,tau", [(1.0, 0.0), (1.0, 0.0137), (1.0, 0.05), (-0.7, 0.05), (2.0, 0.3)])
def test_bessel_taps_equal_the_plane_wave_row(lib, J, tau):
    n = 96
    w = lib.fmx_poisson_width(n, abs(J), 0.3 if tau > 0.05 else 0.05)
    assert w > 0
    t = taps(lib, n, w, J, tau)
    row = lattice.ring_propagator_row(n, J, tau)
    offs = np.arange(-w, w + 1)
    assert np.max(np.abs(t - row[offs % n])) < 1e-15
    # every entry the stencil drops is zero up to the row's own rounding noise
    # (a sum of n unit-modulus terms: about n 2^-53)
    rest = np.delete(row, offs % n)
    assert np.max(np.abs(rest)) < 4 * n * 2.0**-53


def test_full_row_on_short_directions(lib):
    for n in (2, 4, 6):
        t = taps(lib, n, -1, 1.0, 0.04)
        assert np.max(np.abs(t - lattice.ring_propagator_row(n, 1.0, 0.04))) < 1e-15
    # a direction of length 1 has no bond (the hopping matrix has none): identity
    assert taps(lib, 1, -1, 1.0, 0.04)[0] == 1.0


def test_width_is_the_bessel_cut(lib):
    for z_half, n in [(0.05, 64), (0.3, 200), (1.0, 400)]:
        w = lib.fmx_poisson_width(n, 1.0, z_half)
        z = 2.0 * z_half
        assert w >= z
        assert all(abs(special.jv(r, z)) < 1e-17 for r in range(w + 1, w + 30))
        assert abs(special.jv(w, z)) >= 1e-17 or w == 0
    assert lib.fmx_poisson_width(16, 1.0, 0.05) == -1         # stencil reaches the period
    assert lib.fmx_poisson_width(0, 1.0, 0.05) == -2
