"""Pins for the oracle's band-pass filter (signals and model along time).

The paper filters both the raw signals and the model matrix to a band
(Results: 0.5-80 MHz, second simulation; 1-120 MHz, in vivo).  What pins the
oracle's reading of that step:

* the design reduces to the identity for the all-pass band [0, fs/2], and its
  response matches the ideal band-pass within the Blackman window's ripple
  away from the cut-offs, with -6 dB (0.5) at the cut-offs;
* the filter equals numpy's full convolution cut to the centred nt samples (a
  library routine), for tap counts below, at and above nt;
* it is a symmetric operator, and a pure tone far from the A-line's ends comes
  out scaled by the response at its frequency (an even FIR has no phase);
* filtering every slab column gives the same forward and adjoint as filtering
  the predicted signals after A and the signals before A^T, the order the
  device path uses.
"""
import numpy as np
import pytest

import oracle
from oracle import bandpass as bp
from paper_2009_10173_gb300 import configs, inputs

FS = 250e6


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("L", [0, 5, 64])
def test_all_pass_band_is_the_identity(L):
    h = bp.bandpass_taps(0.0, FS / 2, FS, L)
    assert abs(h[0] - 1.0) <= 1e-15
    assert np.abs(h[1:]).max(initial=0.0) <= 1e-15


@pytest.mark.parametrize("f_lo,f_hi,L", [(0.5e6, 80e6, 511), (1e6, 120e6, 511), (0.5e6, 80e6, 1023),
                                         (5e6, 60e6, 127)])
def test_design_matches_the_ideal_band(f_lo, f_hi, L):
    h = bp.bandpass_taps(f_lo, f_hi, FS, L)
    delta = 6.0 * FS / (2 * L + 1)  # Blackman transition half-width is about 2.75 fs / (2L + 1)
    f = np.linspace(0.0, FS / 2, 4001)
    H = bp.response(h, f, FS)
    passband = (f >= f_lo + delta) & (f <= f_hi - delta)
    stopband = (f >= f_hi + delta) | (f <= f_lo - delta)
    assert passband.any()
    assert np.abs(H[passband] - 1.0).max() <= 1e-3
    if stopband.any():
        assert np.abs(H[stopband]).max() <= 1e-3
    assert np.abs(bp.response(h, [f_lo, f_hi], FS) - 0.5).max() <= 2e-3


def test_design_rejects_a_bad_band():
    for args in [(80e6, 0.5e6, FS, 10), (0.5e6, 130e6, FS, 10), (-1.0, 80e6, FS, 10), (0.5e6, 80e6, FS, -1)]:
        with pytest.raises(ValueError):
            bp.bandpass_taps(*args)


@pytest.mark.parametrize("L", [0, 1, 7, 40, 63, 64, 70])
def test_fir_matches_numpy_convolution(L):
    nt = 64
    rng = np.random.Generator(np.random.PCG64(L))
    x = rng.standard_normal((3, nt))
    h = rng.standard_normal(L + 1)
    full = np.concatenate([h[:0:-1], h])  # h[-L..L]
    y = bp.fir_time(x, h)
    for i in range(3):
        ref = np.convolve(x[i], full, mode="full")[L:L + nt]
        assert rel(y[i], ref) <= 1e-13


def test_fir_is_a_symmetric_operator():
    rng = np.random.Generator(np.random.PCG64(5))
    x, z = rng.standard_normal((2, 4, 4, 96))
    h = bp.bandpass_taps(2e6, 70e6, FS, 30)
    lhs = float(np.vdot(bp.fir_time(x, h), z))
    rhs = float(np.vdot(x, bp.fir_time(z, h)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("f", [20e6, 100e6])
def test_tone_is_scaled_by_the_response(f):
    nt, L = 4096, 255
    h = bp.bandpass_taps(0.5e6, 80e6, FS, L)
    n = np.arange(nt)
    x = np.cos(2 * np.pi * f * n / FS + 0.3)
    y = bp.fir_time(x, h)
    gain = float(bp.response(h, f, FS)[0])
    inner = slice(L, nt - L)
    # cos arguments reach ~1e4 rad: ~1e-12 phase rounding per sample, summed over the taps
    assert np.abs(y[inner] - gain * x[inner]).max() <= 1e-11
    if f > 80e6 + 6 * FS / (2 * L + 1):
        assert abs(gain) <= 1e-3
    else:
        assert abs(gain - 1.0) <= 1e-3


def test_filtered_model_equals_filtered_signals():
    cfg = configs.TINY_32
    S = oracle.slab(cfg)
    h = bp.bandpass_taps(0.5e6, 80e6, FS, 40)
    H = inputs.gaussian((cfg["py"], cfg["px"], cfg["nz"]), 41)
    s = inputs.gaussian((cfg["py"], cfg["px"], cfg["nt"]), 42)
    Sf = bp.filter_slab(S, h)
    assert rel(oracle.forward(Sf, H), bp.fir_time(oracle.forward(S, H), h)) <= 1e-12
    assert rel(oracle.adjoint(Sf, s), oracle.adjoint(S, bp.fir_time(s, h))) <= 1e-12
    # the filtered operator and its adjoint stay a transpose pair
    lhs = float(np.vdot(oracle.forward(Sf, H), s))
    rhs = float(np.vdot(H, oracle.adjoint(Sf, s)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
