"""FP64 band-pass filtering of signals and model along time.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

The paper band-pass filters both the raw signals and the model matrix before
inversion (Results: 0.5-80 MHz for the second simulation, 1-120 MHz for the
in vivo scan) and names the band only.  Readings used here:

* the filter is a zero-phase FIR with 2L + 1 taps h[-L..L], h[-m] = h[m],
  designed by the windowed-sinc method: the ideal band-pass impulse response
  2 f_hi/fs sinc(2 f_hi m/fs) - 2 f_lo/fs sinc(2 f_lo m/fs) times the Blackman
  window 0.42 + 0.5 cos(pi m/(L+1)) + 0.08 cos(2 pi m/(L+1)) (the form whose
  end taps stay nonzero);
* it runs along the time axis of every A-line, samples outside [0, nt) count
  as zero, and the output keeps [0, nt) (centred, "same" length);
* filtering the model means filtering every slab column S[b][a][k][:] the same
  way, so the filtered forward operator is F A and its adjoint A^T F (F is
  symmetric).

Functions take and return numpy arrays; ``taps`` is always the half
h[0..L].
"""
import numpy as np


def bandpass_taps(f_lo, f_hi, fs, half_len):
    """Half taps h[0..L] of the Blackman-windowed sinc band-pass [f_lo, f_hi]."""
    if not (0.0 <= f_lo < f_hi <= fs / 2.0) or half_len < 0:
        raise ValueError("need 0 <= f_lo < f_hi <= fs/2 and half_len >= 0")
    L = int(half_len)
    m = np.arange(L + 1, dtype=np.float64)
    window = 0.42 + 0.5 * np.cos(np.pi * m / (L + 1)) + 0.08 * np.cos(2.0 * np.pi * m / (L + 1))
    ideal = 2.0 * f_hi / fs * np.sinc(2.0 * f_hi * m / fs) - 2.0 * f_lo / fs * np.sinc(2.0 * f_lo * m / fs)
    return window * ideal


def response(taps, f, fs):
    """Frequency response of the symmetric FIR at frequency f (real):
    h[0] + 2 sum_{m >= 1} h[m] cos(2 pi f m / fs)."""
    h = np.asarray(taps, np.float64)
    m = np.arange(1, h.size, dtype=np.float64)
    f = np.atleast_1d(np.asarray(f, np.float64))
    return h[0] + 2.0 * (np.cos(2.0 * np.pi * np.outer(f, m) / fs) @ h[1:])


def fir_time(x, taps):
    """y[..., n] = sum_{m=-L}^{L} h[|m|] x[..., n - m], x = 0 outside [0, nt)."""
    x = np.asarray(x, np.float64)
    h = np.asarray(taps, np.float64)
    nt = x.shape[-1]
    y = h[0] * x
    for m in range(1, min(h.size, nt)):  # taps with |m| >= nt never reach [0, nt)
        y[..., m:] += h[m] * x[..., :nt - m]   # x[n - m]
        y[..., :nt - m] += h[m] * x[..., m:]   # x[n + m]
    return y


def filter_slab(S, taps):
    """The filtered model: every slab column S[b][a][k][:] through fir_time."""
    return fir_time(S, taps)
