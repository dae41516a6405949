"""Pins for the oracle's lateral-FFT restatement of A and A^T.

The forward and adjoint operators are 2-D correlations over the scan grid
(Methods, Efficient reconstruction based on scanning symmetries), so with the
grids zero-padded to P >= max(py, px) + R the correlation theorem restates
them exactly.  What pins the restatement:

* the project-written radix-2 FFT equals a brute-force DFT on small sizes and
  numpy's FFT (a test reference only) on larger ones, and inverts exactly;
* the restated A and A^T equal the direct correlations to <= 1e-12 rel-L2
  on the 32x32x48 workload and on a 64x64x64 case, and on a random slab with
  no symmetry at all (so a missing conjugate, a flipped index or a wrong pad
  cannot hide behind the slab's mirror symmetry);
* the cached-spectrum form (``oracle.Spectral``, the slab's half spectrum
  computed once, used for the full-size reference reconstructions) equals
  the direct correlations to <= 1e-12 on both cases and on a random slab
  with no symmetry, and its per-depth bands hold every nonzero slab sample;
* the DFT of a slab slice is real and symmetric under (v, u) -> (u, v) when
  dx = dy, the properties the GPU form relies on (mirror symmetry of the
  patch set, Results, axial symmetry).
"""
import numpy as np
import pytest

import oracle
from paper_2009_10173_gb300 import configs, inputs


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_fft_matches_brute_force_dft(n):
    rng = np.random.Generator(np.random.PCG64(n))
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    W = np.exp(-2j * np.pi * np.outer(j, j) / n)
    assert np.allclose(oracle.fft(x), W @ x, rtol=0, atol=1e-13 * max(1.0, np.abs(x).sum()))
    assert np.allclose(oracle.fft(x, inverse=True), W.conj() @ x, rtol=0, atol=1e-13 * max(1.0, np.abs(x).sum()))


@pytest.mark.parametrize("n", [64, 256, 1024])
def test_fft_matches_reference_and_inverts(n):
    rng = np.random.Generator(np.random.PCG64(100 + n))
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = oracle.fft(x)
    assert rel(X, np.fft.fft(x)) < 1e-14
    assert rel(oracle.fft(X, inverse=True) / n, x) < 1e-14


def test_fft_rejects_non_power_of_two():
    with pytest.raises(oracle.OracleError):
        oracle.fft(np.zeros(12))


def test_fft_size_rule():
    assert oracle.fft_size(32, 32, 11) == 64     # 32 + 5
    assert oracle.fft_size(200, 200, 61) == 256  # 200 + 30
    assert oracle.fft_size(59, 20, 11) == 64     # 59 + 5 = 64 exactly
    assert oracle.fft_size(60, 20, 11) == 128


def _cases():
    tiny = configs.TINY_32
    mid = configs.scaled(configs.TINY_32, px=64, py=64, nz=64, nt=192, win=11, n_patches=400)
    return {"tiny_32x32x48": tiny, "mid_64x64x64": mid}


@pytest.mark.parametrize("name", ["tiny_32x32x48", "mid_64x64x64"])
def test_fft_form_equals_direct_form(name):
    cfg = _cases()[name]
    S = oracle.slab(cfg)
    H = inputs.gaussian((cfg["py"], cfg["px"], cfg["nz"]), 31)
    s = inputs.gaussian((cfg["py"], cfg["px"], cfg["nt"]), 32)
    assert rel(oracle.forward_fft(S, H), oracle.forward(S, H)) <= 1e-12
    assert rel(oracle.adjoint_fft(S, s), oracle.adjoint(S, s)) <= 1e-12


@pytest.mark.parametrize("pad", [None, 64])
def test_fft_form_on_a_slab_without_symmetry(pad):
    rng = np.random.Generator(np.random.PCG64(7))
    win, nz, nt, py, px = 5, 4, 16, 9, 13
    S = rng.standard_normal((win, win, nz, nt))
    S[:, :, :, :3] = 0.0  # a band that starts late, as real slab columns do
    H = rng.standard_normal((py, px, nz))
    s = rng.standard_normal((py, px, nt))
    assert rel(oracle.forward_fft(S, H, pad), oracle.forward(S, H)) <= 1e-12
    assert rel(oracle.adjoint_fft(S, s, pad), oracle.adjoint(S, s)) <= 1e-12


def test_fft_form_rejects_a_pad_that_wraps():
    S = np.zeros((5, 5, 2, 8))
    with pytest.raises(oracle.OracleError):
        oracle.forward_fft(S, np.zeros((15, 15, 2)), 16)  # 15 + 2 > 16


def test_slab_dft_is_real_and_d4_symmetric():
    cfg = configs.TINY_32
    S = oracle.slab(cfg)
    k, n = 15, int(np.argmax(np.abs(S[5, 5, 15])))  # focal depth, peak sample
    Sh = oracle.slab_dft(S, k, n, 64)
    scale = np.abs(Sh.real).max()
    assert scale > 0
    assert np.abs(Sh.imag).max() <= 1e-13 * scale
    assert np.abs(Sh.real - Sh.real.T).max() <= 1e-13 * scale           # (v, u) <-> (u, v), dx = dy
    assert np.abs(Sh.real - np.roll(Sh.real[::-1], 1, axis=0)).max() <= 1e-13 * scale  # v -> -v


@pytest.mark.parametrize("name", ["tiny_32x32x48", "mid_64x64x64"])
def test_cached_spectrum_form_equals_direct_form(name):
    cfg = _cases()[name]
    S = oracle.slab(cfg)
    sp = oracle.Spectral(cfg)
    H = inputs.gaussian((cfg["py"], cfg["px"], cfg["nz"]), 41)
    s = inputs.gaussian((cfg["py"], cfg["px"], cfg["nt"]), 42)
    assert rel(sp.forward(H), oracle.forward(S, H)) <= 1e-12
    assert rel(sp.adjoint(s), oracle.adjoint(S, s)) <= 1e-12
    # every nonzero sample of depth k lies in depth k's band
    nz_samples = (S != 0).any(axis=(0, 1))
    for k in range(cfg["nz"]):
        idx = np.flatnonzero(nz_samples[k])
        assert idx.size == 0 or (sp.klo[k] <= idx[0] and idx[-1] < sp.klo[k] + sp.klen[k])


@pytest.mark.parametrize("shape", [(5, 4, 16, 9, 13), (3, 3, 12, 6, 5)])
def test_cached_spectrum_form_on_a_slab_without_symmetry(shape):
    """A random slab has a complex, non-Hermitian-in-(v) spectrum: a missing
    conjugate, a wrong Hermitian completion or a dropped column fails here."""
    win, nz, nt, py, px = shape
    rng = np.random.Generator(np.random.PCG64(sum(shape)))
    S = rng.standard_normal((win, win, nz, nt))
    S[:, :, :, :3] = 0.0
    S[:, :, 1, 9:] = 0.0  # uneven bands
    H = rng.standard_normal((py, px, nz))
    s = rng.standard_normal((py, px, nt))
    for pad in (None, 32):
        sp = oracle.Spectral.from_dense(S, py, px, pad)
        assert rel(sp.forward(H), oracle.forward(S, H)) <= 1e-12
        assert rel(sp.adjoint(s), oracle.adjoint(S, s)) <= 1e-12


@pytest.mark.parametrize("over", [{}, dict(dy_m=15e-6, px=40, py=24)])
def test_cached_spectrum_symmetric_build_matches_plain_build(over):
    """Evaluating one tap per symmetry orbit and copying it gives the same
    spectrum as evaluating every tap (mirror orbits only when dx != dy)."""
    cfg = configs.scaled(configs.TINY_32, **over)
    a = oracle.Spectral(cfg)
    b = oracle.Spectral(cfg, symmetric=True)
    assert np.array_equal(a.klo, b.klo) and np.array_equal(a.klen, b.klen)
    scale = np.abs(a.re).max()
    assert np.abs(a.re - b.re).max() <= 1e-14 * scale
    assert np.abs(a.im - b.im).max() <= 1e-14 * scale
