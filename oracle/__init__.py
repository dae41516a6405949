"""FP64 CPU oracle for model-based AR-OAM inversion (arXiv:2009.10173).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg import this package; the product path
(``paper_2009_10173_gb300``) never does, and the two share no code.

* ``patches``, ``slab``, ``slab_column``, ``slab_time_slice``: the sensor
  discretisation of Eq. 3 and the per-position model slab of Eq. 4
  (Methods, Forward modeling), computed in C (``oam_oracle.c``).
* ``forward`` / ``adjoint``: A and its transpose as lateral correlations of
  the slab with the volume (Methods, Efficient reconstruction based on
  scanning symmetries).
* ``forward_fft`` / ``adjoint_fft``: the same operators restated exactly
  through the 2-D correlation theorem over the zero-padded scan grid, with a
  project-written radix-2 FFT (``fft``); ``slab_dft`` is the transform of one
  slab slice.  ``Spectral`` keeps the slab's half spectrum per (depth,
  sample) so that large grids (200 x 200 positions, 61 x 61 taps) can be
  applied hundreds of times; ``Spectral.forward`` / ``Spectral.adjoint`` are
  the same two operators.
* ``oracle.solvers``: LSQR for Eq. 5 with Eq. 6 (MB-L2) and FISTA for Eq. 5
  with Eq. 7 (MB-L1), written from the published algorithms the paper names.
* ``tent_radon``, ``slab33_column``: the paper's own discretisation of Eq. 1
  (trilinear interpolation of the voxel values for the surface integral, a
  central finite difference for the time derivative), summed over the patches
  of Eq. 3 and filtered by the sampled EIR.
* ``oracle.bandpass``: the band-pass filtering of signals and model along
  time that precedes inversion in the Results (a windowed-sinc FIR, applied
  as a direct sum).
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in ``oam_oracle.c``; SI units (m, s, Hz)."""

    _fields_ = [(n, ctypes.c_double) for n in (
        "focal_m", "aperture_m", "hole_m", "c_mps", "fc_hz", "frac_bw", "trunc_sigma",
        "dx_m", "dy_m", "dz_m", "z0_rel_m", "fs_hz", "t0_s")] + [
        (n, ctypes.c_int32) for n in ("n_patches", "px", "py", "nz", "nt", "win")]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(Params)
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i32, f64 = ctypes.c_int32, ctypes.c_double
        L.orc_patch_count_rings.argtypes = [P]
        L.orc_patches.argtypes = [P, dp, dp, dp, dp]
        L.orc_eir.argtypes = [P, f64]
        L.orc_eir.restype = f64
        L.orc_eir_dot.argtypes = [P, f64]
        L.orc_eir_dot.restype = f64
        L.orc_distance_range.argtypes = [P, ctypes.POINTER(f64), ctypes.POINTER(f64)]
        L.orc_t0.argtypes = [P, ctypes.POINTER(f64)]
        L.orc_slab_column.argtypes = [P, f64, i32, i32, i32, dp]
        L.orc_slab.argtypes = [P, f64, dp]
        L.orc_slab_time_slice.argtypes = [P, f64, i32, dp]
        L.orc_forward.argtypes = [dp, i32, i32, i32, i32, i32, dp, dp]
        L.orc_adjoint.argtypes = [dp, i32, i32, i32, i32, i32, dp, dp]
        L.orc_forward_at.argtypes = [dp, i32, i32, i32, i32, dp, i32, ip, ip, ip, dp]
        L.orc_fft.argtypes = [dp, dp, i32, i32]
        L.orc_slab_dft.argtypes = [dp, i32, i32, i32, i32, i32, i32, dp, dp]
        L.orc_forward_fft.argtypes = [dp, i32, i32, i32, i32, i32, i32, dp, dp]
        L.orc_adjoint_fft.argtypes = [dp, i32, i32, i32, i32, i32, i32, dp, dp]
        lp = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        L.orc_depth_band.argtypes = [P, f64, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.orc_tent_radon.argtypes = [f64] * 7
        L.orc_tent_radon.restype = f64
        L.orc_slab33_column.argtypes = [P, f64, i32, i32, i32, dp]
        L.orc_spectrum_depth.argtypes = [P, f64, i32, i32, i32, i32, i32, dp, dp]
        L.orc_forward_spec.argtypes = [dp, dp, ip, ip, lp, i32, i32, i32, i32, i32, i32, dp, dp]
        L.orc_adjoint_spec.argtypes = [dp, dp, ip, ip, lp, i32, i32, i32, i32, i32, i32, dp, dp]
        for f in ("orc_patch_count_rings", "orc_patches", "orc_distance_range", "orc_t0",
                  "orc_slab_column", "orc_slab", "orc_slab_time_slice", "orc_forward",
                  "orc_adjoint", "orc_forward_at", "orc_fft", "orc_slab_dft", "orc_forward_fft",
                  "orc_adjoint_fft", "orc_depth_band", "orc_spectrum_depth", "orc_forward_spec",
                  "orc_adjoint_spec", "orc_slab33_column"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc < 0:
        raise OracleError({-1: "invalid argument", -2: "arrival window outside [0, Nt)",
                           -3: "out of memory"}.get(rc, f"error {rc}"))
    return rc


def params(cfg) -> Params:
    """Build the oracle's parameter block from a config mapping (SI units)."""
    p = Params()
    for name, _ in Params._fields_:
        v = cfg.get(name, None)
        if v is None:
            if name == "t0_s":
                v = math.nan
            elif name == "hole_m":
                v = 0.0
            elif name == "trunc_sigma":
                v = 5.0
            else:
                raise KeyError(name)
        setattr(p, name, v)
    return p


def patches(cfg):
    """Sensor patches (Eq. 3): unit normals (nx, ny, nz) and areas w (m^2)."""
    p = params(cfg)
    M = p.n_patches
    nx, ny, nz, w = (np.zeros(M) for _ in range(4))
    _check(lib().orc_patches(ctypes.byref(p), nx, ny, nz, w))
    return nx, ny, nz, w


def ring_count(cfg) -> int:
    p = params(cfg)
    return _check(lib().orc_patch_count_rings(ctypes.byref(p)))


def eir(cfg, tau):
    p = params(cfg)
    return np.array([lib().orc_eir(ctypes.byref(p), float(t)) for t in np.ravel(tau)])


def eir_dot(cfg, tau):
    p = params(cfg)
    return np.array([lib().orc_eir_dot(ctypes.byref(p), float(t)) for t in np.ravel(tau)])


def distance_range(cfg):
    p = params(cfg)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib().orc_distance_range(ctypes.byref(p), ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def t0(cfg) -> float:
    """Time of sample 0 (explicit, or the automatic rule) after the window check."""
    p = params(cfg)
    out = ctypes.c_double()
    _check(lib().orc_t0(ctypes.byref(p), ctypes.byref(out)))
    return out.value


def slab(cfg, t0_s=None):
    """Dense slab S[win][win][nz][nt] (Eq. 4), FP64."""
    p = params(cfg)
    t = t0(cfg) if t0_s is None else t0_s
    S = np.zeros((p.win, p.win, p.nz, p.nt))
    _check(lib().orc_slab(ctypes.byref(p), t, S))
    return S


def slab_column(cfg, b, a, k, t0_s=None):
    """One slab column S[b, a, k, :] with b, a in [-R, R]."""
    p = params(cfg)
    t = t0(cfg) if t0_s is None else t0_s
    out = np.zeros(p.nt)
    _check(lib().orc_slab_column(ctypes.byref(p), t, b, a, k, out))
    return out


def slab_time_slice(cfg, n, t0_s=None):
    """S[:, :, :, n] for every tap and depth."""
    p = params(cfg)
    t = t0(cfg) if t0_s is None else t0_s
    out = np.zeros((p.win, p.win, p.nz))
    _check(lib().orc_slab_time_slice(ctypes.byref(p), t, int(n), out))
    return out


def forward(S, H):
    """A H for a dense slab S[win][win][nz][nt] and volume H[py][px][nz]."""
    S = np.ascontiguousarray(S, np.float64)
    H = np.ascontiguousarray(H, np.float64)
    win, _, nz, nt = S.shape
    py, px, _ = H.shape
    s = np.zeros((py, px, nt))
    _check(lib().orc_forward(S, win, nz, nt, py, px, H, s))
    return s


def adjoint(S, s):
    """A^T s for a dense slab and signals s[py][px][nt]."""
    S = np.ascontiguousarray(S, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    win, _, nz, nt = S.shape
    py, px, _ = s.shape
    H = np.zeros((py, px, nz))
    _check(lib().orc_adjoint(S, win, nz, nt, py, px, s, H))
    return H


def forward_at(slices, H, ys, xs, which):
    """(A H)[y, x, n_i] at chosen points from time slices of the slab."""
    slices = np.ascontiguousarray(slices, np.float64)
    H = np.ascontiguousarray(H, np.float64)
    win, nz = slices.shape[1], slices.shape[3]
    py, px, _ = H.shape
    ys, xs, which = (np.ascontiguousarray(v, np.int32) for v in (ys, xs, which))
    out = np.zeros(len(ys))
    _check(lib().orc_forward_at(slices, win, nz, py, px, H, len(ys), ys, xs, which, out))
    return out


def fft_size(py, px, win):
    """Smallest power of two P with P >= max(py, px) + R: no circular wrap of
    the zero-padded correlation reaches the output window."""
    need = max(py, px) + (win - 1) // 2
    P = 1
    while P < need:
        P *= 2
    return P


def fft(x, inverse=False):
    """Unscaled radix-2 DFT of a complex vector (length a power of two):
    X[f] = sum_j x[j] exp(-+2 pi i j f / n), sign + for ``inverse``."""
    x = np.asarray(x, np.complex128)
    re, im = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    _check(lib().orc_fft(re, im, len(x), 1 if inverse else -1))
    return re + 1j * im


def slab_dft(S, k, n, P):
    """2-D DFT of the slab slice S[:, :, k, n] placed at (b mod P, a mod P)."""
    S = np.ascontiguousarray(S, np.float64)
    win, _, nz, nt = S.shape
    re, im = np.zeros((P, P)), np.zeros((P, P))
    _check(lib().orc_slab_dft(S, win, nz, nt, k, n, P, re, im))
    return re + 1j * im


def forward_fft(S, H, P=None):
    """A H through the lateral correlation theorem (exact restatement)."""
    S = np.ascontiguousarray(S, np.float64)
    H = np.ascontiguousarray(H, np.float64)
    win, _, nz, nt = S.shape
    py, px, _ = H.shape
    P = fft_size(py, px, win) if P is None else P
    s = np.zeros((py, px, nt))
    _check(lib().orc_forward_fft(S, win, nz, nt, py, px, P, H, s))
    return s


def adjoint_fft(S, s, P=None):
    """A^T s through the lateral correlation theorem (exact restatement)."""
    S = np.ascontiguousarray(S, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    win, _, nz, nt = S.shape
    py, px, _ = s.shape
    P = fft_size(py, px, win) if P is None else P
    H = np.zeros((py, px, nz))
    _check(lib().orc_adjoint_fft(S, win, nz, nt, py, px, P, s, H))
    return H


class Spectral:
    """A and A^T of a configuration through the lateral correlation theorem,
    with the slab's spectrum computed once.

    For every depth k the band [klo[k], klo[k] + klen[k]) holds all samples
    any patch's EIR window reaches at that depth (the slab is exactly zero
    elsewhere); for each (k, n) in it the 2-D DFT of the slice S[:, :, k, n]
    placed at (b mod P, a mod P) is stored for columns u = 0 .. P/2 (the
    slab is real, so the other half follows by Hermitian symmetry).  Memory:
    16 * sum(klen) * P * (P/2 + 1) bytes.  Building evaluates every slab
    column once (Eqs. 3-4); each application then costs the 2-D transforms
    of the input and output and the spectral sums.
    """

    def __init__(self, cfg, t0_s=None, P=None, symmetric=False):
        """``symmetric``: evaluate Eq. 3 for one tap per orbit of the patch
        set's mirror (and, for dx == dy, x <-> y) symmetry and copy it to
        the orbit's other taps (same terms, summed in another order)."""
        p = params(cfg)
        self.t0 = t0(cfg) if t0_s is None else float(t0_s)
        self.win, self.nz, self.nt, self.py, self.px = p.win, p.nz, p.nt, p.py, p.px
        self.R = (p.win - 1) // 2
        self.P = fft_size(p.py, p.px, p.win) if P is None else int(P)
        Q = self.P // 2 + 1
        L = lib()
        self.klo = np.zeros(p.nz, np.int32)
        self.klen = np.zeros(p.nz, np.int32)
        lo, ln = ctypes.c_int32(), ctypes.c_int32()
        for k in range(p.nz):
            _check(L.orc_depth_band(ctypes.byref(p), self.t0, k, ctypes.byref(lo), ctypes.byref(ln)))
            self.klo[k], self.klen[k] = lo.value, ln.value
        self.koff = np.zeros(p.nz, np.int64)
        self.koff[1:] = np.cumsum(self.klen.astype(np.int64))[:-1]
        total = int(self.klen.sum())
        self.re = np.zeros((max(total, 1), self.P, Q))
        self.im = np.zeros((max(total, 1), self.P, Q))
        for k in range(p.nz):
            if self.klen[k] == 0:
                continue
            a, b = int(self.koff[k]), int(self.koff[k] + self.klen[k])
            _check(L.orc_spectrum_depth(ctypes.byref(p), self.t0, k, self.P, int(self.klo[k]),
                                        int(self.klen[k]), int(bool(symmetric)), self.re[a:b], self.im[a:b]))

    @classmethod
    def from_dense(cls, S, py, px, P=None):
        """The same operators for a given dense slab S[win][win][nz][nt]
        (any values, no symmetry assumed): depth k's band is the union of its
        nonzero samples over taps, each slice transformed by ``slab_dft``."""
        S = np.ascontiguousarray(S, np.float64)
        self = cls.__new__(cls)
        self.win, _, self.nz, self.nt = S.shape
        self.py, self.px = py, px
        self.R = (self.win - 1) // 2
        self.P = fft_size(py, px, self.win) if P is None else int(P)
        Q = self.P // 2 + 1
        nzmask = (S != 0).any(axis=(0, 1))  # [nz][nt]
        self.klo = np.zeros(self.nz, np.int32)
        self.klen = np.zeros(self.nz, np.int32)
        for k in range(self.nz):
            idx = np.flatnonzero(nzmask[k])
            if len(idx):
                self.klo[k], self.klen[k] = idx[0], idx[-1] - idx[0] + 1
        self.koff = np.zeros(self.nz, np.int64)
        self.koff[1:] = np.cumsum(self.klen.astype(np.int64))[:-1]
        total = int(self.klen.sum())
        self.re = np.zeros((max(total, 1), self.P, Q))
        self.im = np.zeros((max(total, 1), self.P, Q))
        self.t0 = float("nan")
        for k in range(self.nz):
            for i in range(int(self.klen[k])):
                X = slab_dft(S, k, int(self.klo[k]) + i, self.P)
                self.re[self.koff[k] + i] = X.real[:, :Q]
                self.im[self.koff[k] + i] = X.imag[:, :Q]
        return self

    def forward(self, H):
        """A H (Eq. 4 over the scan grid), H[py][px][nz] -> s[py][px][nt]."""
        H = np.ascontiguousarray(H, np.float64)
        assert H.shape == (self.py, self.px, self.nz)
        s = np.zeros((self.py, self.px, self.nt))
        _check(lib().orc_forward_spec(self.re, self.im, self.klo, self.klen, self.koff, self.nz, self.nt,
                                      self.P, self.R, self.py, self.px, H, s))
        return s

    def adjoint(self, s):
        """A^T s, s[py][px][nt] -> H[py][px][nz]."""
        s = np.ascontiguousarray(s, np.float64)
        assert s.shape == (self.py, self.px, self.nt)
        H = np.zeros((self.py, self.px, self.nz))
        _check(lib().orc_adjoint_spec(self.re, self.im, self.klo, self.klen, self.koff, self.nz, self.nt,
                                      self.P, self.R, self.py, self.px, s, H))
        return H


def tent_radon(d, e, s):
    """Planar Radon transform of the trilinear tent with half-widths d = (dx,
    dy, dz) along unit normal e at signed offsets s (any array)."""
    L = lib()
    return np.array([L.orc_tent_radon(d[0], d[1], d[2], e[0], e[1], e[2], float(x)) for x in np.ravel(s)])


def slab33_column(cfg, b, a, k, t0_s=None):
    """One column S33[b, a, k, :] of the discretised model (trilinear voxels,
    finite-difference derivative, EIR at whole samples)."""
    p = params(cfg)
    t = t0(cfg) if t0_s is None else t0_s
    out = np.zeros(p.nt)
    _check(lib().orc_slab33_column(ctypes.byref(p), t, b, a, k, out))
    return out
