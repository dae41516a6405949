"""Band-pass filtered operators and the Tikhonov sweep on the GPU vs the oracle.

Results: the raw signals and the model are band-pass filtered before
inversion (0.5-80 MHz, second simulation).  The oracle filters every slab
column with a direct FP64 sum and runs the plain correlations with that
filtered slab; the device applies F after its forward operator and before its
adjoint (one shared-memory FFT convolution per pair of A-lines).  Tolerances
as the operator parity tests: rel-L2 <= 1e-5 for the FP32 forms, <= 1e-4 for
split-BF16, <= 1e-3 for images.

The sweep solves MB-L2 (Eq. 5 with Eq. 6) for several Tikhonov weights from
one bidiagonalisation; each of its results must equal the single solve with
that damp bit for bit (same kernels, same reduction order) and the oracle's
LSQR to the image tolerance.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
from oracle import bandpass as bp
from oracle import solvers
from paper_2009_10173_gb300 import binding as B
from paper_2009_10173_gb300 import configs, inputs
from paper_2009_10173_gb300.model import Model

pytestmark = pytest.mark.gpu

FS = 250e6
C0 = configs.TINY_32
C1 = configs.VOLUME_200
# 33x31 scan (1023 A-lines: an odd count, so the last line pair is half empty)
ODD = configs.scaled(C0, px=33, py=31)
PRECS = [B.OAM_PREC_FP32, B.OAM_PREC_BF16X3, B.OAM_PREC_FFT]
TOL = {B.OAM_PREC_FP32: 1e-5, B.OAM_PREC_BF16X3: 1e-4, B.OAM_PREC_FFT: 1e-5}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@functools.lru_cache(maxsize=None)
def slab(name):
    return oracle.slab({"c0": C0, "odd": ODD}[name])


_models = {}


def model(name, prec):
    key = (name, prec)
    if key not in _models:
        cfg = {"c0": C0, "odd": ODD, "c1": C1}[name]
        _models[key] = Model(cfg, precision=prec)
    m = _models[key]
    m.set_filter(None)
    return m


# ------------------------------------------------------------------ the filter alone
@pytest.mark.parametrize("L", [0, 5, 40, 191, 300])
@pytest.mark.parametrize("name", ["c0", "odd"])
def test_filter_signals_matches_oracle(name, L):
    """F s on every A-line; L = 191 = nt - 1 is the longest tap set that reaches
    the output, L = 300 has taps beyond it."""
    m = model(name, B.OAM_PREC_FP32)
    taps = bp.bandpass_taps(0.5e6, 80e6, FS, L) if L > 0 else np.array([0.75])
    m.set_filter(list(taps))
    assert m.info.filter_half_len == L
    nt = m.cfg["nt"]
    assert m.info.filter_size >= nt + min(L, nt - 1)
    s = inputs.gaussian(m.sig_shape, 50 + L)
    got = host(m.filter_signals(dev(s)))
    want = bp.fir_time(s.astype(np.float32), taps)
    assert rel(got, want) <= 1e-5
    # in place
    t = dev(s)
    m.filter_signals(t, out=t)
    assert rel(host(t), want) <= 1e-5


def test_filter_errors():
    m = model("c0", B.OAM_PREC_FP32)
    s = dev(inputs.gaussian(m.sig_shape, 1))
    with pytest.raises(B.OamError) as e:
        m.filter_signals(s)  # no filter set
    assert e.value.code == B.OAM_ERR_INVALID_ARG
    for bad in ([float("nan"), 0.1], [0.0] * (B.OAM_MAX_FIR_HALF + 2)):
        with pytest.raises(B.OamError) as e:
            m.set_filter(bad)
        assert e.value.code == B.OAM_ERR_INVALID_ARG
    assert m.info.filter_half_len == -1
    m.set_filter([1.0])
    before = m.info.device_bytes
    m.set_filter(None)
    assert m.info.filter_half_len == -1 and m.info.device_bytes < before


# ------------------------------------------------------------------ filtered operators
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["c0", "odd"])
def test_filtered_operators_match_oracle(name, prec):
    """Device F A and A^T F against the oracle's forward and adjoint with the
    filtered slab (the order the paper states: filter the model)."""
    cfg = {"c0": C0, "odd": ODD}[name]
    taps = bp.bandpass_taps(0.5e6, 80e6, FS, 40)
    Sf = bp.filter_slab(slab(name), taps)
    m = model(name, prec)
    m.set_filter(list(taps))
    H = inputs.gaussian((cfg["py"], cfg["px"], cfg["nz"]), 61).astype(np.float32)
    s = inputs.gaussian((cfg["py"], cfg["px"], cfg["nt"]), 62).astype(np.float32)
    assert rel(host(m.forward(dev(H))), oracle.forward(Sf, H)) <= TOL[prec]
    assert rel(host(m.adjoint(dev(s))), oracle.adjoint(Sf, s)) <= TOL[prec]


@pytest.mark.parametrize("prec", [B.OAM_PREC_FP32, B.OAM_PREC_FFT])
def test_filtered_lsqr_matches_oracle(prec):
    """MB-L2 on filtered signals with the filtered model, 10 iterations."""
    taps = bp.bandpass_taps(0.5e6, 80e6, FS, 40)
    Sf = bp.filter_slab(slab("c0"), taps)
    m = model("c0", prec)
    m.set_filter(list(taps))
    H = inputs.phantom(C0, 3, kind="spheres", count=6)
    raw = oracle.forward(slab("c0"), H) + 0.02 * inputs.gaussian(m.sig_shape, 63)
    s_ref = bp.fir_time(raw.astype(np.float32), taps)
    s = m.filter_signals(dev(raw))
    assert rel(host(s), s_ref) <= 1e-5
    x, info = m.lsqr(s, 10)
    x_ref, info_ref = solvers.lsqr(lambda v: oracle.forward(Sf, v), lambda u: oracle.adjoint(Sf, u), s_ref, 10)
    assert rel(host(x), x_ref) <= 1e-3
    assert abs(info.rnorm - info_ref["rnorm"]) <= 1e-3 * info_ref["rnorm"]


def test_filtered_model_in_a_batch_matches_standalone():
    m = model("c0", B.OAM_PREC_FFT)
    m.set_filter(list(bp.bandpass_taps(0.5e6, 80e6, FS, 40)))
    s = m.filter_signals(dev(inputs.gaussian(m.sig_shape, 64)))
    x_ref, _ = m.lsqr(s, 8)
    x_ref = host(x_ref)
    work = m.workspace(0)
    batch = B.oam_batch_create(1)
    try:
        x = m.empty_volume()
        B.oam_batch_set_job(batch, 0, m.handle, s, x, None, B.OamLsqrOpts(8, 0.0),
                            B.OamFistaOpts(0, 0, 1, 0, -1.0, 1e-3, 0.0, None), work)
        B.oam_batch_run(batch)
        assert np.array_equal(host(x), x_ref)
    finally:
        B.oam_batch_free(batch)


def test_batch_records_again_after_the_filter_changes():
    """A recorded graph holds the filter's buffers: setting another filter (or
    removing it) makes the next run record the graph again."""
    m = model("c0", B.OAM_PREC_FP32)
    s = dev(inputs.gaussian(m.sig_shape, 71))
    work = m.workspace(0)
    batch = B.oam_batch_create(1)
    try:
        x = m.empty_volume()
        B.oam_batch_set_job(batch, 0, m.handle, s, x, None, B.OamLsqrOpts(4, 0.0),
                            B.OamFistaOpts(0, 0, 1, 0, -1.0, 1e-3, 0.0, None), work)
        for taps in (list(bp.bandpass_taps(0.5e6, 80e6, FS, 40)), list(bp.bandpass_taps(2e6, 60e6, FS, 12)), None):
            m.set_filter(taps)
            ref = host(m.lsqr(s, 4)[0])
            B.oam_batch_run(batch)
            assert np.array_equal(host(x), ref)
    finally:
        B.oam_batch_free(batch)


# ------------------------------------------------------------------ Tikhonov sweep
DAMPS = [0.0, 0.3, 3.0, 30.0]


@pytest.mark.parametrize("prec", [B.OAM_PREC_FP32, B.OAM_PREC_FFT])
def test_sweep_equals_single_solves_and_oracle(prec):
    m = model("c0", prec)
    H = inputs.phantom(C0, 4, kind="spheres", count=6)
    s32 = (oracle.forward(slab("c0"), H) + 0.02 * inputs.gaussian(m.sig_shape, 65)).astype(np.float32)
    s = dev(s32)
    xs, infos = m.lsqr_sweep(s, 10, DAMPS)
    S = slab("c0")
    for d, x, inf in zip(DAMPS, xs, infos):
        x1, inf1 = m.lsqr(s, 10, damp=d)
        assert torch.equal(x, x1), d
        assert (inf.rnorm, inf.arnorm, inf.anorm, inf.iters_done) == (inf1.rnorm, inf1.arnorm, inf1.anorm,
                                                                      inf1.iters_done)
        x_ref, info_ref = solvers.lsqr(lambda v: oracle.forward(S, v), lambda u: oracle.adjoint(S, u), s32, 10,
                                       damp=d)
        assert rel(host(x), x_ref) <= 1e-3, d
        assert abs(inf.rnorm - info_ref["rnorm"]) <= 1e-3 * info_ref["rnorm"]


def test_sweep_arguments():
    m = model("c0", B.OAM_PREC_FP32)
    s = dev(inputs.gaussian(m.sig_shape, 66))
    with pytest.raises(B.OamError):
        m.lsqr_sweep(s, 2, [0.1, -1.0])
    with pytest.raises(B.OamError):
        m.lsqr_sweep(s, 2, [0.1] * (B.OAM_MAX_SWEEP + 1))
    with pytest.raises(B.OamError):
        m.lsqr_sweep(s, 2, [float("inf")])
    xs, infos = m.lsqr_sweep(s, 0, [0.5])  # zero iterations: x = 0
    assert not host(xs[0]).any() and infos[0].iters_done == 0


# ------------------------------------------------------------------ full size (200x200x300, 0.5-80 MHz, L = 511)
def test_full_size_filter_sampled_lines():
    """The transform length and block shape the benchmark uses (nt = 1024,
    NF = 2048): sampled A-lines of F s against the direct FP64 sum."""
    m = model("c1", B.OAM_PREC_FFT)
    taps = bp.bandpass_taps(0.5e6, 80e6, FS, 511)
    m.set_filter(list(taps))
    assert m.info.filter_size == 2048
    s = inputs.gaussian(m.sig_shape, 67).astype(np.float32)
    got = host(m.filter_signals(dev(s)))
    rng = np.random.Generator(np.random.PCG64(68))
    ys = np.concatenate([rng.integers(0, 200, 30), [0, 199, 0, 199]])
    xs = np.concatenate([rng.integers(0, 200, 30), [0, 199, 199, 0]])
    want = bp.fir_time(s[ys, xs], taps)
    assert rel(got[ys, xs], want) <= 1e-5


@pytest.mark.parametrize("prec", [B.OAM_PREC_BF16X3, B.OAM_PREC_FFT])
def test_full_size_filtered_adjoint_identity(prec):
    m = model("c1", prec)
    m.set_filter(list(bp.bandpass_taps(0.5e6, 80e6, FS, 511)))
    x = inputs.gaussian(m.vol_shape, 69)
    y = inputs.gaussian(m.sig_shape, 70)
    Ax = host(m.forward(dev(x)))
    ATy = host(m.adjoint(dev(y)))
    lhs = float(np.dot(Ax.ravel(), y.astype(np.float32).ravel()))
    rhs = float(np.dot(x.astype(np.float32).ravel(), ATy.ravel()))
    assert abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(y)) < TOL[prec]


def test_full_size_sweep_equals_single_solves():
    m = model("c1", B.OAM_PREC_FFT)
    m.set_filter(list(bp.bandpass_taps(0.5e6, 80e6, FS, 511)))
    H = inputs.phantom(C1, 1, kind="spheres", count=50)
    s = m.filter_signals(m.forward(dev(H)))
    damps = [0.0, 1.0, 10.0]
    xs, infos = m.lsqr_sweep(s, 3, damps)
    for d, x, inf in zip(damps, xs, infos):
        x1, inf1 = m.lsqr(s, 3, damp=d)
        assert torch.equal(x, x1), d
        assert inf.rnorm == inf1.rnorm
