"""CUDA path vs the FP64 oracle, through the C-ABI (needs a GB300).

Tolerances: rel-L2 <= 1e-5 for the FP32 operators (direct and lateral-FFT
form) and the slab, <= 1e-4 for the split-BF16 tensor-core operators, <= 1e-3
for reconstructed images after the stated iteration counts.  Inputs are seeded; every expected value comes
from ``oracle/``.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
from oracle import solvers
from paper_2009_10173_gb300 import binding as B
from paper_2009_10173_gb300 import configs, inputs
from paper_2009_10173_gb300.model import Model

pytestmark = pytest.mark.gpu

C0 = configs.TINY_32
C1 = configs.VOLUME_200
# 70x37 scan, 52 depths, 200 samples, 15x15 window: ragged position, depth and time tiles
RAGGED = configs.scaled(C0, px=70, py=37, nz=52, nt=200, win=15, n_patches=800, dz_m=8e-6, z0_rel_m=-200e-6)

PRECS = [B.OAM_PREC_FP32, B.OAM_PREC_BF16X3, B.OAM_PREC_FFT]
TOL = {B.OAM_PREC_FP32: 1e-5, B.OAM_PREC_BF16X3: 1e-4, B.OAM_PREC_FFT: 1e-5}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@functools.lru_cache(maxsize=None)
def oracle_slab(name):
    cfg = {"c0": C0, "ragged": RAGGED}[name]
    return oracle.slab(cfg)


_models = {}


def model(name, prec):
    key = (name, prec)
    if key not in _models:
        cfg = {"c0": C0, "ragged": RAGGED, "c1": C1}.get(name) if isinstance(name, str) else name
        try:
            _models[key] = Model(cfg, precision=prec)
        except B.OamError as e:
            if e.code == B.OAM_ERR_UNSUPPORTED and prec == B.OAM_PREC_BF16X3:
                pytest.skip("tensor-core path not built")
            raise
    return _models[key]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


# ------------------------------------------------------------------ slab
@pytest.mark.parametrize("name", ["c0", "ragged"])
def test_slab_matches_oracle(name):
    cfg = {"c0": C0, "ragged": RAGGED}[name]
    S = oracle_slab(name)
    m = model(name, B.OAM_PREC_FP32)
    assert abs(m.info.t0_s - oracle.t0(cfg)) < 1e-15
    R = (cfg["win"] - 1) // 2
    got = np.zeros_like(S)
    for b in range(-R, R + 1):
        for a in range(-R, R + 1):
            for k in range(cfg["nz"]):
                got[b + R, a + R, k] = host(m.slab_column(b, a, k))
    assert rel(got, S) < 1e-6
    # the band layout keeps every nonzero entry
    assert m.info.nnz >= int((S != 0).sum())


# ------------------------------------------------------------------ operators
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["c0", "ragged"])
@pytest.mark.parametrize("kind", ["gaussian", "phantom"])
def test_forward_adjoint_match_oracle(name, prec, kind):
    cfg = {"c0": C0, "ragged": RAGGED}[name]
    S = oracle_slab(name)
    m = model(name, prec)
    shape_v = (cfg["py"], cfg["px"], cfg["nz"])
    shape_s = (cfg["py"], cfg["px"], cfg["nt"])
    if kind == "gaussian":
        H = inputs.gaussian(shape_v, 101)
        s = inputs.gaussian(shape_s, 102)
    else:
        H = inputs.phantom(cfg, 0, count=8)
        s = oracle.forward(S, H)
    # compare against the oracle applied to the same FP32-rounded inputs
    H32 = H.astype(np.float32).astype(np.float64)
    s32 = s.astype(np.float32).astype(np.float64)
    assert rel(host(m.forward(dev(H))), oracle.forward(S, H32)) < TOL[prec]
    assert rel(host(m.adjoint(dev(s))), oracle.adjoint(S, s32)) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_operator_edge_cases(prec):
    # single tap, single row, single column, and zero input
    for over in (dict(win=1), dict(py=1, px=33), dict(px=1, py=9), dict(win=3, px=2, py=2, nz=5, nt=128)):
        cfg = configs.scaled(C0, n_patches=200, **over)
        S = oracle.slab(cfg)
        try:
            m = Model(cfg, precision=prec)
        except B.OamError as e:
            if e.code == B.OAM_ERR_UNSUPPORTED and prec == B.OAM_PREC_BF16X3:
                pytest.skip("tensor-core path not built")
            raise
        H = inputs.gaussian((cfg["py"], cfg["px"], cfg["nz"]), 7)
        s = inputs.gaussian((cfg["py"], cfg["px"], cfg["nt"]), 8)
        assert rel(host(m.forward(dev(H))), oracle.forward(S, H.astype(np.float32))) < TOL[prec]
        assert rel(host(m.adjoint(dev(s))), oracle.adjoint(S, s.astype(np.float32))) < TOL[prec]
        z = m.forward(torch.zeros(m.vol_shape, device="cuda"))
        assert not host(z).any()
        m.close()


def test_window_and_argument_errors():
    with pytest.raises(B.OamError) as e:
        Model(configs.scaled(C0, nt=100))
    assert e.value.code == B.OAM_ERR_WINDOW
    m = model("c0", B.OAM_PREC_FP32)
    L = B.lib()
    H = torch.zeros(m.vol_shape, device="cuda")
    s = torch.zeros(m.sig_shape, device="cuda")
    import ctypes
    assert L.oam_forward(m.handle, ctypes.c_void_p(H.data_ptr() + 4), ctypes.c_void_p(s.data_ptr()), None) == \
        B.OAM_ERR_INVALID_ARG
    assert L.oam_model_slab_column(m.handle, 99, 0, 0, ctypes.c_void_p(s.data_ptr()), None) == B.OAM_ERR_INVALID_ARG


def test_gpu_shift_invariance_bit_exact():
    """(b) on the device: shifting H by one scan step shifts A H by one position."""
    m = model("c0", B.OAM_PREC_FP32)
    R = 5
    H = np.zeros(m.vol_shape)
    H[R + 1:32 - R - 2, R + 1:32 - R - 2] = inputs.uniform((32 - 2 * R - 3, 32 - 2 * R - 3, 48), 9)
    a = host(m.forward(dev(H)))
    bx = host(m.forward(dev(np.roll(H, 1, axis=1))))
    by = host(m.forward(dev(np.roll(H, 1, axis=0))))
    assert np.array_equal(np.roll(a, 1, axis=1), bx)
    assert np.array_equal(np.roll(a, 1, axis=0), by)


# ------------------------------------------------------------------ solvers
def c0_signals():
    S = oracle_slab("c0")
    H = inputs.phantom(C0, 0, count=8)
    s = inputs.add_noise(oracle.forward(S, H), 20.0, 10 ** 6)
    return S, H, s


@pytest.mark.parametrize("prec", PRECS)
def test_lsqr_matches_oracle_c0(prec):
    S, H, s = c0_signals()
    m = model("c0", prec)
    s32 = s.astype(np.float32).astype(np.float64)
    A, AT = (lambda v: oracle.forward(S, v)), (lambda v: oracle.adjoint(S, v))
    x_ref, info_ref = solvers.lsqr(A, AT, s32, 10)
    x, info = m.lsqr(dev(s), 10)
    assert info.iters_done == 10 and info.stop_reason == 0
    assert rel(host(x), x_ref) < 1e-3
    assert abs(info.rnorm - info_ref["rnorm"]) / info_ref["rnorm"] < 1e-3
    # damped (Tikhonov, Eq. 6) variant
    x_ref, _ = solvers.lsqr(A, AT, s32, 10, damp=3.0)
    x, _ = m.lsqr(dev(s), 10, damp=3.0)
    assert rel(host(x), x_ref) < 1e-3


def test_lsqr_zero_signal_stops():
    m = model("c0", B.OAM_PREC_FP32)
    x, info = m.lsqr(torch.zeros(m.sig_shape, device="cuda"), 5)
    assert info.iters_done == 0 and info.stop_reason == 1
    assert not host(x).any()


@pytest.mark.parametrize("prec", PRECS)
def test_fista_matches_oracle_c0(prec):
    S, H, s = c0_signals()
    m = model("c0", prec)
    s32 = s.astype(np.float32).astype(np.float64)
    A, AT = (lambda v: oracle.forward(S, v)), (lambda v: oracle.adjoint(S, v))
    v0 = inputs.gaussian(m.vol_shape, 7).astype(np.float32)
    x_ref, ref = solvers.mb_l1(A, AT, s32, 100, 20, v0.astype(np.float64), lambda_rel=1e-3, nonneg=True)
    x, info = m.fista(dev(s), 100, power_iters=20, lambda_rel=1e-3, nonneg=True, v0=dev(v0),
                      compute_objective=True)
    assert abs(info.L - ref["L"]) / ref["L"] < 1e-4
    assert abs(info.lambda_ - ref["lam"]) / ref["lam"] < 1e-4
    assert rel(host(x), x_ref) < 1e-3
    assert abs(info.objective - ref["objective"]) / ref["objective"] < 1e-3
    assert host(x).min() >= 0


# ------------------------------------------------------------------ full size (200x200x300, 61x61 window)
@functools.lru_cache(maxsize=None)
def c1_t0():
    return oracle.t0(C1)


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_impulse_matches_oracle_columns(prec):
    """A delta voxel gives the slab columns back at every position in its window."""
    m = model("c1", prec)
    assert abs(m.info.t0_s - c1_t0()) < 1e-15
    H = torch.zeros(m.vol_shape, device="cuda")
    y0, x0, k0 = 100, 57, 150
    H[y0, x0, k0] = 1.0
    s = host(m.forward(H))
    got, want = [], []
    for (b, a) in ((0, 0), (1, 0), (0, 30), (-30, 30), (17, -4), (-29, -30)):
        got.append(s[y0 - b, x0 - a])
        want.append(oracle.slab_column(C1, b, a, k0, c1_t0()))
    assert rel(np.array(got), np.array(want)) < TOL[prec]
    # positions outside the window see nothing (the lateral-FFT form: rounding
    # noise of its transforms only)
    outside = np.concatenate([s[y0 + 31].ravel(), s[y0, x0 - 31].ravel()])
    if prec == B.OAM_PREC_FFT:
        assert np.abs(outside).max() <= 1e-6 * np.abs(s).max()
    else:
        assert not outside.any()


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_forward_sampled(prec):
    m = model("c1", prec)
    H = inputs.phantom(C1, 1, kind="spheres", count=50)
    H += 0.1 * inputs.uniform(H.shape, 2, 0.0, 1.0)
    s = host(m.forward(dev(H)))
    ns = [100, 160]
    slices = np.stack([oracle.slab_time_slice(C1, n, c1_t0()) for n in ns])
    rng = np.random.Generator(np.random.PCG64(5))
    ys = np.concatenate([rng.integers(0, 200, 24), [0, 199, 0, 199]])
    xs = np.concatenate([rng.integers(0, 200, 24), [0, 199, 199, 0]])
    which = np.arange(len(ys)) % 2
    want = oracle.forward_at(slices, H.astype(np.float32), ys, xs, which)
    got = np.array([s[y, x, ns[w]] for y, x, w in zip(ys, xs, which)])
    assert rel(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_adjoint_sampled(prec):
    m = model("c1", prec)
    sig = inputs.gaussian(m.sig_shape, 3).astype(np.float32)
    Ht = host(m.adjoint(dev(sig)))
    R = 30
    ks = [40, 220]
    rng = np.random.Generator(np.random.PCG64(6))
    pts = [(int(y), int(x)) for y, x in zip(rng.integers(0, 200, 6), rng.integers(0, 200, 6))] + [(0, 0), (199, 3)]
    got, want = [], []
    for k in ks:
        cols = np.zeros((61, 61, C1["nt"]))
        for b in range(-R, R + 1):
            for a in range(-R, R + 1):
                cols[b + R, a + R] = oracle.slab_column(C1, b, a, k, c1_t0())
        for (y, x) in pts:
            acc = 0.0
            for b in range(-R, R + 1):
                if not 0 <= y - b < 200:
                    continue
                for a in range(-R, R + 1):
                    if 0 <= x - a < 200:
                        acc += float(np.dot(cols[b + R, a + R], sig[y - b, x - a].astype(np.float64)))
            want.append(acc)
            got.append(Ht[y, x, k])
    assert rel(np.array(got), np.array(want)) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_adjoint_identity(prec):
    m = model("c1", prec)
    x = inputs.gaussian(m.vol_shape, 21)
    y = inputs.gaussian(m.sig_shape, 22)
    Ax = host(m.forward(dev(x)))
    ATy = host(m.adjoint(dev(y)))
    lhs = float(np.dot(Ax.ravel(), y.astype(np.float32).ravel()))
    rhs = float(np.dot(x.astype(np.float32).ravel(), ATy.ravel()))
    assert abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(y)) < TOL[prec]


def test_full_size_lsqr_residual_estimate():
    """LSQR's |phibar| equals the true residual ||s - A x_k|| and never increases."""
    m = model("c1", B.OAM_PREC_FP32)
    H = inputs.phantom(C1, 1, kind="spheres", count=50)
    s = m.forward(dev(H))
    prev = np.inf
    for k in (1, 2, 4):
        x, info = m.lsqr(s, k)
        r = host(m.forward(x)) - host(s)
        true = float(np.linalg.norm(r))
        assert abs(info.rnorm - true) / true < 1e-3
        assert info.rnorm <= prev
        prev = info.rnorm


@pytest.mark.parametrize("px", [300, 600, 1100])
def test_fft_form_wide_grids(px):
    """Transform sizes P = 512, 1024 and 2048 (fewer channels per FFT block)
    on thin grids the oracle applies directly."""
    cfg = configs.scaled(C0, px=px, py=3, nz=9, nt=128, win=3, n_patches=200)
    S = oracle.slab(cfg)
    m = Model(cfg, precision=B.OAM_PREC_FFT)
    H = inputs.gaussian((cfg["py"], cfg["px"], cfg["nz"]), 41)
    s = inputs.gaussian((cfg["py"], cfg["px"], cfg["nt"]), 42)
    assert rel(host(m.forward(dev(H))), oracle.forward(S, H.astype(np.float32))) < TOL[B.OAM_PREC_FFT]
    assert rel(host(m.adjoint(dev(s))), oracle.adjoint(S, s.astype(np.float32))) < TOL[B.OAM_PREC_FFT]
    m.close()


def test_fft_form_rejects_grids_beyond_its_transform_size():
    with pytest.raises(B.OamError) as e:
        Model(configs.scaled(C0, px=2100, py=2, nz=4, nt=128, win=3, n_patches=200), precision=B.OAM_PREC_FFT)
    assert e.value.code == B.OAM_ERR_UNSUPPORTED


# ------------------------------------------------------------------ pre-build footprint
@pytest.mark.parametrize("prec", PRECS)
def test_model_bytes_bounds_the_built_model(prec):
    """oam_model_bytes (host only, before any allocation) is an upper bound
    of the built model's device memory, within a few per cent."""
    cases = [C0, RAGGED, configs.batch_job(1000), configs.batch_job(1003), C1]
    for cfg in cases:
        try:
            m = Model(cfg, precision=prec)
        except B.OamError as e:
            if e.code == B.OAM_ERR_WINDOW:  # such a job moves to the next sample count
                continue
            raise
        planned = B.oam_model_bytes(cfg, prec)
        built = m.info.device_bytes
        m.close()
        assert built <= planned <= 1.15 * built + (1 << 20), (cfg["py"], cfg["nz"], built, planned)
