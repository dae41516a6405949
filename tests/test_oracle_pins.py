"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, exact invariants of the scanning geometry, brute force from the true
per-pair geometry, library solvers (scipy / numpy) and hand-derived values in
``tests/golden/closed_forms.json``.  None of them needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import solvers
from paper_2009_10173_gb300 import configs, inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
C0 = configs.TINY_32


def small(**over):
    """A small grid for pins that need many operator applications."""
    base = dict(C0)
    base.update(dict(px=8, py=8, nz=8, nt=96, win=5, n_patches=400, dz_m=20e-6,
                     z0_rel_m=-80e-6))
    base.update(over)
    return base


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# --------------------------------------------------------------------- Eq. 3
def test_patch_area_count_and_rings():
    nx, ny, nz, w = oracle.patches(C0)
    assert len(w) == C0["n_patches"]
    assert abs(w.sum() * 1e6 - GOLD["sensor_area_mm2"]["value"]) < 1e-11
    assert oracle.ring_count(C0) == GOLD["ring_count_m2000"]["value"]
    # every patch lies on the unit sphere and inside the aperture cone
    assert np.allclose(nx ** 2 + ny ** 2 + nz ** 2, 1.0, atol=1e-15)
    assert np.all(np.sqrt(nx ** 2 + ny ** 2) <= 0.375 + 1e-15)


def test_patch_area_with_hole():
    cfg = dict(C0, hole_m=0.9e-3, n_patches=1600)
    nx, ny, nz, w = oracle.patches(cfg)
    F, D, h = 4e-3, 3e-3, 0.9e-3
    exact = 2 * math.pi * F * F * (math.cos(math.asin(h / (2 * F))) - math.cos(math.asin(D / (2 * F))))
    assert abs(w.sum() - exact) / exact < 1e-14
    assert np.all(np.sqrt(nx ** 2 + ny ** 2) >= h / (2 * F) - 1e-15)


@pytest.mark.parametrize("M", [8, 400, 2000, 2008])
def test_patch_d4_symmetry(M):
    """The patch set maps onto itself under x<->y, x->-x and y->-y (axial symmetry, Results)."""
    nx, ny, nz, w = oracle.patches(dict(C0, n_patches=M))
    P = np.stack([nx, ny, nz, w], 1)
    for T in ((1, 0, 0, 1), (0, 1, 1, 0), (-1, 0, 0, 1), (1, 0, 0, -1)):
        Q = P.copy()
        Q[:, 0] = T[0] * P[:, 0] + T[1] * P[:, 1]
        Q[:, 1] = T[2] * P[:, 0] + T[3] * P[:, 1]
        d = np.abs(P[:, None, :] - Q[None, :, :]).max(-1).min(1)
        assert d.max() < 1e-15


def test_patch_invalid():
    with pytest.raises(oracle.OracleError):
        oracle.patches(dict(C0, n_patches=2001))
    with pytest.raises(oracle.OracleError):
        oracle.patches(dict(C0, aperture_m=9e-3))


# ----------------------------------------------------------------------- EIR
def test_eir_sigma_and_bandwidth():
    """-6 dB full width of the EIR amplitude spectrum = frac_bw * fc."""
    fs, fc = C0["fs_hz"], C0["fc_hz"]
    sig = GOLD["eir_sigma_samples"]["value"]
    tau = np.arange(-400, 401) * 0.05  # fine grid, samples
    e = oracle.eir(C0, tau)
    # the envelope at one sigma
    assert abs(oracle.eir(C0, [sig])[0] / math.cos(2 * math.pi * fc / fs * sig) - math.exp(-0.5)) < 1e-9
    spec = np.abs(np.fft.rfft(e, 1 << 16))
    f = np.fft.rfftfreq(1 << 16, d=0.05 / fs)
    spec /= spec.max()
    above = f[spec >= 0.5]
    # the mirrored lobe at -fc moves the half-amplitude points by ~0.3 %
    assert abs((above.max() - above.min()) - C0["frac_bw"] * fc) / fc < 5e-3
    assert abs(f[np.argmax(spec)] - fc) / fc < 5e-3
    # truncation at 5 sigma
    assert oracle.eir(C0, [5.01 * sig])[0] == 0.0


def test_eir_derivative_matches_difference_quotient():
    tau = np.linspace(-14, 14, 57)
    h = 1e-5
    num = (oracle.eir(C0, tau + h) - oracle.eir(C0, tau - h)) / (2 * h)
    ana = oracle.eir_dot(C0, tau)
    assert np.max(np.abs(num - ana)) < 1e-8


# ------------------------------------------------------------------ Eqs. 1-4
def brute_distance_range(cfg, y0=3, x0=5):
    """Shortest and longest voxel-patch distance over the slab window, from
    absolute coordinates: the sensor sits over scan point (y0, x0) (focus at
    (x0 dx, y0 dy, 0), surface points focus - F n_j), the voxels of the
    win x win x nz window around it sit at their absolute positions."""
    nx, ny, nz, _ = oracle.patches(cfg)
    F = cfg["focal_m"]
    R = (cfg["win"] - 1) // 2
    fx, fy = x0 * cfg["dx_m"], y0 * cfg["dy_m"]
    q = np.stack([fx - F * nx, fy - F * ny, -F * nz], 1)                  # (M, 3)
    yy, xx, kk = np.meshgrid(np.arange(y0 - R, y0 + R + 1), np.arange(x0 - R, x0 + R + 1),
                             np.arange(cfg["nz"]), indexing="ij")
    v = np.stack([xx.ravel() * cfg["dx_m"], yy.ravel() * cfg["dy_m"],
                  cfg["z0_rel_m"] + kk.ravel() * cfg["dz_m"]], 1)          # (voxels, 3)
    d = np.sqrt(((v[:, None, :] - q[None, :, :]) ** 2).sum(-1))
    return float(d.min()), float(d.max())


@pytest.mark.parametrize("over", [{}, dict(win=5, nz=8, z0_rel_m=40e-6, dx_m=30e-6, dy_m=10e-6)])
def test_distance_range_matches_brute_force(over):
    """The oracle's distance range equals a numpy min / max over every
    (voxel, patch) pair of the window, taken in absolute coordinates."""
    cfg = dict(C0, **over)
    dmin, dmax = oracle.distance_range(cfg)
    bmin, bmax = brute_distance_range(cfg)
    assert abs(dmin - bmin) <= 1e-15 * bmin and abs(dmax - bmax) <= 1e-15 * bmax
    if not over:  # the tiny workload's window holds the focal voxel: dmin <= F <= dmax
        assert dmin <= C0["focal_m"] <= dmax


def test_time_origin_rule_and_window():
    """Reading of the unstated time origin: the earliest arrival minus the
    EIR half-width falls in [2, 3) samples after t0, and the window check
    passes exactly when the latest arrival plus the half-width is below nt.
    dmin / dmax come from the brute-force range, not from the oracle."""
    t0 = oracle.t0(C0)
    dmin, dmax = brute_distance_range(C0)
    fs, c = C0["fs_hz"], C0["c_mps"]
    cut = 5 * GOLD["eir_sigma_samples"]["value"]
    n_first = fs * (dmin / c - t0) - cut
    assert 2.0 <= n_first < 3.0 + 1e-9
    assert abs(t0 * fs - round(t0 * fs)) < 1e-6          # t0 on the sample grid
    n_last = fs * (dmax / c - t0) + cut
    assert n_last < C0["nt"]
    nt_edge = int(math.floor(n_last))                    # n_last >= nt_edge: rejected
    with pytest.raises(oracle.OracleError):
        oracle.t0(dict(C0, nt=nt_edge))
    assert oracle.t0(dict(C0, nt=nt_edge + 1)) == t0     # t0 does not depend on nt
    with pytest.raises(oracle.OracleError):
        oracle.t0(dict(C0, nt=100))


def test_focal_point_single_arrival():
    """(a) A point at the focus: every patch is at distance F, so the slab
    column is the sensor area / F times one EIR arrival at t = F / c."""
    t0 = oracle.t0(C0)
    kf = int(round(-C0["z0_rel_m"] / C0["dz_m"]))
    assert kf == 15
    col = oracle.slab_column(C0, 0, 0, kf, t0)
    F, c, fs = C0["focal_m"], C0["c_mps"], C0["fs_hz"]
    area_mm2 = GOLD["sensor_area_mm2"]["value"]
    D = fs * (F / c - t0)
    sig = GOLD["eir_sigma_samples"]["value"]
    om = 2 * math.pi * C0["fc_hz"] / fs
    n = np.arange(C0["nt"])
    tau = n - D
    # d/dtau of exp(-tau^2/2sig^2) cos(om tau), written from the product rule
    env = np.exp(-tau ** 2 / (2 * sig ** 2))
    expect = env * (-(tau / sig ** 2) * np.cos(om * tau) - om * np.sin(om * tau))
    expect[np.abs(tau) > 5 * sig] = 0.0
    expect *= area_mm2 / (F * 1e3)
    assert rel(col, expect) < 1e-9  # sigma known to 1e-9 relative in the fixture
    # the exact statement with the oracle's own EIR: to rounding
    exact = area_mm2 / (F * 1e3) * oracle.eir_dot(C0, tau)
    assert rel(col, exact) < 1e-12


def continuum_on_axis(cfg, zeta, t0):
    """Continuous-aperture limit for an on-axis point zeta beyond the focus:
    S(n) = (2 pi F / zeta)(c / fs)[e(n - D(theta_max)) - e(n - D(theta_min))]."""
    F, Dap, c, fs = cfg["focal_m"], cfg["aperture_m"], cfg["c_mps"], cfg["fs_hz"]
    tmax = math.asin(Dap / (2 * F))
    d = lambda th: math.sqrt(F * F + zeta * zeta + 2 * F * zeta * math.cos(th))
    n = np.arange(cfg["nt"])
    e1 = oracle.eir(cfg, n - fs * (d(tmax) / c - t0))
    e0 = oracle.eir(cfg, n - fs * (d(0.0) / c - t0))
    return (2 * math.pi * F / zeta) * (c / fs) * 1e3 * (e1 - e0)


def test_on_axis_converges_to_continuum():
    errs = []
    t0 = oracle.t0(C0)
    for M in (2000, 8000, 32000):
        cfg = dict(C0, n_patches=M)
        k = 30  # 150 um beyond the focus
        zeta = C0["z0_rel_m"] + k * C0["dz_m"]
        col = oracle.slab_column(cfg, 0, 0, k, t0)
        errs.append(rel(col, continuum_on_axis(cfg, zeta, t0)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3


def test_slab_d4_symmetry():
    S = oracle.slab(small())
    assert rel(S.transpose(1, 0, 2, 3), S) < 1e-13
    assert rel(S[::-1], S) < 1e-13
    assert rel(S[:, ::-1], S) < 1e-13


def test_slab_helpers_agree():
    cfg = small()
    t0 = oracle.t0(cfg)
    S = oracle.slab(cfg, t0)
    assert np.array_equal(oracle.slab_column(cfg, -1, 2, 3, t0), S[1, 4, 3])
    sl = oracle.slab_time_slice(cfg, 40, t0)
    assert np.max(np.abs(sl - S[..., 40])) <= 1e-13 * np.abs(S).max()


def test_impulse_response():
    """A delta voxel at (y0, x0, k0) gives s[y, x, :] = S[y0-y, x0-x, k0, :]."""
    cfg = small()
    S = oracle.slab(cfg)
    R = (cfg["win"] - 1) // 2
    H = np.zeros((cfg["py"], cfg["px"], cfg["nz"]))
    y0, x0, k0 = 3, 5, 4
    H[y0, x0, k0] = 1.0
    s = oracle.forward(S, H)
    for y in range(cfg["py"]):
        for x in range(cfg["px"]):
            b, a = y0 - y, x0 - x
            if abs(b) <= R and abs(a) <= R:
                assert np.array_equal(s[y, x], S[b + R, a + R, k0])
            else:
                assert not s[y, x].any()


def test_shift_invariance():
    """(b) Shifting the volume by one scan step shifts the signals by one
    position, bit for bit, when the volume keeps a zero margin of R + 1."""
    cfg = small(px=12, py=10)
    S = oracle.slab(cfg)
    R = (cfg["win"] - 1) // 2
    H = np.zeros((cfg["py"], cfg["px"], cfg["nz"]))
    inner = inputs.uniform((cfg["py"] - 2 * R - 3, cfg["px"] - 2 * R - 3, cfg["nz"]), 3)
    H[R + 1:R + 1 + inner.shape[0], R + 1:R + 1 + inner.shape[1]] = inner
    s = oracle.forward(S, H)
    s_x = oracle.forward(S, np.roll(H, 1, axis=1))
    s_y = oracle.forward(S, np.roll(H, 1, axis=0))
    assert np.array_equal(np.roll(s, 1, axis=1), s_x)
    assert np.array_equal(np.roll(s, 1, axis=0), s_y)


def test_adjoint_identity():
    """(c) <A x, y> = <x, A^T y> to 1e-12 relative."""
    cfg = small(px=9, py=7)
    S = oracle.slab(cfg)
    x = inputs.gaussian((7, 9, cfg["nz"]), 11)
    y = inputs.gaussian((7, 9, cfg["nt"]), 12)
    lhs = float(np.dot(oracle.forward(S, x).ravel(), y.ravel()))
    rhs = float(np.dot(x.ravel(), oracle.adjoint(S, y).ravel()))
    scale = np.linalg.norm(oracle.forward(S, x)) * np.linalg.norm(y)
    assert abs(lhs - rhs) / scale < 1e-12


def _edot(tau, sig, om):
    env = np.exp(-tau ** 2 / (2 * sig ** 2))
    out = env * (-(tau / sig ** 2) * np.cos(om * tau) - om * np.sin(om * tau))
    out[np.abs(tau) > 5 * sig] = 0.0
    return out


def dense_brute_force(cfg, t0):
    """The model matrix built pair by pair (voxel, scan point) from absolute
    coordinates: sensor patches about the scan point's focus, voxels at their
    absolute positions, Eq. 3 summed over patches.  Rows (y, x, n), columns
    (y', x', k); pairs beyond the lateral window are zero."""
    nx, ny, nz, w = oracle.patches(cfg)
    F, c, fs = cfg["focal_m"], cfg["c_mps"], cfg["fs_hz"]
    sig = fs / (2 * math.pi * cfg["fc_hz"] * cfg["frac_bw"] / (2 * math.sqrt(2 * math.log(2))))
    om = 2 * math.pi * cfg["fc_hz"] / fs
    py, px, Nz, nt = cfg["py"], cfg["px"], cfg["nz"], cfg["nt"]
    R = (cfg["win"] - 1) // 2
    A = np.zeros((py * px * nt, py * px * Nz))
    n = np.arange(nt)
    for y in range(py):
        for x in range(px):
            fx, fy = x * cfg["dx_m"], y * cfg["dy_m"]          # focus of this scan point
            qx, qy, qz = fx - F * nx, fy - F * ny, -F * nz     # sensor surface points
            for yy in range(py):
                for xx in range(px):
                    if abs(yy - y) > R or abs(xx - x) > R:
                        continue
                    for k in range(Nz):
                        vx, vy = xx * cfg["dx_m"], yy * cfg["dy_m"]
                        vz = cfg["z0_rel_m"] + k * cfg["dz_m"]
                        d = np.sqrt((vx - qx) ** 2 + (vy - qy) ** 2 + (vz - qz) ** 2)
                        D = fs * (d / c - t0)
                        col = ((w / d * 1e3)[:, None] * _edot(n[None, :] - D[:, None], sig, om)).sum(0)
                        A[(y * px + x) * nt:(y * px + x + 1) * nt, (yy * px + xx) * Nz + k] = col
    return A


def test_dense_brute_force_equals_slab_correlation():
    """(d) The dense model matrix from the true per-pair geometry (8x8x8 grid,
    5x5 window) equals the slab correlation to 1e-13."""
    cfg = small(n_patches=96, nt=64, nz=8, dz_m=20e-6, z0_rel_m=-60e-6)
    t0 = oracle.t0(cfg)
    S = oracle.slab(cfg, t0)
    A = dense_brute_force(cfg, t0)
    H = inputs.gaussian((8, 8, 8), 5)
    s_dense = (A @ H.ravel()).reshape(8, 8, cfg["nt"])
    assert rel(oracle.forward(S, H), s_dense) < 1e-13
    sig = inputs.gaussian((8, 8, cfg["nt"]), 6)
    assert rel(oracle.adjoint(S, sig), (A.T @ sig.ravel()).reshape(8, 8, 8)) < 1e-13


def test_forward_at_matches_forward():
    cfg = small()
    t0 = oracle.t0(cfg)
    S = oracle.slab(cfg, t0)
    H = inputs.gaussian((cfg["py"], cfg["px"], cfg["nz"]), 8)
    s = oracle.forward(S, H)
    ns = [30, 45]
    slices = np.stack([oracle.slab_time_slice(cfg, n, t0) for n in ns])
    ys, xs, which = [0, 3, 7, 5], [0, 4, 7, 1], [0, 1, 0, 1]
    got = oracle.forward_at(slices, H, ys, xs, which)
    want = np.array([s[y, x, ns[i]] for y, x, i in zip(ys, xs, which)])
    assert np.max(np.abs(got - want)) <= 1e-12 * np.abs(s).max()


# ------------------------------------------------------------------ solvers
def _dense_ops(M):
    return (lambda v: M @ v), (lambda v: M.T @ v)


@pytest.mark.parametrize("damp", [0.0, 0.3])
def test_lsqr_matches_scipy_random(damp):
    from scipy.sparse.linalg import lsqr as sp_lsqr
    M = inputs.gaussian((60, 25), 21)
    b = inputs.gaussian(60, 22)
    A, AT = _dense_ops(M)
    for k in (1, 3, 10):
        x, _ = solvers.lsqr(A, AT, b, k, damp=damp)
        ref = sp_lsqr(M, b, damp=damp, atol=0, btol=0, conlim=0, iter_lim=k)[0]
        assert rel(x, ref) < 1e-10


def test_lsqr_matches_scipy_on_slab_operator():
    from scipy.sparse.linalg import lsqr as sp_lsqr
    cfg = small(px=6, py=6, nz=6, n_patches=96, nt=64, z0_rel_m=-60e-6)
    t0 = oracle.t0(cfg)
    S = oracle.slab(cfg, t0)
    Adense = dense_brute_force(cfg, t0)
    s = inputs.gaussian((6, 6, cfg["nt"]), 31)
    A = lambda v: oracle.forward(S, v)
    AT = lambda v: oracle.adjoint(S, v)
    for k in (1, 5, 10):
        x, _ = solvers.lsqr(A, AT, s, k)
        ref = sp_lsqr(Adense, s.ravel(), atol=0, btol=0, conlim=0, iter_lim=k)[0]
        assert rel(x.ravel(), ref) < 1e-10


def test_lsqr_residual_monotone_and_recovers_phantom():
    """(e) LSQR recovers a noiseless tiny phantom; ||r_k|| never increases."""
    cfg = small(px=6, py=6, nz=4, n_patches=96, nt=96, dz_m=40e-6, z0_rel_m=-80e-6, win=3)
    S = oracle.slab(cfg)
    H = inputs.uniform((6, 6, 4), 41, 0.0, 1.0)
    s = oracle.forward(S, H)
    A = lambda v: oracle.forward(S, v)
    AT = lambda v: oracle.adjoint(S, v)
    norms = []
    x, info = solvers.lsqr(A, AT, s, 400, callback=lambda i, x, r: norms.append(r))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(norms, norms[1:]))
    assert rel(x, H) < 1e-6
    # the same least-squares solution as numpy's dense solver
    Ad = dense_brute_force(cfg, oracle.t0(cfg))
    ref = np.linalg.lstsq(Ad, s.ravel(), rcond=None)[0]
    assert rel(x.ravel(), ref) < 1e-6


def test_power_iteration_vs_eigvalsh():
    U = np.linalg.qr(inputs.gaussian((40, 40), 51))[0]
    V = np.linalg.qr(inputs.gaussian((20, 20), 52))[0]
    sv = np.linspace(1.0, 3.0, 20)
    sv[-1] = 6.0
    M = U[:, :20] @ np.diag(sv) @ V.T
    A, AT = _dense_ops(M)
    mu = solvers.power_iteration(A, AT, inputs.gaussian(20, 7), 20)
    top = np.linalg.eigvalsh(M.T @ M)[-1]
    assert mu <= top * (1 + 1e-12)
    assert abs(mu - top) / top < 1e-10


def test_fista_first_iterate_closed_form():
    M = inputs.gaussian((30, 12), 61)
    b = inputs.gaussian(30, 62)
    A, AT = _dense_ops(M)
    L, lam = 2.0 * np.linalg.eigvalsh(M.T @ M)[-1] * 1.01, 0.7
    x1 = solvers.fista(A, AT, b, 1, lam, L, nonneg=True)
    z = (2.0 / L) * (M.T @ b)
    assert np.allclose(x1, np.maximum(z - lam / L, 0.0), rtol=0, atol=1e-15)
    x1s = solvers.fista(A, AT, b, 1, lam, L, nonneg=False)
    assert np.allclose(x1s, np.sign(z) * np.maximum(np.abs(z) - lam / L, 0.0), rtol=0, atol=1e-15)


def test_fista_converges_to_nnls_and_lstsq():
    from scipy.optimize import nnls
    M = inputs.gaussian((40, 15), 71)
    b = inputs.gaussian(40, 72)
    A, AT = _dense_ops(M)
    L = 2.0 * np.linalg.eigvalsh(M.T @ M)[-1] * 1.01
    x = solvers.fista(A, AT, b, 3000, 0.0, L, nonneg=True)
    assert rel(x, nnls(M, b)[0]) < 1e-8
    x = solvers.fista(A, AT, b, 3000, 0.0, L, nonneg=False)
    assert rel(x, np.linalg.lstsq(M, b, rcond=None)[0]) < 1e-8


def test_fista_kkt_and_rate_bound():
    M = inputs.gaussian((50, 20), 81)
    b = inputs.gaussian(50, 82)
    A, AT = _dense_ops(M)
    L = 2.0 * np.linalg.eigvalsh(M.T @ M)[-1] * 1.01
    lam = 2.0
    xs = solvers.fista(A, AT, b, 5000, lam, L, nonneg=True)
    g = 2.0 * M.T @ (M @ xs - b)
    on = xs > 1e-10
    assert np.max(np.abs(g[on] + lam)) < 1e-7
    assert np.all(g[~on] + lam >= -1e-7)
    Fstar = solvers.fista_objective(A, b, xs, lam)
    for k in (1, 5, 20, 100):
        xk = solvers.fista(A, AT, b, k, lam, L, nonneg=True)
        bound = 2 * L * float(np.dot(xs, xs)) / (k + 1) ** 2
        assert solvers.fista_objective(A, b, xk, lam) - Fstar <= bound + 1e-12
