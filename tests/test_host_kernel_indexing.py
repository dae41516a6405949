"""Index arithmetic of the shared-memory FFT kernels, checked on the CPU.

The band-pass filter kernel (``k_fir_lines`` in ``csrc/op_filter.cu``) and the
lateral-FFT form's register-pass transforms (``k_xfft_*`` in
``csrc/op_fft.cu``) address shared memory and global memory through a few
formulas.  This test restates those formulas and checks, for every transform
length the kernels accept:

* the passes cover every transform stage exactly once, largest span first for
  forward (decimation in frequency) and smallest first for inverse (decimation
  in time);
* every pass visits each (point, line) once, its slots are distinct and lie
  inside the shared memory the launch allocates, and the kernels' linear slot
  steps equal the slot formula;
* accesses of 16 consecutive work items (a half-warp of 8-byte accesses, or a
  quarter-warp of 16-byte ones) hit distinct banks where the padding is meant
  to ensure it;
* global offsets of loads and stores stay inside the arrays for ragged line
  counts;
* float64 models of the stage arithmetic, run through the same schedules on
  small sizes, give numpy's DFT and the direct convolution.

The kernels' own arithmetic is checked by the GPU parity tests.
"""
import numpy as np
import pytest


# ------------------------------------------------------------------ k_fir_lines
def fir_slot(KP, i, p):
    return i * KP + p + (i >> 3)


def fir_nslots(KP, NF):  # fir_smem / 16 bytes
    return KP * NF + NF // 8


def fir_pairs_per_block(NF):
    return max(1, min(8, 4096 // NF))


def fir_schedule(lgNF):
    """(k, r) of the forward outer passes, the middle's spans, the inverse passes."""
    r0 = ((lgNF - 3) & 3) or 4
    k0 = lgNF - r0
    fwd = [(k0, r0)] + [(k, 4) for k in range(k0 - 4, 2, -4)]
    inv = [(k, 4) for k in range(3, k0 - 3, 4) if k + 4 <= k0] + [(k0, r0)]
    return fwd, inv


def fir_pass_items(KP, NF, k, r):
    """(pair, i0, slots of the group's points) per work item, as dif_pass / dit_pass."""
    groups = NF >> r
    ds = (KP << k) + (1 << (k - 3))
    for idx in range(groups * KP):
        p, t = idx % KP, idx // KP
        q, blk = t & ((1 << k) - 1), t >> k
        i0 = (blk << (k + r)) | q
        s0 = fir_slot(KP, i0, p)
        yield p, i0, [s0 + m * ds for m in range(1 << r)], [i0 + (m << k) for m in range(1 << r)]


@pytest.mark.parametrize("lgNF", range(4, 14))
def test_fir_schedule_covers_every_stage_once(lgNF):
    fwd, inv = fir_schedule(lgNF)
    spans_f = [k + j for k, r in fwd for j in reversed(range(r))]
    assert spans_f == list(range(lgNF - 1, 2, -1))   # spans NF/2 .. 8, largest first; the middle does 4, 2, 1
    spans_i = [k + j for k, r in inv for j in range(r)]
    assert spans_i == list(range(3, lgNF))            # spans 8 .. NF/2 after the middle
    assert all(k >= 3 for k, _ in fwd + inv)          # point steps 2^k are multiples of 8 (linear slot steps)


@pytest.mark.parametrize("lgNF", range(4, 14))
def test_fir_passes_visit_every_point_once_inside_shared_memory(lgNF):
    NF = 1 << lgNF
    assert 16 * fir_nslots(fir_pairs_per_block(NF), NF) <= 227 * 1024  # the launched shape fits a block
    for KP in sorted({1, 2, fir_pairs_per_block(NF)}):
        n = fir_nslots(KP, NF)
        every = {fir_slot(KP, i, p) for i in range(NF) for p in range(KP)}
        assert len(every) == NF * KP and max(every) < n
        fwd, inv = fir_schedule(lgNF)
        for k, r in set(fwd + inv):
            seen = set()
            for p, _, slots, points in fir_pass_items(KP, NF, k, r):
                assert slots == [fir_slot(KP, i, p) for i in points]
                seen.update((i, p) for i in points)
            assert len(seen) == NF * KP
        # the middle: 8-point groups at base + j KP
        for g in range(NF >> 3):
            for p in range(KP):
                base = fir_slot(KP, 8 * g, p)
                assert [base + j * KP for j in range(8)] == [fir_slot(KP, 8 * g + j, p) for j in range(8)]


@pytest.mark.parametrize("KP", [1, 2, 4, 8])
def test_fir_middle_pass_is_bank_conflict_free(KP):
    """16-byte slots: 8 consecutive groups (one quarter-warp) fall in 8 distinct
    16-byte bank groups for every point j of the group."""
    NF = 2048
    groups = NF >> 3
    for g0 in range(0, groups, 8):
        for j in range(8):
            banks = {(fir_slot(KP, 8 * g + j, 0)) % 8 for g in range(g0, g0 + 8)}
            assert len(banks) == 8


@pytest.mark.parametrize("nt,n_lines", [(1024, 40000), (192, 1023), (4, 3), (1000, 7)])
def test_fir_global_offsets_stay_inside(nt, n_lines):
    L = 511 if nt > 511 else nt - 1
    lgNF = 4
    while (1 << lgNF) < nt + min(L, nt - 1):
        lgNF += 1
    NF = 1 << lgNF
    KP = fir_pairs_per_block(NF)
    blocks = (n_lines + 4 * KP - 1) // (4 * KP)
    fwd, _ = fir_schedule(lgNF)
    k0, r0 = fwd[0]
    for b in sorted({0, blocks - 1}):
        line0 = b * 4 * KP
        for p, _, _, points in fir_pass_items(KP, NF, k0, r0):
            for n in points:
                if n >= nt:
                    continue
                for role in range(4):
                    if line0 + 4 * p + role < n_lines:
                        assert 0 <= (line0 + 4 * p + role) * nt + n < n_lines * nt


# ------------------------------------------------------------------ k_xfft_*
def x_slot(KL, i, l):
    return i * KL + l + ((i >> 4) * KL if KL < 16 else 0)


def x_nslots(KL, P):
    return P * KL + ((P >> 4) * KL if KL < 16 else 0)


def x_schedule(lgP, forward):
    """(kf, r) of each pass in execution order, as xtransform."""
    npass = (lgP + 3) // 4
    r0 = lgP - 4 * (npass - 1)
    out = []
    for pi in range(npass):
        pp = pi if forward else npass - 1 - pi
        out.append((4 * (npass - 1 - pp), r0 if pp == 0 else 4))
    return out


def x_pass_points(KL, P, k, r):
    groups = P >> r
    for idx in range(groups * KL):
        l, t = idx % KL, idx // KL
        q, blk = t & ((1 << k) - 1), t >> k
        i0 = (blk << (k + r)) | q
        yield idx, l, [i0 + (m << k) for m in range(1 << r)]


@pytest.mark.parametrize("lgP", range(4, 12))
def test_xfft_schedule_covers_every_stage_once(lgP):
    f = x_schedule(lgP, True)
    assert [k + j for k, r in f for j in reversed(range(r))] == list(range(lgP - 1, -1, -1))
    i = x_schedule(lgP, False)
    assert [k + j for k, r in i for j in range(r)] == list(range(lgP))
    assert all(k % 4 == 0 for k, _ in f)


@pytest.mark.parametrize("lgP", range(4, 12))
@pytest.mark.parametrize("KL", [1, 2, 4, 8, 16])
def test_xfft_passes_visit_every_point_once_without_bank_conflicts(lgP, KL):
    P = 1 << lgP
    n = x_nslots(KL, P)
    assert 8 * n <= 48 * 1024 or KL * P > 4096  # the shapes the form launches fit the default 48 KB
    every = {x_slot(KL, i, l) for i in range(P) for l in range(KL)}
    assert len(every) == P * KL and max(every) < n
    for k, r in set(x_schedule(lgP, True)):
        items = list(x_pass_points(KL, P, k, r))
        assert len({(i, l) for _, l, pts in items for i in pts}) == P * KL
        # 16 consecutive items (one half-warp of 8-byte accesses): distinct banks per point m
        for h in range(0, len(items) - 15, 16):
            for m in range(1 << r):
                pairs = set()
                for idx, l, pts in items[h:h + 16]:
                    s = x_slot(KL, pts[m], l)
                    pairs.add((2 * s) % 32)
                assert len(pairs) == 16, (k, r, h, m)


# ------------------------------------------------------------------ the schedules carry out the transforms
# Float64 models of the two kernels' stage arithmetic (the twiddle of span S at
# point n is W_2S^(n mod S), factored as W_2S^q times a 16-point constant, the
# q factor from one base twiddle by squaring), run through the schedules above
# and compared with numpy's FFT.  Small sizes only; the GPU tests check the
# kernels themselves.

def _w16(N, u):
    return np.exp(-2j * np.pi * u / N)


def _pass(P, k, r, forward, v_of, put):
    """One pass of r stages over the groups of all lines, as xpass / dif_pass / dit_pass."""
    R = 1 << r
    for t in range(P >> r):
        q, blk = t & ((1 << k) - 1), t >> k
        i0 = (blk << (k + r)) | q
        v = [v_of(i0 + (m << k)) for m in range(R)]
        pw = [None] * r
        pw[r - 1] = np.exp(-2j * np.pi * q / (1 << (k + r)))
        for j in range(r - 2, -1, -1):
            pw[j] = pw[j + 1] ** 2
        order = range(r - 1, -1, -1) if forward else range(r)
        for j in order:
            S = 1 << j
            for m in range(R):
                if m & S:
                    continue
                um = m & (S - 1)
                tw = pw[j] if um == 0 else pw[j] * _w16(2 * S, um)
                u, w = v[m], v[m + S]
                if forward:
                    v[m], v[m + S] = u + w, (u - w) * tw
                else:
                    w = w * np.conj(tw)
                    v[m], v[m + S] = u + w, u - w
        for m in range(R):
            put(i0 + (m << k), v[m])


def _bitrev(x, lg):
    return int(format(x, "0%db" % lg)[::-1], 2) if lg else 0


@pytest.mark.parametrize("lgP", [4, 5, 6, 7, 8, 9])
def test_xfft_schedules_compute_the_dft(lgP):
    P = 1 << lgP
    rng = np.random.Generator(np.random.PCG64(lgP))
    x = rng.standard_normal(P) + 1j * rng.standard_normal(P)
    a = x.copy()
    for k, r in x_schedule(lgP, True):
        _pass(P, k, r, True, lambda i: a[i], a.__setitem__)
    X = np.fft.fft(x)
    assert np.allclose([a[_bitrev(f, lgP)] for f in range(P)], X, atol=1e-10 * np.abs(X).max())
    b = np.array([X[_bitrev(i, lgP)] for i in range(P)])  # inverse input: frequency bitrev(i) at position i
    for k, r in x_schedule(lgP, False):
        _pass(P, k, r, False, lambda i: b[i], b.__setitem__)
    assert np.allclose(b / P, x, atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("lgNF,L", [(4, 3), (5, 10), (7, 40), (8, 100), (9, 200)])
def test_fir_schedule_computes_the_convolution(lgNF, L):
    """Forward outer passes, the 8-point middle (spans 4, 2, 1, product,
    spans 1, 2, 4), inverse outer passes: a circular convolution with the even
    taps, equal to the direct sum on the first NF - L points."""
    NF = 1 << lgNF
    nt = NF - L
    rng = np.random.Generator(np.random.PCG64(100 + lgNF))
    x = rng.standard_normal(nt) + 1j * rng.standard_normal(nt)
    h = rng.standard_normal(L + 1)
    f = np.arange(NF)
    H = h[0] + 2 * sum((h[m] * np.cos(2 * np.pi * f * m / NF) for m in range(1, L + 1)), np.zeros(NF))
    hb = np.array([H[_bitrev(i, lgNF)] for i in range(NF)]) / NF
    a = np.zeros(NF, complex)
    a[:nt] = x
    fwd, inv = fir_schedule(lgNF)
    for k, r in fwd:
        _pass(NF, k, r, True, lambda i: a[i], a.__setitem__)
    for g in range(NF >> 3):  # the middle: forward spans 4, 2, 1 on 8-point groups, product, inverse spans 1, 2, 4
        _pass(8, 0, 3, True, lambda i: a[8 * g + i], lambda i, v: a.__setitem__(8 * g + i, v))
        a[8 * g: 8 * g + 8] *= hb[8 * g: 8 * g + 8]
        _pass(8, 0, 3, False, lambda i: a[8 * g + i], lambda i, v: a.__setitem__(8 * g + i, v))
    for k, r in inv:
        _pass(NF, k, r, False, lambda i: a[i], a.__setitem__)
    full = np.concatenate([h[:0:-1], h])
    want = np.convolve(x, full)[L:L + nt]
    assert np.allclose(a[:nt], want, atol=1e-10 * np.abs(want).max())


# ------------------------------------------------------------------ k_corr_fold
def strip_rows_for(px, R):
    return 128 + ((px + 126) // px + 2) * R


@pytest.mark.parametrize("tiling", ["padded", "scan"])
@pytest.mark.parametrize("px,py,R", [(32, 32, 5), (24, 20, 3), (64, 64, 30), (96, 96, 30), (128, 128, 30),
                                     (160, 160, 30), (200, 200, 30), (256, 256, 30), (33, 7, 4), (1, 9, 5)])
def test_corr_fold_strip_rows_hold_every_tap_of_every_lane(px, py, R, tiling):
    """Tiles of 128 consecutive positions of the padded grid (stride Wp = px + R)
    or the scan grid (stride px): lane m of tile t reads strip row pm + R + a,
    pm its padded offset from the tile's first position, of the strip that
    starts at padded index (R+1)*Wp + q_t + b*Wp - R.  That row must lie in the
    staged strip and be the padded index of (y + b, x + a), which is a zero
    padding column when x + a falls outside the row."""
    wp = px + R
    sp = px if tiling == "scan" else wp
    rows = strip_rows_for(px, R) if tiling == "scan" else 128 + 2 * R
    for t in range((py * sp + 127) // 128):
        y0, x0 = t * 128 // sp, t * 128 % sp
        qt = y0 * wp + x0
        m = np.arange(128)
        o = t * 128 + m
        y, x = o // sp, o % sp
        pm = (y - y0) * wp + (x - x0)
        if tiling == "padded":
            assert np.array_equal(pm, m)
        for a in (-R, -1, 0, 1, R):
            r = pm + R + a
            assert r.min() >= 0 and r.max() < rows
            for b in (-R, 0, R):
                start = (R + 1) * wp + qt + b * wp - R
                q = start + r
                assert np.array_equal(q, (y + b + R + 1) * wp + x + a)
                col = q % wp
                out = x < px  # lanes whose results are kept (padding positions of the padded grid are dropped)
                inside = (x + a >= 0) & (x + a < px)
                assert np.array_equal(col[inside & out], (x + a)[inside & out])
                assert (col[~inside & out] >= px).all()
    if R <= 30 and px >= 64 or tiling == "padded":
        assert rows <= 256  # one TMA box
