"""Pins for the oracle's version of the paper's own discretisation of Eq. 1.

The Methods (Forward modeling, with its ref. [33]) discretise Eq. 1 in two
steps: the surface integral over the sphere |x - x'| = ct of the trilinear
interpolation of the voxel values, and a finite difference for the time
derivative.  The oracle's reading (``oracle.tent_radon``,
``oracle.slab33_column``): each voxel is a trilinear tent, the sphere is
planar across a tent's support (sagitta < 1e-3 voxel), so the surface
integral is the tent's planar Radon transform (a six-box spline in closed
form); the derivative is a central difference on the sample grid; the patch
sum of Eq. 3 and the sampled EIR follow.  What pins it:

* the closed-form Radon transform equals a brute-force quadrature over the
  plane, for generic, axis-aligned and nearly degenerate normals, and
  integrates to the tent's volume;
* every column sums to zero (the central difference telescopes);
* the column has the patch set's mirror and x <-> y symmetry;
* for tents much smaller than a wavelength sampled much finer than the tent,
  the column tends to (V fs / c) times the point-voxel column of the
  independently pinned point model, with second-order convergence.
"""
import numpy as np
import pytest

import oracle
from paper_2009_10173_gb300 import configs


def brute_radon(d, e, s, n=601):
    e = np.asarray(e, float) / np.linalg.norm(e)
    t = np.array([1.0, 0.0, 0.0]) if abs(e[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u1 = np.cross(e, t)
    u1 /= np.linalg.norm(u1)
    u2 = np.cross(e, u1)
    lim = 2.0 * np.linalg.norm(d)
    g = np.linspace(-lim, lim, n)
    h = g[1] - g[0]
    U, V = np.meshgrid(g, g, indexing="ij")
    out = []
    for si in np.ravel(s):
        P = [si * e[i] + U * u1[i] + V * u2[i] for i in range(3)]
        phi = np.prod([np.maximum(0.0, 1.0 - np.abs(P[i]) / d[i]) for i in range(3)], axis=0)
        out.append(phi.sum() * h * h)
    return np.array(out)


@pytest.mark.parametrize("e", [(0.3, -0.5, 0.81), (0.0, 0.0, 1.0), (1e-3, 0.0, 1.0), (0.7, 0.7, 0.14),
                               (1.0, 0.0, 0.0)])
def test_tent_radon_matches_plane_quadrature(e):
    d = (0.010, 0.010, 0.005)
    e = np.asarray(e) / np.linalg.norm(e)
    s = np.linspace(-0.022, 0.022, 11)
    got = oracle.tent_radon(d, e, s)
    want = brute_radon(d, e, s)
    assert np.max(np.abs(got - want)) <= 1e-4 * np.max(np.abs(want))


def test_tent_radon_integrates_to_the_tent_volume():
    d = (0.010, 0.007, 0.005)
    for e in [(0.3, -0.5, 0.81), (0.0, 0.6, 0.8), (0.0, 0.0, 1.0)]:
        e = np.asarray(e) / np.linalg.norm(e)
        s = np.linspace(-0.03, 0.03, 6001)
        area = np.trapezoid(oracle.tent_radon(d, e, s), s)
        assert abs(area - d[0] * d[1] * d[2]) <= 1e-6 * d[0] * d[1] * d[2]


def small_cfg(**over):
    return configs.scaled(configs.TINY_32, n_patches=400, win=5, nz=4, px=6, py=6, nt=256, **over)


def test_columns_telescope_and_are_symmetric():
    cfg = small_cfg()
    t0 = oracle.t0(cfg)
    cols = {}
    for (b, a) in [(1, 2), (2, 1), (-1, 2), (1, -2), (-2, -1)]:
        cols[(b, a)] = oracle.slab33_column(cfg, b, a, 2, t0)
    ref = cols[(1, 2)]
    scale = np.abs(ref).max()
    assert scale > 0
    assert abs(ref.sum()) <= 1e-9 * scale * len(ref)
    for key, col in cols.items():
        assert np.max(np.abs(col - ref)) <= 1e-8 * scale, key  # same terms, other order


def test_tends_to_the_point_voxel_model():
    base = configs.scaled(configs.TINY_32, n_patches=400, win=3, nz=3, px=4, py=4)
    errs = []
    for h_um, fs in [(4, 2e9), (2, 4e9), (1, 8e9)]:
        h = h_um * 1e-6
        cfg = configs.scaled(base, dx_m=h, dy_m=h, dz_m=h, z0_rel_m=-h, fs_hz=fs, nt=int(4096 * fs / 2e9))
        t0 = oracle.t0(cfg)
        scale = cfg["c_mps"] * 1e3 / ((h * 1e3) ** 3 * fs)
        s33 = oracle.slab33_column(cfg, 1, 1, 2, t0) * scale
        sp = oracle.slab_column(cfg, 1, 1, 2, t0)
        errs.append(np.linalg.norm(s33 - sp) / np.linalg.norm(sp))
    assert errs[2] < 3e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5  # second order
