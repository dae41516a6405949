"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the reconstruction arithmetic: it draws absorber
volumes (phantoms), additive Gaussian noise for a given clean signal, and
start vectors.  Every draw uses numpy's PCG64 with an explicit seed in FP64.

The paper's datasets (microsphere and carbon-fibre phantoms, mouse skin) are
measured data; these generators stand in for them with the same kind of
structure: Gaussian microspheres of 20-50 um diameter and a branching tree of
tubes of 5-30 um radius.  ``paraboloids`` draws the truncated paraboloids of
the paper's simulations (no randomness).
"""
import math

import numpy as np


def _grid(cfg):
    px, py, nz = cfg["px"], cfg["py"], cfg["nz"]
    x = np.arange(px) * cfg["dx_m"]
    y = np.arange(py) * cfg["dy_m"]
    z = cfg["z0_rel_m"] + np.arange(nz) * cfg["dz_m"]
    return x, y, z


def microspheres(cfg, count, seed, dmin=20e-6, dmax=50e-6, amin=0.5, amax=1.0, out=None):
    """Gaussian blobs amp * exp(-4 ln2 |x - c|^2 / D^2) (FWHM = diameter D).

    Centres are uniform in the interior, keeping a lateral margin of R scan
    steps and an axial margin of one diameter.  Layout H[py][px][nz], FP64.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x, y, z = _grid(cfg)
    R = (cfg["win"] - 1) // 2
    H = np.zeros((cfg["py"], cfg["px"], cfg["nz"])) if out is None else out
    for _ in range(count):
        D = rng.uniform(dmin, dmax)
        amp = rng.uniform(amin, amax)
        mx = min(R * cfg["dx_m"], 0.45 * x[-1]) if len(x) > 1 else 0.0
        my = min(R * cfg["dy_m"], 0.45 * y[-1]) if len(y) > 1 else 0.0
        cx = rng.uniform(mx, x[-1] - mx) if len(x) > 1 else 0.0
        cy = rng.uniform(my, y[-1] - my) if len(y) > 1 else 0.0
        mz = min(D, 0.45 * (z[-1] - z[0])) if len(z) > 1 else 0.0
        cz = rng.uniform(z[0] + mz, z[-1] - mz) if len(z) > 1 else z[0]
        k = 4.0 * math.log(2.0) / (D * D)
        # only touch voxels within 3 diameters of the centre
        sl = []
        for coord, c in ((y, cy), (x, cx), (z, cz)):
            lo = np.searchsorted(coord, c - 3 * D)
            hi = np.searchsorted(coord, c + 3 * D, side="right")
            sl.append(slice(lo, hi))
        gy, gx, gz = np.meshgrid(y[sl[0]], x[sl[1]], z[sl[2]], indexing="ij")
        blob = amp * np.exp(-k * ((gx - cx) ** 2 + (gy - cy) ** 2 + (gz - cz) ** 2))
        H[sl[0], sl[1], sl[2]] = np.maximum(H[sl[0], sl[1], sl[2]], blob)
    return H


def vessel_tree(cfg, seed, root_radius=30e-6, min_radius=5e-6, out=None):
    """A seeded branching tree of straight tubes, binary inside, merged by max.

    The root enters at the volume's centre depth from one lateral side; each
    segment is 100-400 um long, children shrink by U[0.7, 0.9] and branch
    off at U[20, 60] degrees, and growth stops below ``min_radius`` or when a
    segment leaves the volume.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x, y, z = _grid(cfg)
    H = np.zeros((cfg["py"], cfg["px"], cfg["nz"])) if out is None else out
    lo = np.array([x[0], y[0], z[0]])
    hi = np.array([x[-1], y[-1], z[-1]])

    def inside(p):
        return bool(np.all(p >= lo) and np.all(p <= hi))

    def tube(p0, p1, r):
        bmin, bmax = np.minimum(p0, p1) - r, np.maximum(p0, p1) + r
        sl = []
        for coord, a, b in ((y, bmin[1], bmax[1]), (x, bmin[0], bmax[0]), (z, bmin[2], bmax[2])):
            sl.append(slice(np.searchsorted(coord, a), np.searchsorted(coord, b, side="right")))
        if any(s.stop <= s.start for s in sl):
            return
        gy, gx, gz = np.meshgrid(y[sl[0]], x[sl[1]], z[sl[2]], indexing="ij")
        P = np.stack([gx, gy, gz], axis=-1)
        d = p1 - p0
        L2 = float(np.dot(d, d))
        t = np.clip(((P - p0) @ d) / L2, 0.0, 1.0) if L2 > 0 else np.zeros(P.shape[:-1])
        dist2 = np.sum((P - (p0 + t[..., None] * d)) ** 2, axis=-1)
        H[sl[0], sl[1], sl[2]] = np.maximum(H[sl[0], sl[1], sl[2]], (dist2 <= r * r).astype(np.float64))

    zc = 0.5 * (z[0] + z[-1])
    start = np.array([x[0], y[0] + rng.uniform(0.3, 0.7) * (y[-1] - y[0]), zc])
    ang = rng.uniform(-0.3, 0.3)
    direction = np.array([math.cos(ang), math.sin(ang), rng.uniform(-0.2, 0.2)])
    stack = [(start, direction / np.linalg.norm(direction), root_radius, 0)]
    segments = 0
    while stack and segments < 4000:
        p0, dvec, r, depth = stack.pop()
        length = rng.uniform(100e-6, 400e-6)
        p1 = p0 + length * dvec
        tube(p0, p1, r)
        segments += 1
        if not inside(p1):
            continue
        for sign in (1.0, -1.0):
            rc = r * rng.uniform(0.7, 0.9)
            if rc < min_radius:
                continue
            theta = math.radians(rng.uniform(20.0, 60.0)) * sign
            c, s = math.cos(theta), math.sin(theta)
            nd = np.array([c * dvec[0] - s * dvec[1], s * dvec[0] + c * dvec[1],
                           dvec[2] + rng.uniform(-0.15, 0.15)])
            stack.append((p1, nd / np.linalg.norm(nd), rc, depth + 1))
    return H


def paraboloids(cfg, centres, diameter):
    """Truncated paraboloids max(0, 1 - |x - c|^2 / (D/2)^2) of diameter D at the
    given centres (metres, in the frame of ``_grid``: x = i dx, y = j dy,
    z = z0_rel + k dz), merged by max.  Layout H[py][px][nz], FP64."""
    x, y, z = _grid(cfg)
    gy, gx, gz = np.meshgrid(y, x, z, indexing="ij")
    H = np.zeros((cfg["py"], cfg["px"], cfg["nz"]))
    r2 = (0.5 * diameter) ** 2
    for cx, cy, cz in centres:
        H = np.maximum(H, np.maximum(0.0, 1.0 - ((gx - cx) ** 2 + (gy - cy) ** 2 + (gz - cz) ** 2) / r2))
    return H


def phantom(cfg, seed, kind="spheres", count=8):
    """Named phantoms: 'spheres' (``count`` microspheres) or 'vessels'
    (a vessel tree plus ``count`` microspheres)."""
    if kind == "spheres":
        return microspheres(cfg, count, seed)
    if kind == "vessels":
        H = vessel_tree(cfg, seed)
        return microspheres(cfg, count, seed + 1, out=H)
    raise ValueError(kind)


def add_noise(clean, snr_db, seed):
    """clean + N(0, sigma^2) with sigma = rms(clean) * 10^(-snr_db / 20)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    clean = np.asarray(clean, np.float64)
    rms = float(np.sqrt(np.mean(clean * clean)))
    sigma = rms * 10.0 ** (-snr_db / 20.0)
    return clean + sigma * rng.standard_normal(clean.shape)


def gaussian(shape, seed):
    """Standard normal draws (FP64), e.g. random test vectors or a start vector."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(shape)


def uniform(shape, seed, lo=-1.0, hi=1.0):
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, shape)
