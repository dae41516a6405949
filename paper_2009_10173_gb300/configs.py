"""Named workloads (sensor, grid and EIR parameters, SI units).

Each workload is a flat mapping whose keys are the fields of ``oam_sensor``,
``oam_grid`` and ``oam_eir`` in ``include/oam.h``.  The sensor follows the
paper's spherically focused PVDF detector (AR-OAM set-up) at a 4 mm focal
length and 3 mm aperture; the EIR is a Gaussian-windowed band-pass at 30 MHz
with 100 % fractional bandwidth; sampling is 250 MS/s as in every experiment
of the paper.  The first voxel depth is given relative to the focal depth.
"""
import copy

SENSOR_4MM = dict(focal_m=4e-3, aperture_m=3e-3, hole_m=0.0, c_mps=1500.0, n_patches=2000)
EIR_30MHZ = dict(fc_hz=30e6, frac_bw=1.0, trunc_sigma=5.0)

# 32x32 scan at 20 um, 32x32x48 voxels (20 um lateral, 10 um axial) starting
# 150 um before the focus, 192 samples, 11x11 slab window, 10 LSQR iterations.
TINY_32 = dict(**SENSOR_4MM, **EIR_30MHZ, px=32, py=32, nz=48, nt=192, win=11,
               dx_m=20e-6, dy_m=20e-6, dz_m=10e-6, z0_rel_m=-150e-6, fs_hz=250e6,
               t0_s=float("nan"), lsqr_iters=10)

# 200x200 scan at 10 um, 200x200x300 voxels (10 um lateral, 5 um axial)
# centred on the focus, 1024 samples, 61x61 slab window; 50 LSQR iterations
# and 100 non-negative L1-FISTA iterations (lambda = 1e-3 max|A^T s|).
VOLUME_200 = dict(**SENSOR_4MM, **EIR_30MHZ, px=200, py=200, nz=300, nt=1024, win=61,
                  dx_m=10e-6, dy_m=10e-6, dz_m=5e-6, z0_rel_m=-150 * 5e-6, fs_hz=250e6,
                  t0_s=float("nan"), lsqr_iters=50, fista_iters=100, power_iters=20,
                  lambda_rel=1e-3)

WORKLOADS = {"tiny_32x32x48": TINY_32, "volume_200x200x300": VOLUME_200}


def scaled(base, **over):
    """Copy of a workload with some fields replaced."""
    c = copy.deepcopy(base)
    c.update(over)
    return c


# Sizes drawn for the batched and served workloads: scan grids, depths and
# sample counts; the sensor's focal length and aperture are drawn per job.
BATCH_SCAN = (64, 96, 128, 160, 256)
BATCH_DEPTH = (128, 192, 256, 384)
BATCH_NT = (512, 768, 1024)
BATCH_FOCAL = (3e-3, 6e-3)
BATCH_APERTURE = (2e-3, 4e-3)


def batch_job(seed, base=None, nt_choice=None):
    """One reconstruction of the batched workload: a scan grid, depth count and
    sample count drawn from the batch sets, and a seeded sensor (focal length
    U[3, 6] mm, aperture U[2, 4] mm); other parameters as the 200x200x300
    workload, volume centred on the focus, 30 LSQR + 50 FISTA iterations."""
    import numpy as np
    base = VOLUME_200 if base is None else base
    rng = np.random.Generator(np.random.PCG64(seed))
    scan = int(rng.choice(BATCH_SCAN))
    nz = int(rng.choice(BATCH_DEPTH))
    nt = int(rng.choice(BATCH_NT)) if nt_choice is None else int(nt_choice)
    focal = float(rng.uniform(*BATCH_FOCAL))
    aperture = float(rng.uniform(*BATCH_APERTURE))
    return scaled(base, px=scan, py=scan, nz=nz, nt=nt, focal_m=focal, aperture_m=aperture,
                  z0_rel_m=-(nz / 2) * base["dz_m"], lsqr_iters=30, fista_iters=50, power_iters=20,
                  lambda_rel=1e-3, seed=seed)


def batch_workload(n=16, seed0=1000):
    """The batched workload: jobs with seeds seed0 .. seed0 + n - 1."""
    return [batch_job(seed0 + i) for i in range(n)]


def next_nt(cfg):
    """The next larger sample count of the batch set (used when the arrival
    window check fails), or None."""
    larger = [n for n in BATCH_NT if n > cfg["nt"]]
    return scaled(cfg, nt=larger[0]) if larger else None


def served_request(seed, p_large=0.05):
    """A request of the served workload: sizes as the batched workload, with
    probability p_large a 200x200x300 volume instead."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    if rng.uniform() < p_large:
        return scaled(VOLUME_200, lsqr_iters=30, fista_iters=50, power_iters=20, lambda_rel=1e-3, seed=seed)
    return batch_job(seed + 7919)
