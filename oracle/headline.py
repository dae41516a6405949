"""FP64 reference reconstructions of a full workload (test infrastructure only).

Only the tests and the benchmark's CPU-baseline leg call this module; the
product path never does.  It applies the FP64 oracle's operators in their
cached-spectrum lateral-FFT form (``oracle.Spectral``, an exact restatement
of A and A^T pinned to the direct form) so that a 200 x 200-position,
61 x 61-tap, 300-depth, 1024-sample reconstruction -- about 340 operator
applications -- finishes in minutes on the host cores.  The slab columns are
evaluated once per symmetry orbit of the patch set (``symmetric=True``,
pinned to the tap-by-tap build).

``reference(cfg, ...)`` returns, for the seeded phantom of the workload:

* ``H32``: the phantom rounded to FP32 (what a device operator receives);
* ``AH``: A H32 in FP64 (Eq. 4 over the scan grid) -- the reference of the
  forward operator and the clean signals;
* ``s32``: AH plus seeded Gaussian noise at the given SNR, rounded to FP32
  (the measured signals both sides solve from);
* ``ATs``: A^T s32 in FP64 -- the reference of the adjoint;
* ``x_l2``: MB-L2 (Eq. 5 with Eq. 6, damp 0), ``lsqr_iters`` LSQR iterations
  from zero (Paige & Saunders);
* ``x_l1``: MB-L1 (Eq. 5 with Eq. 7), ``fista_iters`` FISTA iterations from
  zero with L from ``power_iters`` power iterations started at ``v0`` and
  lambda = lambda_rel * max|A^T s32|, non-negative (Beck & Teboulle);
* ``L``, ``lam``, ``lsqr_rnorm``: the scalars of both solvers, and
  ``seconds``: wall time of each part.
"""
import time

import numpy as np

from paper_2009_10173_gb300 import inputs

from . import Spectral, solvers


def reference(cfg, seed=1, n_spheres=50, snr_db=20.0, lsqr_iters=50, fista_iters=100, power_iters=20,
              lambda_rel=1e-3, v0_seed=7, on_signals=None):
    """FP64 references for one seeded volume of ``cfg``.

    ``on_signals(s32, H32)`` is called as soon as the signals exist (before
    the solvers run), so a caller can start its own reconstruction of the
    same signals while this one proceeds."""
    sec = {}
    t = time.perf_counter()
    sp = Spectral(cfg, symmetric=True)
    sec["spectrum"] = time.perf_counter() - t
    H = inputs.phantom(cfg, seed, kind="vessels", count=n_spheres)
    H32 = H.astype(np.float32)
    t = time.perf_counter()
    AH = sp.forward(H32.astype(np.float64))
    s32 = inputs.add_noise(AH, snr_db, seed + 10 ** 6).astype(np.float32)
    sec["forward"] = time.perf_counter() - t
    if on_signals is not None:
        on_signals(s32, H32)
    sd = s32.astype(np.float64)
    t = time.perf_counter()
    ATs = sp.adjoint(sd)
    sec["adjoint"] = time.perf_counter() - t
    t = time.perf_counter()
    x_l2, info = solvers.lsqr(sp.forward, sp.adjoint, sd, lsqr_iters)
    sec["lsqr"] = time.perf_counter() - t
    v0 = inputs.gaussian(H.shape, v0_seed).astype(np.float32).astype(np.float64)
    t = time.perf_counter()
    mu = solvers.power_iteration(sp.forward, sp.adjoint, v0, power_iters)
    L = 2.0 * mu * 1.01
    lam = lambda_rel * float(np.max(np.abs(ATs)))
    x_l1 = solvers.fista(sp.forward, sp.adjoint, sd, fista_iters, lam, L, nonneg=True)
    sec["fista"] = time.perf_counter() - t
    return dict(H32=H32, AH=AH, s32=s32, ATs=ATs, x_l2=x_l2, x_l1=x_l1, L=L, lam=lam,
                lsqr_rnorm=info["rnorm"], seconds=sec, P=sp.P, spectrum_bytes=sp.re.nbytes + sp.im.nbytes)
