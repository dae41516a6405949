"""Reconstructed images at the full 200x200x300 workload against FP64 references.

The workload: a 200 x 200-position scan at 10 um, 200 x 200 x 300 voxels
(10 um lateral, 5 um axial) centred on the focus, 1024 samples at 250 MS/s,
61 x 61-tap slab window, the seeded vessel-tree + 50-microsphere phantom
(seed 1) and 20 dB noise (seed 1 + 10^6).  ``oracle.headline.reference``
computes, in FP64 on the host cores, A H, A^T s, 50 LSQR iterations (MB-L2,
Eq. 5 with Eq. 6) and 100 FISTA iterations (MB-L1, Eq. 5 with Eq. 7; 20
power iterations from a seeded start vector, lambda = 1e-3 max|A^T s|,
non-negative), all from the same FP32 signals the device receives.

Every operator form of the library is compared with them element by element
(rel-L2): the operators at their tolerances (1e-5 FP32 and lateral-FFT
forms, 1e-4 split-BF16), both images at 1e-3.  The reference takes a few
minutes of host time and is computed once for all forms.
"""
import functools
import json

import numpy as np
import pytest
import torch

from oracle import headline
from paper_2009_10173_gb300 import binding as B
from paper_2009_10173_gb300 import configs, inputs
from paper_2009_10173_gb300.model import Model

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

C1 = configs.VOLUME_200
OP_TOL = {B.OAM_PREC_FP32: 1e-5, B.OAM_PREC_BF16X3: 1e-4, B.OAM_PREC_FFT: 1e-5}
IMAGE_TOL = 1e-3
NAMES = {B.OAM_PREC_FP32: "fp32", B.OAM_PREC_BF16X3: "bf16x3", B.OAM_PREC_FFT: "fft"}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@functools.lru_cache(maxsize=None)
def ref():
    return headline.reference(C1, seed=1, n_spheres=50, snr_db=20.0, lsqr_iters=50, fista_iters=100,
                              power_iters=20, lambda_rel=1e-3, v0_seed=7)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.mark.parametrize("prec", [B.OAM_PREC_BF16X3, B.OAM_PREC_FFT, B.OAM_PREC_FP32])
def test_full_size_results_match_fp64_reference(prec):
    r = ref()
    m = Model(C1, precision=prec)
    s = dev(r["s32"])
    err = {"A": rel(host(m.forward(dev(r["H32"]))), r["AH"]),
           "AT": rel(host(m.adjoint(s)), r["ATs"])}
    x2, info2 = m.lsqr(s, 50)
    err["lsqr_image"] = rel(host(x2), r["x_l2"])
    v0 = dev(inputs.gaussian(m.vol_shape, 7))
    x1, info1 = m.fista(s, 100, power_iters=20, lambda_rel=1e-3, nonneg=True, v0=v0)
    err["fista_image"] = rel(host(x1), r["x_l1"])
    err["L"] = abs(info1.L - r["L"]) / r["L"]
    err["lambda"] = abs(info1.lambda_ - r["lam"]) / r["lam"]
    m.close()
    print(json.dumps({"form": NAMES[prec], "rel_err_vs_fp64": err, "oracle_seconds": r["seconds"]}))
    assert err["A"] <= OP_TOL[prec] and err["AT"] <= OP_TOL[prec]
    assert err["lsqr_image"] <= IMAGE_TOL
    assert err["fista_image"] <= IMAGE_TOL
    assert err["L"] < 1e-4 and err["lambda"] < 1e-4
