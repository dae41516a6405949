"""The paper's own discretisation of Eq. 1 on the GPU (OAM_DISC_TRILINEAR).

Methods, Forward modeling: the surface integral of Eq. 1 is taken of the
trilinear interpolation of the voxel values and the time derivative by a
finite difference.  The library builds that slab on the device in FP64
(k_slab33_values) and every operator form, the solvers and the filter use it
unchanged.  Expected values come from ``oracle.slab33_column`` (pinned in
tests/test_oracle_discretised.py) and the oracle's direct A / A^T on the dense
discretised slab.  Tolerances as everywhere: slab 1e-6, FP32 operators 1e-5,
split-BF16 1e-4 (rel-L2).
"""
import functools
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2009_10173_gb300 import binding as B
from paper_2009_10173_gb300 import configs, inputs
from paper_2009_10173_gb300.model import Model

pytestmark = pytest.mark.gpu

CFG = configs.scaled(configs.TINY_32, px=24, py=20, nz=16, nt=256, win=7, n_patches=400, z0_rel_m=-80e-6)
TOL = {B.OAM_PREC_FP32: 1e-5, B.OAM_PREC_BF16X3: 1e-4, B.OAM_PREC_FFT: 1e-5}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def margin(cfg):
    """Samples by which trilinear voxels reach beyond point voxels (the library's rule)."""
    return math.ceil(cfg["fs_hz"] * (cfg["dx_m"] + cfg["dy_m"] + cfg["dz_m"]) / cfg["c_mps"]) + 2


@functools.lru_cache(maxsize=None)
def dense():
    t0 = oracle.t0(CFG) - margin(CFG) / CFG["fs_hz"]
    R, W = (CFG["win"] - 1) // 2, CFG["win"]
    S = np.zeros((W, W, CFG["nz"], CFG["nt"]))
    for b in range(-R, R + 1):
        for a in range(-R, R + 1):
            for k in range(CFG["nz"]):
                S[b + R, a + R, k] = oracle.slab33_column(CFG, b, a, k, t0)
    return t0, S


def model(prec):
    return Model(CFG, precision=prec, discretisation=B.OAM_DISC_TRILINEAR)


def test_slab_and_time_origin_match_oracle():
    t0, S = dense()
    m = model(B.OAM_PREC_FP32)
    assert abs(m.info.t0_s - t0) * CFG["fs_hz"] < 1e-6  # automatic origin: point rule minus the margin
    R = (CFG["win"] - 1) // 2
    got = np.zeros_like(S)
    col = torch.empty(CFG["nt"], device="cuda")
    for b in range(-R, R + 1):
        for a in range(-R, R + 1):
            for k in range(CFG["nz"]):
                B.oam_model_slab_column(m.handle, b, a, k, col)
                got[b + R, a + R, k] = col.cpu().numpy()
    assert rel(got, S) < 1e-6
    m.close()


@pytest.mark.parametrize("prec", [B.OAM_PREC_FP32, B.OAM_PREC_BF16X3, B.OAM_PREC_FFT])
def test_operators_match_oracle(prec):
    _, S = dense()
    m = model(prec)
    H = inputs.gaussian(m.vol_shape, 61)
    s = inputs.gaussian(m.sig_shape, 62)
    got = m.forward(torch.from_numpy(H.astype(np.float32)).cuda()).double().cpu().numpy()
    assert rel(got, oracle.forward(S, H.astype(np.float32).astype(np.float64))) < TOL[prec]
    got = m.adjoint(torch.from_numpy(s.astype(np.float32)).cuda()).double().cpu().numpy()
    assert rel(got, oracle.adjoint(S, s.astype(np.float32).astype(np.float64))) < TOL[prec]
    m.close()


def test_model_bytes_bounds_the_discretised_model():
    for prec in (B.OAM_PREC_FP32, B.OAM_PREC_BF16X3, B.OAM_PREC_FFT):
        m = model(prec)
        planned = B.oam_model_bytes(CFG, prec, B.OAM_DISC_TRILINEAR)
        assert m.info.device_bytes <= planned <= 1.15 * m.info.device_bytes + (1 << 20)
        m.close()


def test_two_absorber_demonstration_separates_as_the_paper_reports():
    """The second simulation (Methods, Numerical simulations; Results, Fig. 2a,b)
    on synthetic signals of the discretised model: both methods resolve two
    20 um absorbers 60 um apart, only MB-L1 resolves them 40 um apart, and
    MB-L1's profile of one absorber is narrower than MB-L2's.  Qualitative
    checks only (the paper's FWHM values are context)."""
    from paper_2009_10173_gb300 import demo_two_absorbers as D
    r = D.run((60, 40))["results"]
    assert r["60.0um"]["MB-L2"]["resolved"] and r["60.0um"]["MB-L1"]["resolved"]
    assert r["40.0um"]["MB-L1"]["resolved"] and not r["40.0um"]["MB-L2"]["resolved"]
    assert r["single"]["MB-L1"]["fwhm_um"] < r["single"]["MB-L2"]["fwhm_um"]
