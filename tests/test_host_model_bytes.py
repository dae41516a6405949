"""oam_model_bytes: the pre-build device-memory query, on the host.

The model is one scanning position's slab (Results; Methods, Efficient
reconstruction based on scanning symmetries), so its size is set by the
window, depths, samples and sensor, not by how many positions are scanned;
only the split-BF16 operators' staging buffers grow with the scan.  These
checks run without a GPU: the query makes no device call.  The bound against
built models is checked on a GPU in tests/test_gpu_parity.py.
"""
import pytest

from paper_2009_10173_gb300 import binding as B
from paper_2009_10173_gb300 import configs

PRECS = (B.OAM_PREC_FP32, B.OAM_PREC_BF16X3, B.OAM_PREC_FFT)


@pytest.mark.parametrize("prec", PRECS)
def test_answers_without_a_device(prec):
    n = B.oam_model_bytes(configs.TINY_32, prec)
    assert 0 < n < 64 << 20


def test_slab_memory_does_not_grow_with_the_scan():
    small = B.oam_model_bytes(configs.scaled(configs.VOLUME_200, px=100, py=100), B.OAM_PREC_FP32)
    full = B.oam_model_bytes(configs.VOLUME_200, B.OAM_PREC_FP32)
    assert small == full
    # the tensor-core form adds per-position staging (input copy, per-|b| partial sums)
    tc_small = B.oam_model_bytes(configs.scaled(configs.VOLUME_200, px=100, py=100), B.OAM_PREC_BF16X3)
    tc_full = B.oam_model_bytes(configs.VOLUME_200, B.OAM_PREC_BF16X3)
    assert tc_full > tc_small > full


def test_grows_with_the_window_and_depths():
    base = B.oam_model_bytes(configs.TINY_32, B.OAM_PREC_FP32)
    assert B.oam_model_bytes(configs.scaled(configs.TINY_32, win=15), B.OAM_PREC_FP32) > base
    assert B.oam_model_bytes(configs.scaled(configs.TINY_32, nz=96, nt=256, z0_rel_m=-300e-6), B.OAM_PREC_FP32) > base


def test_errors_match_the_build():
    with pytest.raises(B.OamError) as e:
        B.oam_model_bytes(configs.scaled(configs.TINY_32, win=10), B.OAM_PREC_FP32)
    assert e.value.code == B.OAM_ERR_INVALID_ARG
    with pytest.raises(B.OamError) as e:
        B.oam_model_bytes(configs.scaled(configs.TINY_32, nt=100), B.OAM_PREC_FP32)
    assert e.value.code == B.OAM_ERR_WINDOW
    with pytest.raises(B.OamError) as e:  # lateral-FFT transforms are at most 2048 points
        B.oam_model_bytes(configs.scaled(configs.TINY_32, px=2100), B.OAM_PREC_FFT)
    assert e.value.code == B.OAM_ERR_UNSUPPORTED
    with pytest.raises(B.OamError) as e:
        B.oam_model_bytes(configs.TINY_32, 7)
    assert e.value.code == B.OAM_ERR_INVALID_ARG


def test_server_footprint_adds_buffers_and_workspace():
    cfg = configs.TINY_32
    sn, g, e = B.structs_from_config(cfg)
    vol = cfg["px"] * cfg["py"] * cfg["nz"] * 4
    sig = cfg["px"] * cfg["py"] * cfg["nt"] * 4
    for prec in PRECS:
        need = B.oam_request_footprint(prec, sn, g, e)
        assert need >= B.oam_model_bytes(cfg, prec) + 3 * sig + 5 * vol
