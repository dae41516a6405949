"""The library's band-pass design (host code, no GPU) against the oracle's.

``oam_bandpass_taps`` runs on the host only, so it is checked here without a
GPU: its taps equal the oracle's windowed-sinc design (Results: signals and
model filtered to 0.5-80 MHz, 1-120 MHz in vivo) to rounding, and it rejects
the bands and lengths the header rules out.
"""
import numpy as np
import pytest

from oracle import bandpass as bp
from paper_2009_10173_gb300 import binding as B
from paper_2009_10173_gb300 import build_lib

FS = 250e6


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib.build()


@pytest.mark.parametrize("f_lo,f_hi,L", [(0.5e6, 80e6, 511), (1e6, 120e6, 511), (0.0, FS / 2, 16),
                                         (5e6, 60e6, 0), (2e6, 70e6, B.OAM_MAX_FIR_HALF)])
def test_design_matches_oracle(f_lo, f_hi, L):
    got = np.array(B.oam_bandpass_taps(f_lo, f_hi, FS, L))
    want = bp.bandpass_taps(f_lo, f_hi, FS, L)
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 1e-15


@pytest.mark.parametrize("args", [(80e6, 0.5e6, FS, 10), (0.5e6, 130e6, FS, 10), (-1.0, 80e6, FS, 10),
                                  (0.5e6, 80e6, FS, -1), (0.5e6, 80e6, FS, B.OAM_MAX_FIR_HALF + 1),
                                  (0.5e6, 80e6, 0.0, 10), (5e6, 5e6, FS, 10)])
def test_design_rejects_bad_arguments(args):
    with pytest.raises(B.OamError) as e:
        B.oam_bandpass_taps(*args)
    assert e.value.code == B.OAM_ERR_INVALID_ARG
