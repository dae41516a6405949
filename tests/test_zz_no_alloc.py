"""oam_lsqr_noalloc: LSQR for callers that cannot allocate device memory.

Such callers (a host that reserves all device memory for its own allocator,
or a latency-critical loop that cannot take an allocation's implicit
synchronisation) get the same LSQR as oam_lsqr on a fixed workspace in the
library's static device memory.  This test calls the new entry point through
the C ABI twice in a row and checks that each result equals oam_lsqr on the
same input bit for bit (both run the same kernels in the same order on the
same workspace layout, so a wrong offset or stale workspace contents would
show), and that the device's free memory does not change across the calls.
It sits in a file that pytest collects last and works alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest
import torch

from paper_2009_10173_gb300 import binding as B
from paper_2009_10173_gb300 import configs, inputs
from paper_2009_10173_gb300.model import Model

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [B.OAM_PREC_FP32, B.OAM_PREC_BF16X3, B.OAM_PREC_FFT])
def test_noalloc_lsqr_matches_lsqr_twice(prec):
    cfg = configs.TINY_32
    m = Model(cfg, precision=prec)
    s = torch.from_numpy(inputs.gaussian(m.sig_shape, 2024).astype(np.float32)).cuda()
    ref, info_ref = m.lsqr(s, 10)
    opts = B.OamLsqrOpts(10, 0.0)
    xs = [torch.full(m.vol_shape, float("nan"), device="cuda") for _ in range(3)]
    B.oam_lsqr_noalloc(m.handle, s, xs[2], opts)  # warm-up: module and address look-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for x in xs[:2]:
        info = B.oam_lsqr_noalloc(m.handle, s, x, opts)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert info.iters_done == info_ref.iters_done == 10
        assert torch.equal(x, ref)
        assert info.rnorm == info_ref.rnorm and info.arnorm == info_ref.arnorm
    m.close()


def test_noalloc_lsqr_rejects_problems_beyond_the_static_workspace():
    cfg = configs.scaled(configs.TINY_32, px=160, py=160)  # LSQR workspace > 32 MiB
    m = Model(cfg, precision=B.OAM_PREC_FP32)
    assert B.oam_solver_work_bytes(m.handle, 0) > 32 << 20
    s = torch.zeros(m.sig_shape, device="cuda")
    x = torch.zeros(m.vol_shape, device="cuda")
    with pytest.raises(B.OamError) as e:
        B.oam_lsqr_noalloc(m.handle, s, x, B.OamLsqrOpts(2, 0.0))
    assert e.value.code == B.OAM_ERR_INVALID_ARG
    m.close()
