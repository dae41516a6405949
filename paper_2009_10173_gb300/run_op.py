"""Run one operator (or solver) repeatedly on a synthetic workload.

A small command-line driver for profiling and timing through the C-ABI:

    python -m paper_2009_10173_gb300.run_op --op forward --prec bf16x3 \\
        --px 96 --py 96 --nz 300 --nt 1024 --win 61 --reps 3

prints one JSON line with the mean CUDA-event time per call.  ``--op filter``
times the band-pass filter on the signals (one k_fir_lines launch per call,
``--band`` and ``--filter-half`` set the FIR); ``--op sweep`` times an LSQR
sweep over ``--damps`` Tikhonov weights.
"""
import argparse
import json

import torch

from . import binding as B
from . import configs, inputs
from .model import Model


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--op", default="forward", choices=["forward", "adjoint", "lsqr", "fista", "filter", "sweep"])
    p.add_argument("--band", type=float, nargs=2, default=[0.5e6, 80e6], metavar=("F_LO", "F_HI"))
    p.add_argument("--filter-half", type=int, default=511)
    p.add_argument("--damps", type=int, default=8)
    p.add_argument("--prec", default="bf16x3", choices=["fp32", "bf16x3", "fft"])
    p.add_argument("--workload", default="volume_200x200x300", choices=sorted(configs.WORKLOADS))
    for k in ("px", "py", "nz", "nt", "win", "iters"):
        p.add_argument(f"--{k}", type=int, default=None)
    p.add_argument("--fold-warps", type=int, default=None, help="split-BF16 kernels: fold warps (4, 8, 16)")
    p.add_argument("--ring", type=int, default=0, help="split-BF16 kernels: item-ring depth (0 = deepest)")
    p.add_argument("--tiling", type=int, default=None, help="split-BF16 kernels: 0 auto, 1 padded grid, 2 scan grid")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=1)
    a = p.parse_args()
    over = {k: getattr(a, k) for k in ("px", "py", "nz", "nt", "win") if getattr(a, k) is not None}
    cfg = configs.scaled(configs.WORKLOADS[a.workload], **over)
    prec = {"bf16x3": B.OAM_PREC_BF16X3, "fp32": B.OAM_PREC_FP32, "fft": B.OAM_PREC_FFT}[a.prec]
    m = Model(cfg, precision=prec)
    if a.fold_warps is not None and prec == B.OAM_PREC_BF16X3:
        for d in (0, 1):
            B.oam_model_set_tiles(m.handle, d, a.fold_warps, a.ring)
    if a.tiling is not None and prec == B.OAM_PREC_BF16X3:
        for d in (0, 1):
            B.oam_model_set_tiling(m.handle, d, a.tiling)
    H = torch.from_numpy(inputs.phantom(cfg, 1, count=20)).float().cuda()
    s = m.forward(H)
    iters = a.iters or 5
    extra = {}
    if a.op == "filter":
        m.set_filter(B.oam_bandpass_taps(a.band[0], a.band[1], cfg["fs_hz"], a.filter_half))
        sf = torch.empty_like(s)
        extra = {"filter_size": m.info.filter_size, "bytes_per_call": 2 * s.numel() * 4}
    damps = [0.0] + [10.0 ** (-4 + 0.5 * i) for i in range(a.damps - 1)]
    run = {"forward": lambda: m.forward(H, out=s), "adjoint": lambda: m.adjoint(s),
           "lsqr": lambda: m.lsqr(s, iters, want_info=False),
           "fista": lambda: m.fista(s, iters, power_iters=2, want_info=False),
           "filter": lambda: m.filter_signals(s, out=sf),
           "sweep": lambda: m.lsqr_sweep(s, iters, damps, want_info=False)}[a.op]
    for _ in range(a.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    print(json.dumps({"op": a.op, "prec": a.prec, "grid": [cfg["py"], cfg["px"], cfg["nz"], cfg["nt"], cfg["win"]],
                      "ms_per_call": ms, "flops_per_op": m.info.flops_per_op,
                      "alg_tflops": m.info.flops_per_op / ms / 1e9 if a.op in ("forward", "adjoint") else None,
                      "model_bytes": m.info.device_bytes, "op_bytes": m.info.op_bytes,
                      "tiles": [B.oam_model_get_tiles(m.handle, d) + (B.oam_model_get_tiling(m.handle, d),) for d in (0, 1)]
                      if prec == B.OAM_PREC_BF16X3 else None, **extra}))
    m.close()


if __name__ == "__main__":
    main()
