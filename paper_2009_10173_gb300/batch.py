"""Batched reconstructions: many uneven volumes in one CUDA-graph launch.

    python -m paper_2009_10173_gb300.batch --jobs 16 --reps 3

builds the batched workload (seeded sensors, sizes and vessel phantoms),
autotunes each model's tensor-core tile shape (position tiling, fold warps
and item-ring depth per direction), records one graph with every
job's LSQR and FISTA on its own branch, and times graph launches.  Marshalling
only: all arithmetic runs in liboam.so.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import binding as B
from . import configs, inputs
from .model import Model


def build_model(cfg, precision):
    """Model for cfg, moving to the next sample count if arrivals miss the window."""
    while True:
        try:
            return cfg, Model(cfg, precision=precision)
        except B.OamError as e:
            if e.code != B.OAM_ERR_WINDOW:
                raise
            nxt = configs.next_nt(cfg)
            if nxt is None:
                raise
            cfg = nxt


class Batch:
    """Jobs (model, device signals, two images, workspace) bound to one graph."""

    def __init__(self, cfgs, signals, precision=B.OAM_PREC_BF16X3, autotune=True):
        self.jobs = []
        self.handle = B.oam_batch_create(len(cfgs))
        for j, (cfg, s) in enumerate(zip(cfgs, signals)):
            m = cfg["_model"]
            if autotune:
                B.oam_model_autotune(m.handle, 2)
            x2, x1 = m.empty_volume(), m.empty_volume()
            nbytes = max(B.oam_solver_work_bytes(m.handle, 0), B.oam_solver_work_bytes(m.handle, 1))
            raw = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            work = raw[(-raw.data_ptr()) % 256:][:nbytes]
            lo = B.OamLsqrOpts(cfg["lsqr_iters"], 0.0)
            fo = B.OamFistaOpts(cfg["fista_iters"], cfg["power_iters"], 1, 0, -1.0, cfg["lambda_rel"], 0.0, None)
            B.oam_batch_set_job(self.handle, j, m.handle, s, x2, x1, lo, fo, work)
            self.jobs.append(dict(cfg=cfg, model=m, s=s, x2=x2, x1=x1, work=work, raw=raw))

    def run(self, stream=None):
        B.oam_batch_run(self.handle, stream)

    def close(self):
        if self.handle:
            B.oam_batch_free(self.handle)
            self.handle = None
        for j in self.jobs:
            j["model"].close()


def prepare(cfgs, precision=B.OAM_PREC_BF16X3):
    """Build models and synthetic noisy signals (vessel phantom, 20 dB) per job."""
    out_cfgs, signals = [], []
    for cfg in cfgs:
        cfg, m = build_model(cfg, precision)
        H = inputs.phantom(cfg, cfg.get("seed", 0), kind="vessels", count=10)
        clean = m.forward(torch.from_numpy(H.astype(np.float32)).cuda()).cpu().numpy()
        s = torch.from_numpy(inputs.add_noise(clean, 20.0, cfg.get("seed", 0) + 10 ** 6).astype(np.float32)).cuda()
        cfg = dict(cfg, _model=m)
        out_cfgs.append(cfg)
        signals.append(s)
    return out_cfgs, signals


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--jobs", type=int, default=16)
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=1)
    p.add_argument("--prec", default="bf16x3", choices=["bf16x3", "fft", "fp32"],
                   help="operator form: split-BF16 tensor cores, FP32 lateral-FFT form, or plain FP32")
    a = p.parse_args()
    prec = {"bf16x3": B.OAM_PREC_BF16X3, "fft": B.OAM_PREC_FFT, "fp32": B.OAM_PREC_FP32}[a.prec]
    cfgs, signals = prepare(configs.batch_workload(a.jobs), prec)
    batch = Batch(cfgs, signals, precision=prec, autotune=(prec == B.OAM_PREC_BF16X3))
    for _ in range(a.warmup):
        batch.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        batch.run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    flops = sum((1 + 2 * c["lsqr_iters"] + 2 * c["power_iters"] + 1 + 2 * c["fista_iters"]) *
                c["_model"].info.flops_per_op for c in cfgs)
    print(json.dumps({"workload": f"batch of {a.jobs} uneven reconstructions (30 LSQR + 50 FISTA each)",
                      "prec": a.prec,
                      "ms_per_batch": ms, "volumes_per_s": a.jobs / (ms / 1e3),
                      "op_tflops_algorithmic": flops / (ms * 1e-3) / 1e12,
                      "jobs": [[c["py"], c["px"], c["nz"], c["nt"], round(c["focal_m"] * 1e3, 2),
                                round(c["aperture_m"] * 1e3, 2)] for c in cfgs],
                      "tiles": [[B.oam_model_get_tiles(c["_model"].handle, d) + (B.oam_model_get_tiling(c["_model"].handle, d),)
                                 for d in (0, 1)] for c in cfgs]
                      if prec == B.OAM_PREC_BF16X3 else None,
                      "tiles_fields": "per job and direction (forward, adjoint): fold warps, item-ring depth, "
                                      "position tiling (1 padded grid, 2 scan grid)"}))
    batch.close()


if __name__ == "__main__":
    main()
