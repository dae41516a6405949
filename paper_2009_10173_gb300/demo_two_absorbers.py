"""Two absorbers below the acoustic diffraction limit (Methods, Numerical
simulations, second simulation; Results, Fig. 2a,b).

    python -m paper_2009_10173_gb300.demo_two_absorbers --sep 60 40

Two truncated paraboloids of 20 um diameter at the focal depth, separated
along x by each given distance, in a 200 x 200 x 150 um^3 field of view
sampled at 5 um; the AR-OAM set-up's sensor (7 mm focal distance, NA 0.43,
0.9 mm central hole, 1200 surface patches) at 250 MS/s; the model built with
the paper's discretisation of Eq. 1 (trilinear voxels, finite-difference
derivative; OAM_DISC_TRILINEAR) and a broadband EIR (-6 dB from 0 to
80 MHz), so that the band-pass filter of the simulation, 0.5-80 MHz on the
signals and on the model, sets the detection band.  The signals are that
model applied to the absorbers (the paper computed them analytically),
normalised to their maximum, without noise.  Both reconstructions of the
paper run on them: MB-L2 (LSQR) and MB-L1 (non-negative FISTA).

Printed per separation and method, from the lateral profile through both
centres at the focal depth: the two peak values, the value midway between
the centres relative to the smaller peak ("dip"; two absorbers count as
resolved when the dip is below 0.81, the Rayleigh criterion's dip), and the
profile's full width at half maximum of one absorber alone.  These are
demonstration numbers on synthetic data; the paper's (FWHM 13 um MB-L1 vs
41 um MB-L2; 40 um resolved by MB-L1 only) are context, not a target.
Marshalling only: all arithmetic runs in liboam.so.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import binding as B
from . import configs, inputs
from .model import Model

STEP = 5e-6
SENSOR = dict(focal_m=7e-3, aperture_m=2 * 7e-3 * 0.43, hole_m=0.9e-3, c_mps=1500.0, n_patches=1200)
EIR_BROAD = dict(fc_hz=40e6, frac_bw=2.0, trunc_sigma=5.0)
DIAMETER = 20e-6
BAND = (0.5e6, 80e6)
FIR_HALF = 511


def config(precision_window=79):
    """40 x 40 scan at 5 um, 40 x 40 x 30 voxels centred on the focus, 256
    samples, a window that covers every voxel-position pair of the field."""
    return dict(**SENSOR, **EIR_BROAD, px=40, py=40, nz=30, nt=256, win=precision_window, dx_m=STEP, dy_m=STEP,
                dz_m=STEP, z0_rel_m=-15 * STEP, fs_hz=250e6, t0_s=float("nan"))


def profile_metrics(x, sep_um, centre_x):
    """Peak values, midway dip and FWHM on the lateral profile x (sampled at STEP)."""
    pos = np.arange(len(x)) * STEP
    i1 = int(round((centre_x - 0.5 * sep_um * 1e-6) / STEP))
    i2 = int(round((centre_x + 0.5 * sep_um * 1e-6) / STEP))
    im = int(round(centre_x / STEP))
    p1, p2 = float(x[max(0, i1 - 1):i1 + 2].max()), float(x[max(0, i2 - 1):i2 + 2].max())
    return {"peaks": [p1, p2], "dip": float(x[im] / max(min(p1, p2), 1e-30)), "positions_um": [pos[i1] * 1e6,
                                                                                                pos[i2] * 1e6]}


def fwhm_um(x):
    """Full width at half maximum of a single-peaked profile (linear interpolation)."""
    i = int(np.argmax(x))
    half = 0.5 * x[i]
    lo = i
    while lo > 0 and x[lo - 1] > half:
        lo -= 1
    hi = i
    while hi < len(x) - 1 and x[hi + 1] > half:
        hi += 1
    left = lo - 1 + (half - x[lo - 1]) / (x[lo] - x[lo - 1]) if lo > 0 else lo
    right = hi + (x[hi] - half) / (x[hi] - x[hi + 1]) if hi < len(x) - 1 else hi
    return float((right - left) * STEP * 1e6)


def reconstruct(m, s, lsqr_iters, fista_iters, lambda_rel):
    """MB-L2 and MB-L1 images of the filtered signals, with each solve's device time (ms)."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    s_f = m.filter_signals(s)
    ev[0].record()
    x2, _ = m.lsqr(s_f, lsqr_iters)
    ev[1].record()
    x1, _ = m.fista(s_f, fista_iters, power_iters=30, lambda_rel=lambda_rel, nonneg=True)
    ev[2].record()
    torch.cuda.synchronize()
    return x2.cpu().numpy(), x1.cpu().numpy(), (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]))


def run(separations_um=(60, 40), precision=B.OAM_PREC_FFT, lsqr_iters=50, fista_iters=400, lambda_rel=1e-3):
    cfg = config()
    torch.cuda.synchronize()
    t_build = time.perf_counter()
    m = Model(cfg, precision=precision, discretisation=B.OAM_DISC_TRILINEAR)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    m.set_filter(B.oam_bandpass_taps(BAND[0], BAND[1], cfg["fs_hz"], FIR_HALF))
    cx, cy, cz = 20 * STEP, 20 * STEP, 0.0
    j, k = 20, 15  # profile row (y = cy) and focal depth (z = 0)
    out = {"workload": "two 20 um truncated paraboloids at the focus, 200x200x150 um^3 at 5 um, "
                       "F 7 mm / NA 0.43 sensor, 0.5-80 MHz band-pass, discretised model (trilinear voxels, "
                       "finite-difference derivative), noiseless normalised signals",
           "lsqr_iters": lsqr_iters, "fista_iters": fista_iters, "lambda_rel": lambda_rel,
           "model_build_s": t_build, "model_bytes": m.info.device_bytes, "results": {}}
    single = inputs.paraboloids(cfg, [(cx, cy, cz)], DIAMETER)
    for name, H in [("single", single)] + [(f"{float(sep):.1f}um", inputs.paraboloids(
            cfg, [(cx - 0.5 * sep * 1e-6, cy, cz), (cx + 0.5 * sep * 1e-6, cy, cz)], DIAMETER))
            for sep in separations_um]:
        s = m.forward(torch.from_numpy(H.astype(np.float32)).cuda())  # F A H: the filtered model's signals
        s = s / s.abs().max()
        x2, x1, ms = reconstruct(m, s, lsqr_iters, fista_iters, lambda_rel)
        res = {"lsqr_ms": ms[0], "fista_ms": ms[1]}
        for method, x in (("MB-L2", x2), ("MB-L1", x1)):
            prof = x[j, :, k]
            if name == "single":
                res[method] = {"fwhm_um": fwhm_um(prof)}
            else:
                sep = float(name[:-2])
                met = profile_metrics(prof, sep, cx)
                met["resolved"] = bool(met["dip"] < 0.81)
                res[method] = met
        out["results"][name] = res
    m.close()
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--sep", type=float, nargs="+", default=[60.0, 40.0])
    p.add_argument("--prec", default="fft", choices=["fft", "bf16x3", "fp32"])
    p.add_argument("--lsqr-iters", type=int, default=50)
    p.add_argument("--fista-iters", type=int, default=400)
    p.add_argument("--lambda-rel", type=float, default=1e-3)
    a = p.parse_args()
    prec = {"fft": B.OAM_PREC_FFT, "bf16x3": B.OAM_PREC_BF16X3, "fp32": B.OAM_PREC_FP32}[a.prec]
    print(json.dumps(run(a.sep, prec, a.lsqr_iters, a.fista_iters, a.lambda_rel)))


if __name__ == "__main__":
    main()
