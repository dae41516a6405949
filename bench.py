#!/usr/bin/env python
"""Benchmark: model-based AR-OAM reconstructions per second on GB300.

One step = one full reconstruction of a 200x200-position scan (200x200x300
voxels, 1024 samples, 61x61 slab window): build the model slab on the
device, run 50 LSQR iterations (MB-L2) and 100 FISTA iterations (MB-L1,
20 power iterations for L, lambda = 1e-3 max|A^T s|, non-negative) on
signals already resident in HBM.  value = volumes/s over all ranks.

Each rank reconstructs its own seeded volume (independent replicas, weak
scaling); there is no data-path collective.  ``--impl reference`` times the
FP64 CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LSQR/FISTA volumes/s and A+A^T TFLOP/s at <=1e-3 rel err vs FP64; p50/p99"
WORKLOAD = "volume_200x200x300"
LSQR_ITERS, FISTA_ITERS, POWER_ITERS, LAMBDA_REL = 50, 100, 20, 1e-3
# operator applications per step: LSQR 1 + 2*50; FISTA 2*20 power + 1 lambda + 2*100
OPS_PER_STEP = (1 + 2 * LSQR_ITERS) + (2 * POWER_ITERS + 1 + 2 * FISTA_ITERS)
FP32_LANES_PER_SM = 128
# DRAM bytes per launch of the tensor-core operator kernel (k_corr_fold) per
# direction on this workload: dram__bytes_read.sum + dram__bytes_write.sum of an
# ncu capture of the same kernel on a 96x96-position case of this workload (576
# blocks), scaled by blocks processed (2504 / 576; profiles/k_corr_fold_fwd_ and
# k_corr_fold_adj_96x96x300_win61.md).  Set to None when the kernel changes.
TC_TRAFFIC_BYTES = {"forward": (106.70e6 + 61.04e6) * 2504 / 576, "adjoint": (100.98e6 + 56.94e6) * 2504 / 576}
# DRAM bytes per application of the lateral-FFT form on this workload:
# dram__bytes_read.sum + dram__bytes_write.sum over the five launches of one
# forward, from an ncu capture of the full 200x200x300 workload (1.191 GB read,
# 0.250 GB written).  Set to None when those kernels change.
FFT_TRAFFIC_BYTES = 1.4414e9
# Band-pass filter along time: half length of the 0.5-80 MHz FIR, and the DRAM
# bytes of one application (ncu, profiles/k_fir_lines_200x200x1024_L511.md).
FIR_HALF = 511
FIR_TRAFFIC_BYTES = 163.96e6 + 120.01e6


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="auto", choices=["auto", "fp32", "bf16x3", "fft"],
                   help="operator form: auto = split-BF16 tensor cores when built; fft = FP32 lateral-FFT form")
    p.add_argument("--no-cpu-baseline", action="store_true",
                   help="skip the oracle leg: the timed FP64 CPU baseline and the FP64 accuracy references")
    p.add_argument("--no-accuracy", action="store_true",
                   help="skip the per-result error against the FP64 oracle (A, A^T, LSQR and FISTA images)")
    p.add_argument("--serve", action="store_true",
                   help="instead of the volume benchmark, run the served workload: Poisson arrivals at --rates, "
                        "--requests per rate, with the small requests' images checked against the FP64 oracle")
    p.add_argument("--rates", type=float, nargs="+", default=[2.0, 20.0])
    p.add_argument("--requests", type=int, default=500)
    p.add_argument("--pool", type=int, default=32)
    p.add_argument("--slots", type=int, default=8)
    p.add_argument("--no-forms", action="store_true",
                   help="skip the short measurements of the other operator form, the band-pass filter and "
                        "the Tikhonov sweep in the default run")
    return p.parse_args()


def config_dict(prec_name):
    from paper_2009_10173_gb300 import configs
    c = configs.VOLUME_200
    return {"workload": WORKLOAD, "scan": f"{c['py']}x{c['px']} positions at {c['dx_m']*1e6:g} um",
            "voxels": f"{c['py']}x{c['px']}x{c['nz']} ({c['dx_m']*1e6:g} um lateral, {c['dz_m']*1e6:g} um axial)",
            "nt": c["nt"], "fs_hz": c["fs_hz"], "slab_window": f"{c['win']}x{c['win']}",
            "sensor": "F=4 mm, D=3 mm, 2000 patches, EIR 30 MHz 100% BW", "lsqr_iters": LSQR_ITERS,
            "fista_iters": FISTA_ITERS, "power_iters": POWER_ITERS, "lambda_rel": LAMBDA_REL, "nonneg": True,
            "phantom": "seeded vessel tree + 50 microspheres, 20 dB Gaussian noise", "precision": prec_name,
            "step": "slab build + 50 LSQR + 100 FISTA (+20 power iterations) per volume",
            "l2": "inputs larger than L2 (164 MB signals) and a 256 MB L2 flush between timed steps",
            "parallelism": "independent replicas (one volume per GPU per step)"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (SM clock, reasons) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle sample
def oracle_sample():
    """Time the FP64 oracle on a bounded sample of the workload and scale it
    to one full reconstruction.  Sample: the full workload's depths (300) and
    samples (1024) on a 40x40-position scan with an 11x11 slab window; the
    slab cost scales per column, the operator cost per algorithmic flop."""
    import numpy as np

    import oracle
    from paper_2009_10173_gb300 import configs, inputs
    full = configs.VOLUME_200
    samp = configs.scaled(full, px=40, py=40, win=11)
    t = time.perf_counter()
    t0 = oracle.t0(samp)
    S = oracle.slab(samp, t0)
    t_slab = time.perf_counter() - t
    nnz_col = (S != 0).sum(axis=3).sum(axis=2)  # [win][win]
    R = 5
    flops = 0.0
    for b in range(-R, R + 1):
        for a in range(-R, R + 1):
            flops += 2.0 * (40 - abs(b)) * (40 - abs(a)) * nnz_col[b + R, a + R]
    H = inputs.phantom(samp, 1, kind="spheres", count=8)
    t = time.perf_counter()
    s = oracle.forward(S, H)
    oracle.adjoint(S, s)
    t_ops = time.perf_counter() - t
    rate = 2 * flops / t_ops  # flop/s of the direct FP64 operators
    cols_full = full["win"] ** 2 * full["nz"]
    cols_samp = samp["win"] ** 2 * samp["nz"]
    slab_full = t_slab * cols_full / cols_samp
    return dict(t_slab=t_slab, t_ops=t_ops, rate=rate, slab_full=slab_full, flops_sample=flops)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def cpu_baseline_entry(flops_per_op):
    m = oracle_sample()
    per_volume = m["slab_full"] + OPS_PER_STEP * flops_per_op / m["rate"]
    return {"value": 1.0 / per_volume, "unit": "volumes/s", "cores": int(os.environ.get("OMP_NUM_THREADS", cpu_cores())),
            "kind": "oracle",
            "sample": (f"FP64 oracle: slab of a 40x40-position, 11x11-window, 300-depth, 1024-sample grid "
                       f"({m['t_slab']:.1f} s) and one direct A + A^T on it ({m['t_ops']:.1f} s, "
                       f"{m['rate']/1e9:.2f} GFLOP/s); scaled to the full volume by slab columns "
                       f"({m['slab_full']:.0f} s) and by algorithmic flops ({OPS_PER_STEP} operator "
                       f"applications of {flops_per_op:.3e} flop)"),
            "seconds_per_volume": per_volume}


# ---------------------------------------------------------------- oracle leg: FP64 references
# The oracle leg runs the FP64 oracle on the host cores: the timed CPU
# baseline above, and the FP64 references of this workload's results (A H,
# A^T s, the LSQR and FISTA images) that every operator form is compared with.
# The references take minutes of host time, so they run in a spawned process
# (started before the first CUDA call) while the GPU legs are timed; the
# CPU baseline is timed afterwards, on idle cores.
def _reference_proc(workdir, threads):
    os.environ["OMP_NUM_THREADS"] = str(threads)  # read when the oracle library loads
    import numpy as np

    from oracle import headline
    from paper_2009_10173_gb300 import configs

    def on_signals(s32, H32):
        np.save(os.path.join(workdir, "s32.npy"), s32)
        np.save(os.path.join(workdir, "H32.npy"), H32)
        os.replace(os.path.join(workdir, "s32.npy"), os.path.join(workdir, "signals.npy"))

    try:
        r = headline.reference(configs.VOLUME_200, seed=1, n_spheres=50, snr_db=20.0, lsqr_iters=LSQR_ITERS,
                               fista_iters=FISTA_ITERS, power_iters=POWER_ITERS, lambda_rel=LAMBDA_REL,
                               v0_seed=7, on_signals=on_signals)
        np.savez(os.path.join(workdir, "ref_tmp.npz"), AH=r["AH"], ATs=r["ATs"], x_l2=r["x_l2"], x_l1=r["x_l1"],
                 L=r["L"], lam=r["lam"], seconds=json.dumps(r["seconds"]), threads=threads)
        os.replace(os.path.join(workdir, "ref_tmp.npz"), os.path.join(workdir, "ref.npz"))
    except Exception as e:  # reported in the bench line
        with open(os.path.join(workdir, "error.txt"), "w") as f:
            f.write(repr(e))


class AccuracyLeg:
    """FP64 references in a spawned process; device results compared at the end."""

    def __init__(self):
        import multiprocessing as mp
        import tempfile
        self.dir = tempfile.mkdtemp(prefix="oam_ref_")
        self.threads = max(1, cpu_cores() - 2)  # two cores stay with the GPU process
        self.proc = mp.get_context("spawn").Process(target=_reference_proc, args=(self.dir, self.threads),
                                                    daemon=True)
        self.t0 = time.perf_counter()
        self.proc.start()
        self.results = {}

    def _wait_for(self, name, timeout_s):
        path = os.path.join(self.dir, name)
        t = time.perf_counter()
        while not os.path.exists(path):
            if os.path.exists(os.path.join(self.dir, "error.txt")) or not self.proc.is_alive() and \
                    not os.path.exists(path):
                return None
            if time.perf_counter() - t > timeout_s:
                return None
            time.sleep(0.5)
        return path

    def run_device(self, forms, make_model):
        """Device results of each form on the oracle's signals (FP32 in, FP32 out)."""
        import numpy as np
        import torch
        if self._wait_for("signals.npy", 1800) is None:
            return
        s32 = np.load(os.path.join(self.dir, "signals.npy"))
        H32 = np.load(os.path.join(self.dir, "H32.npy"))
        s = torch.from_numpy(s32).cuda()
        H = torch.from_numpy(H32).cuda()
        from paper_2009_10173_gb300 import inputs
        v0 = torch.from_numpy(inputs.gaussian(H32.shape, 7).astype(np.float32)).cuda()
        for name, prec in forms:
            m = make_model(prec)
            out = {"A": m.forward(H).cpu().numpy(), "AT": m.adjoint(s).cpu().numpy()}
            x2, _ = m.lsqr(s, LSQR_ITERS)
            out["lsqr_image"] = x2.cpu().numpy()
            x1, inf = m.fista(s, FISTA_ITERS, power_iters=POWER_ITERS, lambda_rel=LAMBDA_REL, nonneg=True, v0=v0)
            out["fista_image"] = x1.cpu().numpy()
            out["L"], out["lambda"] = inf.L, inf.lambda_
            m.close()
            self.results[name] = out

    def finish(self):
        import numpy as np
        path = self._wait_for("ref.npz", 3600)
        self.proc.join(timeout=60)
        if path is None:
            err = "reference process failed"
            ep = os.path.join(self.dir, "error.txt")
            if os.path.exists(ep):
                err = open(ep).read().strip()
            return {"error": err}
        ref = np.load(path)

        def rel(a, b):
            a = np.asarray(a, np.float64)
            return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))

        out = {"reference": "FP64 oracle (lateral-FFT restatement with the slab spectrum computed once, pinned to "
                            "the direct form at 1e-12) on the host cores, same seeded FP32 signals",
               "oracle_threads": int(ref["threads"]), "oracle_seconds": json.loads(str(ref["seconds"])),
               "wall_s": time.perf_counter() - self.t0, "tolerance": {"A, A^T fp32/fft": 1e-5,
                                                                       "A, A^T bf16x3": 1e-4, "images": 1e-3}}
        for name, r in self.results.items():
            out[name] = {"A": rel(r["A"], ref["AH"]), "AT": rel(r["AT"], ref["ATs"]),
                         "lsqr_image": rel(r["lsqr_image"], ref["x_l2"]),
                         "fista_image": rel(r["fista_image"], ref["x_l1"]),
                         "L": abs(r["L"] - float(ref["L"])) / float(ref["L"]),
                         "lambda": abs(r["lambda"] - float(ref["lam"])) / float(ref["lam"])}
        import shutil
        shutil.rmtree(self.dir, ignore_errors=True)
        return out


# ---------------------------------------------------------------- served workload
SERVE_ITERS = (30, 50, 20)  # LSQR, FISTA, power iterations per served request


def _serve_reference_proc(workdir, threads, cfgs):
    """Oracle leg of the served workload: for each small prepared request, the
    signals (FP64 oracle's A on the request's phantom, 20 dB noise) and its
    FP64 LSQR and FISTA images."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    import numpy as np

    import oracle
    from oracle import solvers
    from paper_2009_10173_gb300 import configs, inputs
    try:
        sps = {}
        for j, cfg in cfgs:
            while True:  # the same sample-count fallback as the library's window check
                try:
                    oracle.t0(cfg)
                    break
                except oracle.OracleError:
                    cfg = configs.next_nt(cfg)
                    if cfg is None:
                        raise
            sp = oracle.Spectral(cfg, symmetric=True)
            H = inputs.phantom(cfg, cfg.get("seed", 0), kind="vessels", count=10)
            s32 = inputs.add_noise(sp.forward(H.astype(np.float32).astype(np.float64)), 20.0,
                                   cfg.get("seed", 0) + 10 ** 6).astype(np.float32)
            np.save(os.path.join(workdir, f"sig{j}_tmp.npy"), s32)
            os.replace(os.path.join(workdir, f"sig{j}_tmp.npy"), os.path.join(workdir, f"sig{j}.npy"))
            with open(os.path.join(workdir, f"nt{j}.txt"), "w") as f:
                f.write(str(cfg["nt"]))
            sps[j] = (sp, s32)
        for j, (sp, s32) in sps.items():
            sd = s32.astype(np.float64)
            x2, _ = solvers.lsqr(sp.forward, sp.adjoint, sd, SERVE_ITERS[0])
            x1, _ = solvers.mb_l1(sp.forward, sp.adjoint, sd, SERVE_ITERS[1], SERVE_ITERS[2],
                                  np.ones(x2.shape), lambda_rel=LAMBDA_REL, nonneg=True)
            np.savez(os.path.join(workdir, f"ref{j}_tmp.npz"), x2=x2, x1=x1)
            os.replace(os.path.join(workdir, f"ref{j}_tmp.npz"), os.path.join(workdir, f"ref{j}.npz"))
    except Exception as e:
        with open(os.path.join(workdir, "error.txt"), "w") as f:
            f.write(repr(e))


def run_serve(args):
    """Served workload: requests drawn from a pool of prepared
    instances (sizes as the batched workload plus occasional 200x200x300
    volumes), submitted at Poisson arrival times to one request server with a
    150 GB device-memory budget.  Requests on small instances (64x64 scans,
    <= 192 depths) carry signals made by the FP64 oracle and every one of
    them is compared with the oracle's FP64 LSQR and FISTA images."""
    import multiprocessing as mp
    import tempfile

    import numpy as np

    from paper_2009_10173_gb300 import configs
    cfgs = [configs.served_request(2000 + j) for j in range(args.pool)]
    from paper_2009_10173_gb300.serve import is_small
    small = [(j, c) for j, c in enumerate(cfgs) if is_small(c)]
    workdir = tempfile.mkdtemp(prefix="oam_serve_ref_")
    proc = None
    if small and not args.no_cpu_baseline:
        proc = mp.get_context("spawn").Process(target=_serve_reference_proc,
                                               args=(workdir, max(1, cpu_cores() - 2), small), daemon=True)
        proc.start()

    import torch

    from paper_2009_10173_gb300 import binding as B
    from paper_2009_10173_gb300 import serve
    torch.cuda.set_device(0)
    prec = {"auto": B.OAM_PREC_BF16X3, "bf16x3": B.OAM_PREC_BF16X3, "fft": B.OAM_PREC_FFT,
            "fp32": B.OAM_PREC_FP32}[args.prec]

    def wait_file(name, timeout_s=3600):
        t = time.perf_counter()
        path = os.path.join(workdir, name)
        while not os.path.exists(path):
            if os.path.exists(os.path.join(workdir, "error.txt")) or time.perf_counter() - t > timeout_s or \
                    (proc is not None and not proc.is_alive() and not os.path.exists(path)):
                return None
            time.sleep(0.5)
        return path

    pool, checked_pool = [], set()
    for j, cfg in enumerate(cfgs):
        sig = None
        if proc is not None and is_small(cfg):
            pth = wait_file(f"sig{j}.npy")
            final = serve.final_config(cfg, prec)
            if pth is not None and open(os.path.join(workdir, f"nt{j}.txt")).read().strip() == str(final["nt"]):
                sig = np.load(pth)
                checked_pool.add(j)
        pool.append(serve.Instance(cfg, prec, signals=sig))

    refs = {}

    def check(j, x2, x1):
        if j not in checked_pool:
            return None
        if j not in refs:
            pth = wait_file(f"ref{j}.npz")
            if pth is None:
                return None
            refs[j] = np.load(pth)
        r = refs[j]

        def rel(a, b):
            a = np.asarray(a, np.float64)
            return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
        return {"rel_err_lsqr": rel(x2.numpy(), r["x2"]), "rel_err_fista": rel(x1.numpy(), r["x1"])}

    results = []
    for k, rate in enumerate(args.rates):
        server = serve.make_server(150e9, args.slots, precision=prec, lsqr_iters=SERVE_ITERS[0],
                                   fista_iters=SERVE_ITERS[1], power_iters=SERVE_ITERS[2], lambda_rel=LAMBDA_REL)
        res = serve.run_rate(server, pool, rate, args.requests, seed=3000 + k, check=check, check_picks=checked_pool)
        B.oam_server_stop(server)
        results.append(res)
    err = None
    if os.path.exists(os.path.join(workdir, "error.txt")):
        err = open(os.path.join(workdir, "error.txt")).read().strip()
    import shutil
    shutil.rmtree(workdir, ignore_errors=True)
    line = {"metric": "served reconstructions: volumes/s and p50/p99 latency", "unit": "volumes/s",
            "value": max(r["volumes_per_s"] for r in results), "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16" if prec == B.OAM_PREC_BF16X3 else "f32", "data": "synthetic",
            "config": {"workload": "served: Poisson arrivals, sizes as the batched workload (scan 64-256^2, "
                                   "128-384 depths, 512-1024 samples, seeded sensors) plus 5 % 200x200x300 "
                                   "volumes; 30 LSQR + 50 FISTA (+20 power) each",
                       "pool_instances": args.pool, "slots": args.slots, "budget_gb": 150,
                       "oracle_checked_instances": sorted(checked_pool),
                       "check": "every request on a small instance (64x64 scan, <= 192 depths) against the "
                                "FP64 oracle's LSQR and FISTA images of the same oracle-made signals"},
            "rates": results}
    if err:
        line["oracle_error"] = err
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2009_10173_gb300 import configs
    full = configs.VOLUME_200
    times, vals = [], []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        m = oracle_sample()
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
            vals.append(m)
    # Full-size algorithmic flops: the band width grows with lateral offset, so
    # take the mean nonzero count of a spread of full-size oracle slab columns.
    R = 30
    t0 = oracle.t0(full)
    widths = []
    for (b, a) in ((0, 0), (0, 10), (10, 10), (0, 20), (20, 20), (0, 30), (30, 30), (15, 25)):
        for k in (0, 100, 200, 299):
            widths.append(int((oracle.slab_column(full, b, a, k, t0) != 0).sum()))
    mean_w = float(np.mean(widths))
    flops_full = 0.0
    for b in range(-R, R + 1):
        for a in range(-R, R + 1):
            flops_full += 2.0 * (200 - abs(b)) * (200 - abs(a)) * full["nz"] * mean_w
    m = vals[-1]
    per_volume = m["slab_full"] + OPS_PER_STEP * flops_full / m["rate"]
    value = 1.0 / per_volume
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "volumes/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict("fp64 oracle (direct form)"),
            "cpu_baseline": {"value": value, "unit": "volumes/s", "kind": "oracle", "cores": cpu_cores(),
                             "sample": "each step: FP64 oracle slab (40x40 scan, 11x11 window, 300 depths, 1024 "
                                       "samples) plus one direct A and A^T on it, scaled to a full 200x200x300 "
                                       "reconstruction by slab columns and algorithmic flops"},
            "e2e": {"value": value, "unit": "volumes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "seconds_per_volume": per_volume}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, acc=None):
    import numpy as np
    import torch

    from paper_2009_10173_gb300 import binding as B
    from paper_2009_10173_gb300 import configs, inputs
    from paper_2009_10173_gb300.model import Model

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    cfg = configs.VOLUME_200

    def make_model(prec):
        return Model(cfg, precision=prec)

    # precision: the tensor-core form when it is built, else plain FP32
    if args.prec == "fp32":
        prec = B.OAM_PREC_FP32
    elif args.prec == "bf16x3":
        prec = B.OAM_PREC_BF16X3
    elif args.prec == "fft":
        prec = B.OAM_PREC_FFT
    else:
        try:
            make_model(B.OAM_PREC_BF16X3).close()
            prec = B.OAM_PREC_BF16X3
        except B.OamError as e:
            if e.code != B.OAM_ERR_UNSUPPORTED:
                raise
            prec = B.OAM_PREC_FP32
    prec_name = {B.OAM_PREC_FP32: "fp32 CUDA-core operators",
                 B.OAM_PREC_BF16X3: "split-BF16 (hi*hi+hi*lo+lo*hi) tcgen05 operators, FP32 accumulate",
                 B.OAM_PREC_FFT: "FP32 lateral-FFT form of the same operators (correlation theorem on a "
                                 "256x256 zero-padded grid, real slab spectrum per frequency orbit)"}[prec]

    # synthetic input for this rank: vessel tree + microspheres, clean signals by A, 20 dB noise
    from paper_2009_10173_gb300 import replicas
    seed = replicas.replica_seed(1, rank)
    H = inputs.phantom(cfg, seed, kind="vessels", count=50)
    m0 = make_model(B.OAM_PREC_FP32)
    clean = m0.forward(torch.from_numpy(H.astype(np.float32)).cuda()).cpu().numpy()
    info0 = m0.info
    m0.close()
    s_host = torch.from_numpy(inputs.add_noise(clean, 20.0, seed + 10 ** 6).astype(np.float32)).pin_memory()
    s_dev = s_host.cuda()
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    vol_bytes = int(np.prod(H.shape)) * 4

    keep = []

    def step(s_in, profile=False, form=None):
        m = make_model(prec if form is None else form)
        if profile:
            B.oam_profile_enable(m.handle, True)
        x2, _ = m.lsqr(s_in, LSQR_ITERS, want_info=False)
        x1, _ = m.fista(s_in, FISTA_ITERS, power_iters=POWER_ITERS, lambda_rel=LAMBDA_REL, nonneg=True,
                        want_info=False)
        return m, x2, x1

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    def other_form(form, steps=3, warmup=2):
        # the same reconstruction with another operator form, timed the same way
        for _ in range(warmup):
            mm, _, _ = step(s_dev, form=form)
            mm.close()
        barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        models = []
        evs[0].record()
        for i in range(steps):
            mm, _, _ = step(s_dev, profile=True, form=form)
            models.append(mm)
            flush.zero_()
            evs[i + 1].record()
        barrier()
        ms = evs[0].elapsed_time(evs[-1]) / steps
        pr = [B.oam_profile_read(mm.handle) for mm in models]
        inf = models[0].info
        for mm in models:
            mm.close()
        f_ms = sum(q.forward_ms for q in pr) / max(1, sum(q.forward_calls for q in pr))
        a_ms = sum(q.adjoint_ms for q in pr) / max(1, sum(q.adjoint_calls for q in pr))
        gbs = inf.op_bytes / (f_ms * 1e-3) / 1e9
        hbm = 6800.0
        try:
            hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", hbm)
        except Exception:
            pass
        return {"precision": "FP32 lateral-FFT form of the same operators (exact restatement)",
                "value": steps / (evs[0].elapsed_time(evs[-1]) / 1e3), "unit": "volumes/s", "ms_per_step": ms,
                "op_ms": {"forward": f_ms, "adjoint": a_ms},
                "roofline": {"bound": "hbm", "kernel": "forward (lateral-FFT form, 5 launches)", "achieved": gbs,
                             "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": FFT_TRAFFIC_BYTES,
                             "bytes_per_op": inf.op_bytes}}

    def extensions(reps=20, n_damps=8):
        # band-pass filter along time (0.5-80 MHz, 1023 taps: the second
        # simulation's band) and the Tikhonov sweep, on the lateral-FFT model
        mm = make_model(B.OAM_PREC_FFT)
        taps = B.oam_bandpass_taps(0.5e6, 80e6, cfg["fs_hz"], FIR_HALF)
        mm.set_filter(taps)
        sig = s_dev.clone()
        out = torch.empty_like(sig)
        for _ in range(3):
            mm.filter_signals(sig, out)
        barrier()
        ev_f = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev_f[0].record()
        for _ in range(reps):  # 2 x 164 MB per application, more than L2 holds
            mm.filter_signals(sig, out)
        ev_f[1].record()
        barrier()
        fir_ms = ev_f[0].elapsed_time(ev_f[1]) / reps
        fir_bytes = 2 * sig.numel() * 4
        hbm = 6800.0
        try:
            hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", hbm)
        except Exception:
            pass
        gbs = fir_bytes / (fir_ms * 1e-3) / 1e9
        # filtered MB-L2: signals through F, then LSQR with F A
        sf = mm.filter_signals(sig)
        _, inf = mm.lsqr(sf, LSQR_ITERS)
        damps = [0.0] + [inf.anorm * f for f in (1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1)][:n_damps - 1]
        mm.lsqr_sweep(sf, 2, damps, want_info=False)
        barrier()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        mm.lsqr_sweep(sf, LSQR_ITERS, damps, want_info=False)
        e[1].record()
        for d in damps:
            mm.lsqr(sf, LSQR_ITERS, damp=d, want_info=False)
        e[2].record()
        barrier()
        sweep_ms, single_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
        fir_size = mm.info.filter_size
        mm.close()
        return {"bandpass_filter": {"band_hz": [0.5e6, 80e6], "taps": 2 * FIR_HALF + 1, "transform": fir_size,
                                    "ms": fir_ms, "roofline": {"bound": "hbm", "kernel": "k_fir_lines",
                                                               "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                                               "frac": gbs / hbm, "bytes_per_launch": fir_bytes,
                                                               "traffic": FIR_TRAFFIC_BYTES}},
                "tikhonov_sweep": {"damps": len(damps), "iters": LSQR_ITERS, "filtered": True,
                                   "sweep_ms": sweep_ms, "separate_solves_ms": single_ms,
                                   "speedup": single_ms / sweep_ms,
                                   "solves_per_s": len(damps) / (sweep_ms / 1e3)}}

    for _ in range(args.warmup):
        m, _, _ = step(s_dev)
        m.close()
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = B.oam_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    t_wall = time.perf_counter()
    ev[0].record()
    for i in range(args.steps):
        m, x2, x1 = step(s_dev, profile=True)
        keep.append(m)
        flush.zero_()
        ev[i + 1].record()
    barrier()
    wall = time.perf_counter() - t_wall
    launches = B.oam_launch_count() - launches0 - 0  # the flush is a torch kernel, not counted
    clk = clocks.stop()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    elapsed_ms = ev[0].elapsed_time(ev[-1])
    prof = [B.oam_profile_read(mm.handle) for mm in keep]
    info = keep[0].info
    for mm in keep:
        mm.close()
    keep.clear()

    # end to end through the public API: pinned host signals in, both images out
    img2 = torch.empty(H.shape, dtype=torch.float32).pin_memory()
    img1 = torch.empty(H.shape, dtype=torch.float32).pin_memory()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        s_in = s_host.cuda(non_blocking=True)
        m, x2, x1 = step(s_in)
        img2.copy_(x2, non_blocking=True)
        img1.copy_(x1, non_blocking=True)
        torch.cuda.synchronize()
        m.close()
    e1.record()
    barrier()
    e2e_ms = e0.elapsed_time(e1)

    if dist:
        elapsed_ms, e2e_ms = replicas.max_over_ranks([elapsed_ms, e2e_ms], device="cuda")
    if rank != 0:
        return

    per_step = elapsed_ms / args.steps
    value = world * args.steps / (elapsed_ms / 1e3)
    fwd_ms = sum(p.forward_ms for p in prof) / max(1, sum(p.forward_calls for p in prof))
    adj_ms = sum(p.adjoint_ms for p in prof) / max(1, sum(p.adjoint_calls for p in prof))
    fwd_tot = sum(p.forward_ms for p in prof)
    adj_tot = sum(p.adjoint_ms for p in prof)
    dom, dom_ms = ("adjoint", adj_ms) if adj_tot >= fwd_tot else ("forward", fwd_ms)
    achieved = info.flops_per_op / (dom_ms * 1e-3) / 1e12
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    if prec == B.OAM_PREC_FFT:
        # bytes one application must move: the spectral slab, the input and the
        # output, and each transform stage's buffer written once and read once
        gbs = info.op_bytes / (dom_ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "kernel": f"{dom} (lateral-FFT form, 5 launches)", "achieved": gbs, "peak": peak,
                "unit": "GB/s", "frac": gbs / peak, "traffic": FFT_TRAFFIC_BYTES, "bytes_per_op": info.op_bytes,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    elif prec == B.OAM_PREC_FP32:
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": f"{dom} (FP32 FFMA)", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {mhz:g} MHz"}
    else:
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        roof = {"bound": "tensor", "kernel": f"{dom} (tcgen05 split-BF16, mirror-folded)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TC_TRAFFIC_BYTES[dom] if TC_TRAFFIC_BYTES else None,
                "executed_tflops": (info.exec_flops_adjoint if dom == "adjoint" else info.exec_flops_forward) /
                                   (dom_ms * 1e-3) / 1e12,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"}
    line = {"metric": METRIC, "value": value, "unit": "volumes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if prec == B.OAM_PREC_BF16X3 else "f32", "data": "synthetic",
            "config": config_dict(prec_name),
            "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
            "op_tflops_algorithmic": OPS_PER_STEP * info.flops_per_op / (per_step * 1e-3) / 1e12,
            "op_ms": {"forward": fwd_ms, "adjoint": adj_ms}, "flops_per_op": info.flops_per_op,
            "roofline": roof, "gpu_launches": int(launches),
            "e2e": {"value": world * args.steps / (e2e_ms / 1e3), "unit": "volumes/s",
                    "h2d_bytes_per_step": int(s_host.numel() * 4), "d2h_bytes_per_step": 2 * vol_bytes},
            "clocks": clk, "wall_s_timed": wall}
    if world == 1 and args.prec == "auto" and not args.no_forms:
        line["forms"] = {"lateral_fft": other_form(B.OAM_PREC_FFT)}
    if world == 1 and not args.no_forms:
        line["extensions"] = extensions()
    if acc is not None:
        forms = [("bf16x3", B.OAM_PREC_BF16X3), ("fft", B.OAM_PREC_FFT), ("fp32", B.OAM_PREC_FP32)]
        if prec != B.OAM_PREC_BF16X3:
            forms = [f for f in forms if f[1] != B.OAM_PREC_BF16X3]
        acc.run_device(forms, make_model)
        line["accuracy_vs_fp64"] = acc.finish()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_entry(info.flops_per_op)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", 1))
    rank = int(os.environ.get("RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.serve:
        if rank == 0:
            run_serve(args)
        return
    # the oracle leg's references start before the first CUDA call (spawned process)
    acc = AccuracyLeg() if world == 1 and not args.no_cpu_baseline and not args.no_accuracy else None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
    run_ours(args, rank, world, acc)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
