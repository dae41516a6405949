"""Served reconstructions: Poisson-arriving requests over the C request server.

    python -m paper_2009_10173_gb300.serve --rates 2 20 --requests 60

For each arrival rate, requests (sizes as the batched workload, with an
occasional 200x200x300 volume) are submitted at exponential inter-arrival
times to one oam_server with a 150 GB device-memory budget; the server admits
them as slots and memory free up, and their work overlaps on the GPU.  Prints
one JSON line per rate: offered and achieved load, volumes/s, p50/p99 latency.
Signals come from a pool of prepared instances (vessel phantom, 20 dB noise),
prepared before the clock starts.  Marshalling only: all arithmetic runs in
liboam.so.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import binding as B
from . import configs, inputs
from .batch import build_model


def is_small(cfg):
    """Requests whose FP64 reference a host can compute in well under a minute
    (64 x 64 scans with at most 192 depths)."""
    return cfg["py"] <= 64 and cfg["px"] <= 64 and cfg["nz"] <= 192


def final_config(cfg, precision):
    """The request's configuration after the sample-count fallback of build_model."""
    cfg, m = build_model(cfg, precision)
    m.close()
    return cfg


class Instance:
    """A prepared request: configuration, pinned host signals and image buffers.

    The noisy signals are seeded noise (20 dB) on clean signals A H of the
    request's vessel phantom; A is the library's FP32 operator unless the
    caller passes the noisy signals (``signals``, e.g. made by a reference
    implementation for requests whose results it checks)."""

    def __init__(self, cfg, precision, signals=None):
        cfg, m = build_model(cfg, precision)
        if signals is None:
            H = inputs.phantom(cfg, cfg.get("seed", 0), kind="vessels", count=10)
            clean = m.forward(torch.from_numpy(H.astype(np.float32)).cuda()).cpu().numpy()
            noisy = inputs.add_noise(clean, 20.0, cfg.get("seed", 0) + 10 ** 6).astype(np.float32)
        else:
            noisy = np.ascontiguousarray(signals, np.float32)
        m.close()
        self.cfg = cfg
        self.structs = B.structs_from_config(cfg)
        self.h_s = torch.from_numpy(noisy).pin_memory()
        self.vol_shape = (cfg["py"], cfg["px"], cfg["nz"])

    def new_outputs(self):
        return (torch.empty(self.vol_shape, dtype=torch.float32).pin_memory(),
                torch.empty(self.vol_shape, dtype=torch.float32).pin_memory())


def make_server(budget_bytes=150 * 10 ** 9, slots=8, precision=B.OAM_PREC_BF16X3, lsqr_iters=30, fista_iters=50,
                power_iters=20, lambda_rel=1e-3):
    opts = B.OamServerOpts(int(budget_bytes), int(slots), int(precision), int(lsqr_iters), int(fista_iters),
                           int(power_iters), float(lambda_rel))
    return B.oam_server_create(opts)


def run_rate(server, pool, rate, n_requests, seed, timeout_s=3600.0, check=None, check_picks=None,
             buffers_per_instance=None, host_bytes=48e9):
    """Submit n_requests at Poisson arrival times (rate per second), wait for all.

    Output images go into pinned host buffers allocated before the clock
    starts: ``buffers_per_instance`` pairs per prepared instance, or by default
    one pair per request of the schedule (no allocation while the clock runs,
    at the cost of host memory for every request's images; scaled down, to at
    least two pairs per instance, when that would exceed ``host_bytes``).  A pair is reused
    once the request that held it has completed, and a new pair is allocated
    only when every pair of that instance is still in flight (counted in
    ``output_allocs``).  Latency is reported from submission (the
    server's clock) and from the scheduled arrival time (adds any delay of the
    submission itself).  ``check(index_in_pool, x_l2, x_l1)``, if given, is
    called for every completed request; it
    returns None (not checked) or a dict of errors, summarised in the result.
    Checks run after the clock stops, on copies of the images of the instances
    in ``check_picks`` (every instance if None)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, n_requests)
    picks = rng.integers(0, len(pool), n_requests)
    counts = np.bincount(picks, minlength=len(pool))
    if buffers_per_instance is None:
        pairs = [int(c) for c in counts]
        pair_bytes = [8 * int(np.prod(getattr(inst, "vol_shape", (0,)))) for inst in pool]
        total = sum(n * b for n, b in zip(pairs, pair_bytes))
        if total > host_bytes:
            pairs = [min(n, max(2, int(n * host_bytes / total))) for n in pairs]
    else:
        pairs = [min(int(c), buffers_per_instance) for c in counts]
    free = {j: [inst.new_outputs() for _ in range(pairs[j])] for j, inst in enumerate(pool)}
    busy = {j: [] for j in range(len(pool))}  # (request id, submit lag, x2, x1), oldest first
    lat, lat_arrival, to_check = [], [], []
    state = {"failed": 0, "allocs": 0}

    def finish(pick, rid, lag, x2, x1):
        info = B.oam_server_poll(server, rid)
        if info.state != 2:
            state["failed"] += 1
            return
        lat.append(info.latency_s)
        lat_arrival.append(lag + info.latency_s)
        if check is not None and (check_picks is None or pick in check_picks):
            to_check.append((pick, x2.clone(), x1.clone()))

    def take(j):
        if free[j]:
            return free[j].pop()
        if busy[j] and B.oam_server_poll(server, busy[j][0][0]).state >= 2:
            rid, lag, x2, x1 = busy[j].pop(0)
            finish(j, rid, lag, x2, x1)
            return x2, x1
        state["allocs"] += 1
        return pool[j].new_outputs()

    t0 = time.perf_counter()
    t_next = t0
    for i in range(n_requests):
        t_next += gaps[i]
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        j = int(picks[i])
        x2, x1 = take(j)
        s, g, e = pool[j].structs
        rid = B.oam_server_submit(server, s, g, e, pool[j].h_s, x2, x1)
        busy[j].append((rid, max(0.0, time.perf_counter() - t_next), x2, x1))
    t_last_submit = time.perf_counter() - t0
    for j in busy:
        for rid, lag, x2, x1 in busy[j]:
            rc = B.oam_server_wait(server, rid, timeout_s)
            if rc != B.OAM_OK:
                state["failed"] += 1
                continue
            finish(j, rid, lag, x2, x1)
    makespan = time.perf_counter() - t0
    stats = B.oam_server_stats(server)
    pct = (lambda v, q: float(np.percentile(v, q)) if v else None)
    out = {"rate_offered_per_s": rate, "rate_achieved_submit_per_s": n_requests / t_last_submit,
           "requests": n_requests, "completed": len(lat), "failed": state["failed"], "makespan_s": makespan,
           "volumes_per_s": len(lat) / makespan,
           "p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99),
           "p50_latency_from_arrival_s": pct(lat_arrival, 50), "p99_latency_from_arrival_s": pct(lat_arrival, 99),
           "output_allocs": state["allocs"],
           "peak_running": stats.peak_running, "peak_reserved_gb": stats.peak_reserved_bytes / 1e9}
    if check is not None:
        errs = [e for e in (check(p, x2, x1) for p, x2, x1 in to_check) if e is not None]
        out["checked"] = len(errs)
        if errs:
            for key in errs[0]:
                out[f"max_{key}"] = max(float(e[key]) for e in errs)
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--rates", type=float, nargs="+", default=[2.0, 20.0])
    p.add_argument("--requests", type=int, default=60)
    p.add_argument("--pool", type=int, default=12)
    p.add_argument("--slots", type=int, default=8)
    p.add_argument("--budget-gb", type=float, default=150.0)
    p.add_argument("--prec", default="bf16x3", choices=["bf16x3", "fft", "fp32"],
                   help="operator form of the served models")
    a = p.parse_args()
    prec = {"bf16x3": B.OAM_PREC_BF16X3, "fft": B.OAM_PREC_FFT, "fp32": B.OAM_PREC_FP32}[a.prec]
    pool = [Instance(configs.served_request(2000 + j), prec) for j in range(a.pool)]
    for k, rate in enumerate(a.rates):
        server = make_server(a.budget_gb * 1e9, a.slots, precision=prec)
        res = run_rate(server, pool, rate, a.requests, seed=3000 + k)
        B.oam_server_stop(server)
        res.update({"workload": "served: Poisson arrivals, sizes as the batched workload plus occasional "
                                "200x200x300 volumes, 30 LSQR + 50 FISTA each",
                    "slots": a.slots, "budget_gb": a.budget_gb, "pool_instances": a.pool, "prec": a.prec})
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
