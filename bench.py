#!/usr/bin/env python3
"""Benchmark of the GB300 P-APG iteration (pair-updates/s and % of HBM roofline).

Workload (default): recipe (2) of the configs -- N = 20,000 points in n = 10
dimensions, f0 = max of 8 affine functions, FP32 multiplier array (two 1.6 GB
arrays, far larger than L2).  One step = one P-APG iteration (Fig. 2 steps
1-4): the fold, the pass over all N(N-1) pairs that streams the multiplier
array once (read theta^(1)_l and theta^(1)_{l-1}, write theta^(1)_{l+1}), and
the FP64 reduction of its partial sums.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores (one oracle
iteration on a bounded sample of the same recipe per step).  With --gpus N > 1
(under torchrun) every rank solves its own independent instance (replicas; no
collective), so the work per GPU is fixed ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1407_7220_gb300 import datagen  # noqa: E402

RECIPE, N_DEF, n_DEF, GAMMA = "maxaff", 20000, 10, 1e-2
HBM_FALLBACK = 6800.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ---------------------------------------------------------------------------
def oracle_rate(N: int, steps: int, warmup: int):
    """Pair-updates/s of the oracle (as it stands) on an N-point sample of the recipe."""
    from oracle import oracle as O
    X, yb, _ = datagen.make(RECIPE, N=N, n=n_DEF)
    s = O.Solver(X, yb, gamma=GAMMA, restart=False)
    if warmup:
        s.iterate(warmup)
    t0 = time.perf_counter()
    s.iterate(steps)
    dt = time.perf_counter() - t0
    return N * (N - 1) * steps / dt, dt, O.num_threads()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    Ns = 2000
    steps = max(1, args.steps)
    rate, dt, cores = oracle_rate(Ns, steps, min(args.warmup, 3))
    line = {
        "impl": "reference", "metric": "pair-updates/s", "value": rate, "unit": "pair-updates/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{RECIPE} recipe, oracle sample N={Ns} n={n_DEF} (full workload N={N_DEF})",
                   "N": Ns, "n": n_DEF, "gamma": GAMMA},
        "cpu_baseline": {"value": rate, "unit": "pair-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{steps} P-APG iterations at N={Ns}, n={n_DEF} (FP64, OpenMP)"},
        "e2e": {"value": rate, "unit": "pair-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_1407_7220_gb300 as crg

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    N, n = args.N, args.n
    # each rank solves its own instance (seeded by rank): replicas, weak scaling
    X, yb, _ = datagen.make(RECIPE, N=N, n=n, seed=datagen.default_seed(RECIPE) + rank)
    stream = torch.cuda.Stream(device=dev)
    opts = dict(gamma=GAMMA, theta_dtype=args.dtype, stochastic_round=1, restart=0, driver=args.driver,
                profile=1, stream=stream.cuda_stream)

    # --- device-resident throughput (value) ---
    s = crg.Solver(X, yb, **opts)
    s.iterate(args.warmup)
    torch.cuda.synchronize()
    for k in range(4):
        s.profile(k)  # drop warm-up timings
    barrier = (lambda: torch.distributed.barrier()) if ws > 1 else (lambda: None)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ev0.record(stream)
        s.iterate(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    pair_ms, pair_n = s.profile(crg.PROFILE_PAIR)
    fold_ms, fold_n = s.profile(crg.PROFILE_FOLD)
    pers_ms, pers_n = s.profile(crg.PROFILE_PERSISTENT)
    kkt_ms, kkt_n = s.profile(crg.PROFILE_KKT)
    launches = pair_n + fold_n + pers_n + kkt_n
    info = s.info()
    s.close()

    pairs = N * (N - 1)
    b = 4 if args.dtype == "f32" else 2
    value = ws * pairs * args.steps / (ms / 1e3)
    peak, peak_kind = peaks()
    # dominant kernel: the pair pass (phase driver) or the persistent launch
    if pair_n:
        dom_ms, per_launch_units, dom_name = pair_ms / pair_n, 1, "pair pass"
    else:
        dom_ms, per_launch_units, dom_name = pers_ms / max(pers_n, 1), args.steps / max(pers_n, 1), "persistent"
    alg_bytes = 3 * b * pairs * per_launch_units
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9

    # --- end to end through the public API with host buffers (e2e) ---
    opts_e2e = dict(opts)
    opts_e2e["profile"] = 0
    Xp = torch.from_numpy(X).pin_memory().numpy()
    ybp = torch.from_numpy(yb).pin_memory().numpy()
    yout = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e = crg.Solver(Xp, ybp, **opts_e2e)          # H2D copy of X, ybar + set-up
    e.iterate(args.steps)
    y_out, xi_out = e.solution()                # D2H of the fitted values and subgradients
    yout[:] = y_out
    e.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if ws > 1:
        t = torch.tensor([e2e_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        Ns = 2000
        rate, dt, cores = oracle_rate(Ns, 8, 1)
        cpu = {"value": rate, "unit": "pair-updates/s", "cores": cores, "kind": "oracle",
               "sample": f"8 P-APG iterations of the FP64 oracle at N={Ns}, n={n} of the same recipe ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": "pair-updates/s", "value": value, "unit": "pair-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"{RECIPE} recipe (max of 8 affine), N={N}, n={n}, theta {args.dtype}, "
                                   f"gamma={GAMMA}, stochastic rounding, plain P-APG momentum",
                       "N": N, "n": n, "gamma": GAMMA, "theta_bytes": b, "driver": info and args.driver,
                       "l2": "inputs larger than L2 (2 theta arrays of %.2f GB)" % (pairs * b / 1e9),
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": dom_name, "algorithmic_bytes_per_launch": alg_bytes},
            "hbm_frac_whole_step": (3 * b * pairs * args.steps / (ms / 1e3) / 1e9) / peak,
            "e2e": {"value": ws * pairs * args.steps / e2e_s, "unit": "pair-updates/s",
                    "h2d_bytes_per_step": (N * n + N) * 8 / args.steps,
                    "d2h_bytes_per_step": (N * n + N) * 8 / args.steps,
                    "note": "create from pinned host arrays + K iterations + fitted values back, per run"},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "kernel_ms": {"pair": pair_ms, "fold": fold_ms, "persistent": pers_ms, "kkt": kkt_ms},
        }
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=N_DEF)
    ap.add_argument("--n", type=int, default=n_DEF)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--driver", type=int, default=2, help="1 persistent, 2 phase kernels")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
