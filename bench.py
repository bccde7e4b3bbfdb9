#!/usr/bin/env python3
"""Benchmark of the MeCuCo Fast-mode curvature hot path on GB300.

One step = one full pass of the hot path over the workload: kNN (distance
search + exact re-rank), gather/centre/Gram/moments, the k x k eigensolves and
the Fast estimator, for every point.  Default workload: 1,000,000 points in
R^4096 stored in BF16 (32 curved 8-dimensional patches), k = 64, the chosen
(BF16-mixed) form.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Inputs are generated on the host, copied to HBM before the timed region, and
are larger than L2 (8.2 GB).  Under torchrun every rank runs an independent
replica (the path shards only over independent problems; no collective is on
the data path); ``value`` counts the points of all ranks.

Besides the device-timed value the line carries: ``e2e`` (the same metric
through the host-buffer C entry point with copies inside the timed region),
``roofline`` (the dominant kernel against the measured peak), ``plain_fp32``
(the plain FP32 form on a timed sample of query rows), ``cpu_baseline`` (the
FP64 oracle on a bounded sample, host cores), ``stages`` and ``clocks``.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "curvature points/s at N=1M,m=4096,k=64 vs plain FP32 form; % of roofline"

WORKLOADS = {
    "curved_patches_1m": dict(kind="curved_patches", N=1_000_000, m=4096, k=64, n_patches=32,
                              desc="32 curved 8-dim quadratic patches in R^4096 + N(0,0.005^2) noise, BF16"),
    "curved_patches_100k": dict(kind="curved_patches", N=100_000, m=4096, k=64, n_patches=32,
                                desc="curved patches, reduced N (development size)"),
    "sparse_clusters_70k": dict(kind="sparse_clusters", N=70_000, m=784, k=50,
                                desc="10 sparse [0,1] Gaussian clusters, 80% zeros, FP32 (MNIST-class shape)"),
}


def _rank_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _make_workload(name: str, seed: int = 1):
    import numpy as np
    from paper_2606_06329_gb300 import synth
    w = WORKLOADS[name]
    if w["kind"] == "curved_patches":
        bits = synth.curved_patches(n=w["N"], m=w["m"], n_patches=w["n_patches"], seed=seed)
        return bits, "bf16"
    X = synth.sparse_clusters(n=w["N"], m=w["m"], seed=seed)
    return X, "f32"


def _to_torch(host, kind):
    import numpy as np
    import torch
    if kind == "bf16":
        return torch.from_numpy(host.view(np.int16)).view(torch.bfloat16)
    return torch.from_numpy(host)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

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
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sms.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sms.sort()
        med = sms[len(sms) // 2] if sms else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _profile_traffic(N: int, nq: int):
    """DRAM bytes per launch of the distance-search kernel, from the line
    ``bench-traffic: kernel=knn_tc_kernel pairs=P bytes=B source_sha1=H`` of a
    committed ncu summary under profiles/ (one capture of P query-candidate
    pairs), scaled to this launch's nq * N pairs; None when no summary matches
    the current kernel source."""
    import glob
    import hashlib
    src = os.path.join(ROOT, "paper_2606_06329_gb300", "csrc", "knn_tc.cu")
    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for ln in open(path):
            if not ln.startswith("bench-traffic:"):
                continue
            kv = dict(tok.split("=", 1) for tok in ln.split()[1:] if "=" in tok)
            if kv.get("kernel") != "knn_tc_kernel" or kv.get("source_sha1") != sha:
                continue
            return float(kv["bytes"]) * (nq * N) / float(kv["pairs"])
    return None


def _cpu_baseline(host, kind, k, n_rows, seed=7):
    """The FP64 oracle (brute-force kNN over all N points + Alg. 1 Fast branch)
    on a bounded sample of query rows, timed on the host cores."""
    import numpy as np
    import oracle
    oracle.build()
    N = host.shape[0]
    rows = np.random.default_rng(seed).choice(N, n_rows, replace=False)
    bf = kind == "bf16"
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    idx, _ = oracle.knn(host, k, rows=rows, bf16_bits=bf, nthreads=cores)
    full = np.zeros((N, k), dtype=np.int32)
    full[rows] = idx
    oracle.curvature(host, k, full, rows=rows, bf16_bits=bf, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": n_rows / dt, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_rows} random query rows of the same workload, each a brute-force FP64 kNN scan "
                      f"over all {N} points plus the FP64 Fast estimator; {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    host, kind = _make_workload(args.workload)
    vals, times = [], []
    for step in range(args.warmup + args.steps):
        res = _cpu_baseline(host, kind, w["k"], args.ref_rows, seed=100 + step)
        if step >= args.warmup:
            vals.append(res["value"])
            times.append(args.ref_rows / res["value"] * 1e3)
    value = sum(vals) / len(vals)
    # n_gpus: the N this run was launched with (the pairing with our line of that N);
    # the oracle itself runs on rank 0's host cores, as config.device says
    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.workload}: {w['desc']}", "N": w["N"], "m": w["m"], "k": w["k"],
                       "variant": "literal", "precision": "fp64 oracle", "device": "host cores (rank 0)",
                       "sample_rows_per_step": args.ref_rows},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"]},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_timing(elapsed_ms: float, n_per_rank: int, steps: int, dist=None, device="cpu"):
    """Whole-job timing of replicas: the slowest rank's timed region (max over
    ranks) and the points all ranks processed per second in it."""
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    slowest = float(t.item())
    return slowest, n_per_rank * world * steps / (slowest * 1e-3)


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = _rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2606_06329_gb300 import api, build, _native as NAT
    build.build()
    w = WORKLOADS[args.workload]
    N, m, k = w["N"], w["m"], w["k"]
    host, kind = _make_workload(args.workload, seed=1 + rank)
    Xh = _to_torch(host, kind)
    Xh_pinned = Xh.pin_memory() if not args.no_e2e else None
    Xd = Xh.cuda()
    ctx = api.Context(local)
    if args.jacobi_fp64 is not None:
        ctx.set_option(NAT.OPT_JACOBI_FP64, args.jacobi_fp64)
    prec, var = args.precision, args.variant
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        return ctx.mecuco_curvature(Xd, k, precision=prec, variant=var)

    for _ in range(args.warmup):
        kap = step()
    torch.cuda.synchronize()
    status = ctx.mecuco_get_last_status()
    ctx.set_option(NAT.OPT_PROFILE, 1)
    ctx.mecuco_get_stage_times()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        kap = step()
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    stats = ctx.mecuco_get_stats()
    stages = ctx.mecuco_get_stage_times()
    ctx.set_option(NAT.OPT_PROFILE, 0)
    launches = stats["kernel_launches"] * args.steps
    elapsed_ms, value = aggregate_timing(elapsed_ms, N, args.steps, dist, device="cuda")
    ms_per_step = elapsed_ms / args.steps

    # roofline of the dominant kernel
    peaks, src = _peaks()
    dom = max(stages, key=lambda s: stages[s][0])
    roof = None
    knn_ms, knn_n = stages["knn_search"]
    if knn_n:
        if prec == "bf16_mixed":
            flops_per_launch = 2.0 * N * N * m / knn_n * args.steps
            ach = flops_per_launch / (knn_ms / knn_n * 1e-3) / 1e12
            pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
            nq_launch = N / knn_n * args.steps
            traffic = _profile_traffic(N, nq_launch)
            roof = {"kernel": "knn_tc_kernel (distance GEMM + fused candidate select)", "bound": "tensor",
                    "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                    "traffic": traffic,
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a smaller capture, "
                                      "scaled by query-candidate pairs (profiles/)" if traffic else None,
                    "peak_source": f"{src} bf16_tflops_sustained (kernel timed inside a multi-second step)",
                    "algorithmic": "2*N*N*m FLOP per step (dot products of every query with every point)",
                    "share_of_step": knn_ms / elapsed_ms}
        else:
            flops_per_launch = 2.0 * N * N * m / knn_n * args.steps
            ach = flops_per_launch / (knn_ms / knn_n * 1e-3) / 1e12
            roof = {"kernel": "knn_simt_kernel", "bound": "alu", "achieved": ach, "peak": 2 * 128 * 152 * 2.07e9 / 1e12,
                    "unit": "TFLOP/s", "frac": ach / (2 * 128 * 152 * 2.07e9 / 1e12), "traffic": None,
                    "peak_source": "FP32 FFMA: 128 lanes x 152 SMs x 2 FLOP x 2.07 GHz",
                    "share_of_step": knn_ms / elapsed_ms}

    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "bf16-gemm/f32/f32x2-refine" if prec == "bf16_mixed" else "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w['desc']}", "N": N, "m": m, "k": k, "variant": var,
                       "precision": prec, "l2": "inputs larger than L2 (X is %.1f GB)" % (Xd.numel() * Xd.element_size() / 1e9),
                       "parallelism": f"replicas x{world}", "jacobi_fp64": args.jacobi_fp64},
            "roofline": roof, "gpu_launches": launches, "clocks": clk, "status": status,
            "stages": {s: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                       for s, v in stages.items()},
            "knn_stats": {kk: stats[kk] for kk in ("knn_uncertified", "knn_fallback_rows", "jacobi_max_sweeps",
                                                  "jacobi_not_converged", "rank_deficient")}}

    # plain FP32 form on a sample of query rows (all N points remain candidates)
    if rank == 0 and not args.no_plain and prec != "fp32":
        S = min(args.plain_rows, N)
        ctx.mecuco_knn_range(Xd, k, 0, S, precision="fp32")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        idx = ctx.mecuco_knn_range(Xd, k, 0, S, precision="fp32")
        ctx.mecuco_curvature_range(Xd, k, 0, S, idx=idx, precision="fp32", variant=var)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        line["plain_fp32"] = {"value": S / (pms * 1e-3), "unit": "points/s",
                              "sample": f"query rows [0,{S}) of the same workload against all {N} points, "
                                        f"kNN + estimator in plain FP32; {pms:.0f} ms",
                              "chosen_over_plain": value / world / (S / (pms * 1e-3))}

    # end to end through the host-buffer C entry point (copies inside the timed region)
    if rank == 0 and not args.no_e2e:
        kap_h = torch.empty(N, dtype=torch.float32).pin_memory()
        ctx.mecuco_curvature_host(Xh_pinned, k, precision=prec, variant=var, kappa_out=kap_h)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.mecuco_curvature_host(Xh_pinned, k, precision=prec, variant=var, kappa_out=kap_h)
        dt = time.perf_counter() - t0
        line["e2e"] = {"value": N * args.e2e_steps / dt, "unit": "points/s",
                       "h2d_bytes_per_step": int(Xh_pinned.numel() * Xh_pinned.element_size()),
                       "d2h_bytes_per_step": int(N * 4), "steps": args.e2e_steps}

    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = _cpu_baseline(host, kind, k, args.cpu_rows)

    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="curved_patches_1m")
    ap.add_argument("--precision", choices=["bf16_mixed", "fp32"], default="bf16_mixed")
    ap.add_argument("--variant", choices=["literal", "haar"], default="literal")
    ap.add_argument("--jacobi-fp64", type=int, choices=[0, 1], default=None)
    ap.add_argument("--plain-rows", type=int, default=4096)
    ap.add_argument("--cpu-rows", type=int, default=32)
    ap.add_argument("--ref-rows", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
