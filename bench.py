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
    "curved_patches_200k": dict(kind="curved_patches", N=200_000, m=4096, k=64, n_patches=32,
                                desc="curved patches, reduced N (one search launch, 1.6 GB: traffic captures)"),
    "sparse_clusters_70k": dict(kind="sparse_clusters", N=70_000, m=784, k=50,
                                desc="10 sparse [0,1] Gaussian clusters, 80% zeros, FP32 (MNIST-class shape)"),
    "batched_256": dict(kind="batched", nsets=256,
                        desc="256 independent datasets in one batched call: N ~ U[500, 20000], m in {64, 128, 256, "
                             "512, 1024}, k ~ U[10, 64]; seeded 2-layer tanh MLP images of d-dim Gaussian latents "
                             "(d ~ U[2, 16]) + N(0, 0.01^2) noise, FP32"),
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


def _cpu_baseline(host, kind, k, rows):
    """The FP64 oracle (brute-force kNN over all N points + Alg. 1 Fast branch)
    on a bounded sample of query rows, timed on the host cores.  Returns the
    cpu_baseline object and the oracle's lists, distances and curvatures of
    those rows (the accuracy reference)."""
    import numpy as np
    import oracle
    oracle.build()
    N = host.shape[0]
    rows = np.asarray(rows, dtype=np.int64)
    bf = kind == "bf16"
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    idx, dist = oracle.knn(host, k, rows=rows, bf16_bits=bf, nthreads=cores)
    full = np.zeros((N, k), dtype=np.int32)
    full[rows] = idx
    kap = oracle.curvature(host, k, full, rows=rows, bf16_bits=bf, nthreads=cores)
    dt = time.perf_counter() - t0
    res = {"value": rows.size / dt, "unit": "points/s", "cores": cores, "kind": "oracle",
           "sample": f"{rows.size} random query rows of the same workload, each a brute-force FP64 kNN scan "
                     f"over all {N} points plus the FP64 Fast estimator; {dt:.1f} s"}
    return res, idx, dist, kap


def _row_f64(host, kind, r):
    import numpy as np
    x = host[r]
    if kind == "bf16":
        return (x.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return x.astype(np.float64)


def _accuracy(host, kind, rows, idx_gpu, kap_gpu, ref_idx, ref_d, ref_kap, tie_rel=1e-6):
    """Relative curvature error against the FP64 oracle and neighbour-list
    mismatches the tie rule does not excuse (positions may differ only between
    distances equal within tie_rel relative), on the sampled rows."""
    import numpy as np
    err = np.abs(np.asarray(kap_gpu, np.float64) - ref_kap) / np.abs(ref_kap)
    bad = 0
    for i, q in enumerate(rows):
        g = idx_gpu[i]
        if np.array_equal(g, ref_idx[i]):
            continue
        if len(set(g.tolist())) != g.size or g.min() < 0 or g.max() >= host.shape[0]:
            bad += 1
            continue
        xq = _row_f64(host, kind, q)
        dg = np.array([((_row_f64(host, kind, j) - xq) ** 2).sum() for j in g])
        if np.any(np.abs(dg - ref_d[i]) > tie_rel * np.maximum(np.abs(ref_d[i]), 1e-300)):
            bad += 1
    return {"kappa_max_rel": float(err.max()), "kappa_median_rel": float(np.median(err)),
            "knn_mismatch_rows": int(bad), "rows": int(len(rows))}


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    if w["kind"] == "batched":
        return run_reference_batched(args)
    host, kind = _make_workload(args.workload)
    vals, times = [], []
    import numpy as np
    for step in range(args.warmup + args.steps):
        rows = np.random.default_rng(100 + step).choice(host.shape[0], args.ref_rows, replace=False)
        res = _cpu_baseline(host, kind, w["k"], rows)[0]
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


def run_reference_batched(args):
    """The oracle on the batched workload: each step a bounded sample of rows
    from randomly chosen datasets of the batch (brute-force FP64 kNN over the
    dataset + the FP64 Fast estimator), host cores, rank 0."""
    import numpy as np
    import oracle
    from paper_2606_06329_gb300 import synth
    w = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    sets = synth.batched_mlp_datasets(nsets=w["nsets"], seed=1)
    oracle.build()
    cores = os.cpu_count() or 1
    vals, times = [], []
    for step in range(args.warmup + args.steps):
        rng = np.random.default_rng(100 + step)
        pick = rng.choice(len(sets), min(args.cpu_sets, len(sets)), replace=False)
        t0 = time.perf_counter()
        nrows = 0
        for i in pick:
            X, k = sets[i]["X"], sets[i]["k"]
            r = np.sort(rng.choice(X.shape[0], min(args.cpu_rows_per_set, X.shape[0]), replace=False))
            ridx, _ = oracle.knn(X, k, rows=r, nthreads=cores)
            full = np.zeros((X.shape[0], k), dtype=np.int32)
            full[r] = ridx
            oracle.curvature(X, k, full, rows=r, nthreads=cores)
            nrows += r.size
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            vals.append(nrows / dt)
            times.append(dt * 1e3)
    value = sum(vals) / len(vals)
    sample = (f"{nrows} random rows of {len(pick)} random datasets of the batch per step, each a brute-force FP64 "
              f"kNN scan of its dataset plus the FP64 Fast estimator")
    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.workload}: {w['desc']}", "datasets": len(sets), "variant": "literal",
                       "precision": "fp64 oracle", "device": "host cores (rank 0)"},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle", "sample": sample},
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


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 lanes x FMA (2 FLOP) x 2.07 GHz


def _stage_fracs(stages, steps, shapes, prec, rotations, peaks, elt=2):
    """Per-stage achieved rate against its binding roof, from one profiled step
    (CUDA events around every launch).  shapes: the (N, m, k) of every dataset
    of the step; the algorithmic work per stage is summed over them:
      knn_search  2 N^2 m FLOP (tensor, BF16; FP32 lanes in the plain form)
      knn_rerank  N x 128 candidate rows x m x elt bytes read (2 lists of 64 per
                  row from the tensor-core search), against HBM
      gram        the gathered patches, N k m elements, against HBM
      rotate      the gathered patches plus the rotated patches written
                  (N x k rows x m BF16), against HBM
      moments     k(k+1)(k+2)/6 m multiply-adds per point (the distinct third
                  moments), x 2 FLOP (tensor, BF16)
      jacobi      18 k FLOP per plane rotation (two-sided update of A and the
                  eigenvector update; k weighted by the rotations a k x k patch
                  takes, ~k^2: sum N k^3 / sum N k^2) + 8 k^3 per patch for the
                  refinement's three products, against the FP32 lanes
      estimator   k (2 k^2 p + k p (p + 1)) FLOP per point (B = M_j W and the
                  upper triangle of W^T B), p = k - 1, against the FP32 lanes"""
    bf = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    hbm = peaks.get("hbm_gbs")
    tot = {key: 0.0 for key in ("knn_search", "knn_rerank", "gram", "rotate", "moments", "jacobi_ref", "estimator",
                                "nk3", "nk2")}
    for N, m, k in shapes:
        N, m, k = float(N), float(m), float(k)
        p = k - 1
        tot["knn_search"] += 2.0 * N * N * m
        tot["knn_rerank"] += N * 128.0 * m * elt
        tot["gram"] += N * k * m * elt
        tot["rotate"] += N * k * m * elt + N * k * m * 2.0
        tot["moments"] += 2.0 * k * (k + 1) * (k + 2) / 6.0 * m * N
        tot["jacobi_ref"] += 8.0 * k ** 3 * N
        tot["estimator"] += k * (2.0 * k * k * p + k * p * (p + 1)) * N
        tot["nk3"] += N * k ** 3
        tot["nk2"] += N * k ** 2
    kw = tot["nk3"] / tot["nk2"]
    work = {
        "knn_search": (tot["knn_search"], "tensor" if prec == "bf16_mixed" else "alu"),
        "knn_rerank": (tot["knn_rerank"], "hbm"),
        "gram": (tot["gram"], "hbm"),
        "rotate": (tot["rotate"], "hbm"),
        "moments": (tot["moments"], "tensor"),
        "jacobi": (18.0 * kw * rotations + tot["jacobi_ref"], "alu"),
        "estimator": (tot["estimator"], "alu"),
    }
    out = {}
    for name, (ms, n) in stages.items():
        if n == 0:
            continue
        ent = {"ms_per_step": ms / steps, "launches_per_step": n / steps}
        if name in work:
            w, bound = work[name]
            sec = ms / steps * 1e-3
            if bound == "hbm":
                ach, pk, unit = w / sec / 1e9, hbm, "GB/s"
            elif bound == "tensor":
                ach, pk, unit = w / sec / 1e12, bf, "TFLOP/s"
            else:
                ach, pk, unit = w / sec / 1e12, FP32_PEAK_TFLOPS, "TFLOP/s"
            ent.update({"bound": bound, "achieved": ach, "peak": pk, "unit": unit, "frac": ach / pk,
                        "work_per_step": w})
        out[name] = ent
    return out


def run_ours(args):
    if WORKLOADS[args.workload]["kind"] == "batched":
        return run_batched(args)
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
    knn_stage = NAT.STAGES.index("knn_search")

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
    # timed region: only the distance-search launches are bracketed by events
    # (4 launches per step), the rest of the path runs un-instrumented
    ctx.set_option(NAT.OPT_PROFILE_STAGES, 1 << knn_stage)
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
    timed = ctx.mecuco_get_stage_times()
    launches = stats["kernel_launches"] * args.steps
    elapsed_ms, value = aggregate_timing(elapsed_ms, N, args.steps, dist, device="cuda")
    ms_per_step = elapsed_ms / args.steps
    status = status or ctx.mecuco_get_last_status()

    # stage times: one more step with every launch bracketed (outside the timed region)
    ctx.set_option(NAT.OPT_PROFILE_STAGES, 0)
    ctx.mecuco_get_stage_times()
    step()
    torch.cuda.synchronize()
    stages = ctx.mecuco_get_stage_times()
    stats1 = ctx.mecuco_get_stats()
    ctx.set_option(NAT.OPT_PROFILE, 0)

    # roofline of the dominant kernel, its launches timed inside the timed region
    peaks, src = _peaks()
    roof = None
    knn_ms, knn_n = timed["knn_search"]
    if knn_n:
        flops_per_launch = 2.0 * N * N * m / knn_n * args.steps
        ach = flops_per_launch / (knn_ms / knn_n * 1e-3) / 1e12
        nq_launch = N / knn_n * args.steps
        if prec == "bf16_mixed":
            pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
            traffic = _profile_traffic(N, nq_launch)
            roof = {"kernel": "knn_tc_kernel (distance GEMM + fused candidate select)", "bound": "tensor",
                    "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk, "traffic": traffic,
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, scaled "
                                      "by query-candidate pairs (profiles/)" if traffic else None,
                    "peak_source": f"{src} bf16_tflops_sustained (kernel timed inside a multi-second step)",
                    "algorithmic": "2*N*N*m FLOP per step (dot products of every query with every point)",
                    "launches_timed": knn_n, "share_of_step": knn_ms / elapsed_ms}
        else:
            roof = {"kernel": "knn_simt_kernel", "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS, "traffic": None,
                    "peak_source": "derived: FP32 FMA lanes 152 SMs x 128 x 2 FLOP x 2.07 GHz",
                    "share_of_step": knn_ms / elapsed_ms}

    jac = args.jacobi_fp64 if args.jacobi_fp64 is not None else (1 if prec == "bf16_mixed" else 0)
    jac_desc = {0: "FP32 sweeps", 1: "FP32 sweeps (to 2^-14), then one Ogita-Aishima refinement step with "
                                     "two-term-FP32 products (~2^-48)",
                2: "every sweep in FP64"}[jac]
    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "bf16-gemm/f32/f32x2-refine" if prec == "bf16_mixed" else "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w['desc']}", "N": N, "m": m, "k": k, "variant": var,
                       "precision": prec, "l2": "inputs larger than L2 (X is %.1f GB)" % (Xd.numel() * Xd.element_size() / 1e9),
                       "parallelism": f"replicas x{world}", "jacobi": jac_desc,
                       "timing": "headline with only the distance-search launches event-bracketed; stage "
                                 "times from one further step with every launch bracketed"},
            "roofline": roof, "gpu_launches": launches, "clocks": clk, "status": status,
            "stages": _stage_fracs(stages, 1, [(N, m, k)], prec, stats1["jacobi_rotations"], peaks,
                                   elt=Xd.element_size()),
            "knn_stats": {kk: stats[kk] for kk in ("knn_uncertified", "knn_fallback_rows", "jacobi_max_sweeps",
                                                  "jacobi_not_converged", "rank_deficient", "jacobi_rotations")}}

    S = min(args.plain_rows, N)
    rows = np.sort(np.random.default_rng(7).choice(S, min(args.cpu_rows, S), replace=False))
    kap_chosen = kap.cpu().numpy()
    if rank == 0 and prec != "fp32":
        idx_chosen = ctx.mecuco_knn_range(Xd, k, 0, S, precision=prec).cpu().numpy()
    # plain FP32 form on query rows [0, S) (all N points remain candidates)
    plain = None
    if rank == 0 and not args.no_plain and prec != "fp32":
        ctx.mecuco_knn_range(Xd, k, 0, min(S, 256), precision="fp32")
        torch.cuda.synchronize()
        ctx.set_option(NAT.OPT_PROFILE, 1)
        ctx.mecuco_get_stage_times()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        idx_p = ctx.mecuco_knn_range(Xd, k, 0, S, precision="fp32")
        kap_p = ctx.mecuco_curvature_range(Xd, k, 0, S, idx=idx_p, precision="fp32", variant=var)
        e1.record(stream)
        torch.cuda.synchronize()
        pst = ctx.mecuco_get_stage_times()
        ctx.set_option(NAT.OPT_PROFILE, 0)
        pms = e0.elapsed_time(e1)
        pk_ms, pk_n = pst["knn_search"]
        p_ach = 2.0 * S * N * m / (pk_ms * 1e-3) / 1e12 if pk_n else None
        plain = {"idx": idx_p.cpu().numpy(), "kappa": kap_p.cpu().numpy()}
        line["plain_fp32"] = {"value": S / (pms * 1e-3), "unit": "points/s",
                              "sample": f"query rows [0,{S}) of the same workload against all {N} points, "
                                        f"kNN + estimator in plain FP32 (FP32 search, FP64 centring, rotated "
                                        f"patch, FP32 Jacobi + two-term-FP32 refinement); {pms:.0f} ms",
                              "chosen_over_plain": value / world / (S / (pms * 1e-3)),
                              "knn_simt_roofline": {"bound": "alu", "achieved": p_ach, "peak": FP32_PEAK_TFLOPS,
                                                    "unit": "TFLOP/s",
                                                    "frac": p_ach / FP32_PEAK_TFLOPS if p_ach else None}}

    # FP64-sweep Jacobi arm on a row range: its stage time and how far K moves
    if rank == 0 and prec == "bf16_mixed" and args.fp64_rows > 0:
        R = min(args.fp64_rows, N)
        idx_r = ctx.mecuco_knn_range(Xd, k, 0, R, precision=prec)
        arm = {}
        for mode in (1, 2):
            ctx.set_option(NAT.OPT_JACOBI_FP64, mode)
            ctx.mecuco_curvature_range(Xd, k, 0, R, idx=idx_r, precision=prec, variant=var)
            torch.cuda.synchronize()
            ctx.set_option(NAT.OPT_PROFILE, 1)
            ctx.mecuco_get_stage_times()
            kr = ctx.mecuco_curvature_range(Xd, k, 0, R, idx=idx_r, precision=prec, variant=var)
            torch.cuda.synchronize()
            jt = ctx.mecuco_get_stage_times()["jacobi"][0]
            ctx.set_option(NAT.OPT_PROFILE, 0)
            arm[mode] = (kr.cpu().numpy().astype(np.float64), jt)
        ctx.set_option(NAT.OPT_JACOBI_FP64, -1 if args.jacobi_fp64 is None else args.jacobi_fp64)
        dev = np.abs(arm[2][0] - arm[1][0]) / np.abs(arm[2][0])
        line["jacobi_fp64_arm"] = {
            "rows": f"query rows [0,{R}) of the same workload (BF16-mixed moments, same neighbour lists)",
            "default_jacobi_ms": arm[1][1], "fp64_sweeps_jacobi_ms": arm[2][1],
            "kappa_max_rel_dev": float(dev.max()), "kappa_median_rel_dev": float(np.median(dev)),
            "fp64_kappa_rows": arm[2][0]}

    # end to end through the host-buffer C entry point (copies inside the timed region)
    if rank == 0 and not args.no_e2e:
        kap_h = torch.empty(N, dtype=torch.float32).pin_memory()
        ctx.mecuco_curvature_host(Xh_pinned, k, precision=prec, variant=var, kappa_out=kap_h)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.mecuco_curvature_host(Xh_pinned, k, precision=prec, variant=var, kappa_out=kap_h)
        dt = time.perf_counter() - t0
        # the bare host-to-device copy of X for comparison (CUDA events)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        Xd.copy_(Xh_pinned, non_blocking=True)
        h1.record(stream)
        torch.cuda.synchronize()
        nbytes = int(Xh_pinned.numel() * Xh_pinned.element_size())
        line["e2e"] = {"value": N * args.e2e_steps / dt, "unit": "points/s",
                       "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": int(N * 4), "steps": args.e2e_steps,
                       "ms_per_step": dt / args.e2e_steps * 1e3,
                       "bare_h2d_ms": h0.elapsed_time(h1), "bare_h2d_gbs": nbytes / (h0.elapsed_time(h1) * 1e-3) / 1e9}

    if rank == 0 and not args.no_cpu:
        cpu, ref_idx, ref_d, ref_kap = _cpu_baseline(host, kind, k, rows)
        line["cpu_baseline"] = cpu
        acc = {"reference": "FP64 oracle: brute-force kNN over all N points, Alg. 1 Fast branch on its lists",
               "tie_rule": "list positions may differ only between distances equal within 1e-6 relative"}
        if prec != "fp32":
            acc["chosen"] = _accuracy(host, kind, rows, idx_chosen[rows], kap_chosen[rows], ref_idx, ref_d, ref_kap)
        if plain is not None:
            acc["plain_fp32"] = _accuracy(host, kind, rows, plain["idx"][rows], plain["kappa"][rows], ref_idx,
                                          ref_d, ref_kap)
        if "jacobi_fp64_arm" in line:
            kr = line["jacobi_fp64_arm"]["fp64_kappa_rows"][rows]
            e = np.abs(kr - ref_kap) / np.abs(ref_kap)
            acc["chosen_fp64_sweeps"] = {"kappa_max_rel": float(e.max()), "kappa_median_rel": float(np.median(e)),
                                         "rows": int(len(rows))}
        line["accuracy"] = acc
    if "jacobi_fp64_arm" in line:
        del line["jacobi_fp64_arm"]["fp64_kappa_rows"]

    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


STAGE_KERNELS = {
    "knn_search": "knn_tc_kernel (distance GEMM + fused candidate select)",
    "knn_rerank": "knn_rerank_kernel", "gram": "gram_tc_kernel", "rotate": "rotate_tc_kernel",
    "moments": "tthird_tc_kernel (third moments of the rotated patch + estimator)",
    "jacobi": "jacobi_kernel + jacobi_refine_ff_kernel", "estimator": "estimator_kernel",
}


def run_batched(args):
    """The batched workload: every dataset of the batch through one
    mecuco_curvature_batched call, captured once into a CUDA graph; a step is
    one replay.  The configuration comes from mecuco_autotune_batched (run
    before the warm-up, untimed)."""
    import numpy as np
    import torch
    rank, world, local = _rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2606_06329_gb300 import api, build, synth, _native as NAT
    build.build()
    w = WORKLOADS[args.workload]
    sets = synth.batched_mlp_datasets(nsets=w["nsets"], seed=1 + rank)
    ks = [d["k"] for d in sets]
    shapes = [(d["X"].shape[0], d["X"].shape[1], d["k"]) for d in sets]
    npts = sum(sh[0] for sh in shapes)
    in_bytes = sum(d["X"].nbytes for d in sets)
    Xh = [torch.from_numpy(d["X"]).pin_memory() for d in sets]
    Xs = [x.cuda() for x in Xh]
    idx_out = [torch.empty((n, k), dtype=torch.int32, device="cuda") for n, _, k in shapes]
    ctx = api.Context(local)
    prec, var = args.precision, args.variant
    stream = torch.cuda.current_stream()
    tuned = ctx.mecuco_autotune_batched(Xs, ks, precision=prec, variant=var)

    def call():
        return ctx.mecuco_curvature_batched(Xs, ks, precision=prec, variant=var, idx_out=idx_out)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    # stage table: one eager call with every launch bracketed by events
    ctx.set_option(NAT.OPT_PROFILE_STAGES, 0)
    ctx.set_option(NAT.OPT_PROFILE, 1)
    ctx.mecuco_get_stage_times()
    call()
    torch.cuda.synchronize()
    stages = ctx.mecuco_get_stage_times()
    stats = ctx.mecuco_get_stats()
    ctx.set_option(NAT.OPT_PROFILE, 0)
    launches_per_call = stats["kernel_launches"]
    # the call captured once (tables and workspace exist after the eager calls)
    gs = torch.cuda.Stream()
    gs.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gs):
        with torch.cuda.graph(graph, stream=gs):
            kap_g = call()
    stream.wait_stream(gs)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    status = ctx.mecuco_get_last_status()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms, value = aggregate_timing(ev0.elapsed_time(ev1), npts, args.steps, dist, device="cuda")
    status = status or ctx.mecuco_get_last_status()

    # roofline of the dominant stage's kernel: K eager calls with only its
    # launches bracketed, right after the graph replays
    peaks, src = _peaks()
    elt = 4
    fr = _stage_fracs(stages, 1, shapes, prec, stats["jacobi_rotations"], peaks, elt=elt)
    dom = max((n for n in fr if "bound" in fr[n]), key=lambda n: fr[n]["ms_per_step"])
    ctx.set_option(NAT.OPT_PROFILE_STAGES, 1 << NAT.STAGES.index(dom))
    ctx.set_option(NAT.OPT_PROFILE, 1)
    ctx.mecuco_get_stage_times()
    for _ in range(args.steps):
        call()
    torch.cuda.synchronize()
    dms, dn = ctx.mecuco_get_stage_times()[dom]
    ctx.set_option(NAT.OPT_PROFILE, 0)
    dwork = fr[dom]["work_per_step"]
    dsec = dms / args.steps * 1e-3
    ach = dwork / dsec / (1e9 if fr[dom]["bound"] == "hbm" else 1e12)
    pk = fr[dom]["peak"]
    roof = {"kernel": STAGE_KERNELS.get(dom, dom), "stage": dom, "bound": fr[dom]["bound"], "achieved": ach,
            "peak": pk, "unit": fr[dom]["unit"], "frac": ach / pk, "traffic": None,
            "peak_source": (f"{src} bf16_tflops_sustained" if fr[dom]["bound"] == "tensor" else
                            f"{src} hbm_gbs" if fr[dom]["bound"] == "hbm" else
                            "derived: FP32 FMA lanes 152 SMs x 128 x 2 FLOP x 2.07 GHz"),
            "algorithmic": "the stage's work summed over the batch's datasets (see stages)",
            "launches_timed": dn, "share_of_step": dms / args.steps / (elapsed_ms / args.steps),
            "timing": f"{args.steps} eager calls with only this stage's launches event-bracketed, after the "
                      f"graph replays"}

    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16-gemm/f32/f32x2-refine" if prec == "bf16_mixed" else "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w['desc']}", "datasets": len(sets), "points": npts,
                       "m_mean": float(np.mean([sh[1] for sh in shapes])),
                       "k_mean": float(np.mean(ks)), "variant": var, "precision": prec,
                       "l2": "inputs larger than L2 (%.1f GB in all)" % (in_bytes / 1e9),
                       "parallelism": f"replicas x{world}", "tuned": tuned,
                       "timing": "one step = one replay of a CUDA graph of the batched call; stage table from one "
                                 "eager call with every launch bracketed"},
            "roofline": roof, "gpu_launches": launches_per_call * args.steps, "launches_per_call": launches_per_call,
            "clocks": clk, "status": status, "stages": fr,
            "knn_stats": {kk: stats[kk] for kk in ("knn_uncertified", "knn_fallback_rows", "jacobi_max_sweeps",
                                                  "jacobi_not_converged", "rank_deficient", "jacobi_rotations")}}

    # sampled rows for the accuracy check and the oracle's timing
    rng = np.random.default_rng(7)
    pick = rng.choice(len(sets), min(args.cpu_sets, len(sets)), replace=False)
    rows = {int(i): np.sort(rng.choice(shapes[i][0], min(args.cpu_rows_per_set, shapes[i][0]), replace=False))
            for i in pick}
    chosen = {i: (idx_out[i].cpu().numpy()[r], kap_g[i].cpu().numpy()[r]) for i, r in rows.items()}
    plain = None
    if rank == 0 and not args.no_plain and prec != "fp32":
        kf = ctx.mecuco_curvature_batched(Xs, ks, precision="fp32", variant=var)
        torch.cuda.synchronize()
        idx_f = [torch.empty_like(t) for t in idx_out]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kf = ctx.mecuco_curvature_batched(Xs, ks, precision="fp32", variant=var, idx_out=idx_f)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {i: (idx_f[i].cpu().numpy()[r], kf[i].cpu().numpy()[r]) for i, r in rows.items()}
        line["plain_fp32"] = {"value": npts / (pms * 1e-3), "unit": "points/s",
                              "sample": f"the whole batch in the plain FP32 form (stream lanes), one eager call; "
                                        f"{pms:.0f} ms",
                              "chosen_over_plain": value / world / (npts / (pms * 1e-3))}

    if rank == 0 and not args.no_e2e:
        kap_h = [torch.empty(n, dtype=torch.float32).pin_memory() for n, _, _ in shapes]

        def e2e_step():
            for xd, xh in zip(Xs, Xh):
                xd.copy_(xh, non_blocking=True)
            kk = call()
            for a, b in zip(kap_h, kk):
                a.copy_(b, non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        dt = time.perf_counter() - t0
        line["e2e"] = {"value": npts * args.e2e_steps / dt, "unit": "points/s", "h2d_bytes_per_step": int(in_bytes),
                       "d2h_bytes_per_step": int(npts * 4), "steps": args.e2e_steps,
                       "ms_per_step": dt / args.e2e_steps * 1e3,
                       "path": "per step: pinned-host to device copy of every dataset, one eager batched call "
                               "(public Python binding over the C ABI), device to pinned-host copy of every kappa"}

    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        ref = {}
        for i, r in rows.items():
            X = sets[i]["X"]
            ridx, rd = oracle.knn(X, ks[i], rows=r, nthreads=cores)
            full = np.zeros((X.shape[0], ks[i]), dtype=np.int32)
            full[r] = ridx
            ref[i] = (ridx, rd, oracle.curvature(X, ks[i], full, rows=r, nthreads=cores))
        dt = time.perf_counter() - t0
        nrows = sum(len(r) for r in rows.values())
        line["cpu_baseline"] = {"value": nrows / dt, "unit": "points/s", "cores": cores, "kind": "oracle",
                                "sample": f"{nrows} random rows of {len(rows)} random datasets of the batch, each a "
                                          f"brute-force FP64 kNN scan of its dataset plus the FP64 Fast estimator; "
                                          f"{dt:.1f} s"}

        def acc_of(got):
            errs, bad = [], 0
            for i, r in rows.items():
                a = _accuracy(sets[i]["X"], "f32", r, got[i][0], got[i][1], *ref[i])
                bad += a["knn_mismatch_rows"]
                errs.append(np.abs(np.asarray(got[i][1], np.float64) - ref[i][2]) / np.abs(ref[i][2]))
            e = np.concatenate(errs)
            return {"kappa_max_rel": float(e.max()), "kappa_median_rel": float(np.median(e)),
                    "knn_mismatch_rows": int(bad), "rows": int(e.size)}

        acc = {"reference": "FP64 oracle: brute-force kNN over each dataset, Alg. 1 Fast branch on its lists",
               "tie_rule": "list positions may differ only between distances equal within 1e-6 relative",
               "chosen": acc_of(chosen)}
        if plain is not None:
            acc["plain_fp32"] = acc_of(plain)
        line["accuracy"] = acc

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
    ap.add_argument("--jacobi-fp64", type=int, choices=[0, 1, 2], default=None)
    ap.add_argument("--plain-rows", type=int, default=4096)
    ap.add_argument("--cpu-rows", type=int, default=32)
    ap.add_argument("--cpu-sets", type=int, default=16, help="batched workload: datasets sampled for the oracle")
    ap.add_argument("--cpu-rows-per-set", type=int, default=4)
    ap.add_argument("--ref-rows", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-rows", type=int, default=16384)
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
