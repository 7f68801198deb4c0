#!/usr/bin/env python
"""Benchmark: dense symmetric EVD (eigenvalues + eigenvectors) on GB300.

One step = one whole solve A -> (Lambda, Q) through the C ABI: SBR (panel QR + Eq. 1
trailing update), bulge chasing, divide and conquer, back transformation, on a
synthetic A = Q Lambda Q^T with a known spectrum.  The metric is effective TFLOP/s
with the tridiagonalization counted as 4n^3/3 and the back transformation as 2n^3;
seconds per solve are in the JSON line too.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--n N] [--prec fp64|split_bf16]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

Multi-GPU: one process per GPU (torchrun); the single-matrix EVD does not shard, so
each rank solves its own replica ("replicas only") and the value is the whole-job
throughput, timed as the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import signal
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "n=49152 EVD seconds & effective TFLOPS; split-precision vs FP64 at equal residual"
DEFAULT_N = 49152
FP64_ALU_PEAK_TFLOPS = 1.26  # FP64 CUDA-core rate of GB300: 152 SMs x 2 FMA/clk x 2 x 2.07 GHz


AUTOTUNE_FILE = ROOT / "paper_2511_16174_gb300" / "autotune_gb300.json"


def tuned_entry(n, job=1, prec=0):
    """The autotuner's cached (b, nb) for n's power-of-two bucket in the committed
    cache (measured on GB300), or None."""
    try:
        entries = json.loads(AUTOTUNE_FILE.read_text())
    except Exception:
        return None
    bucket = 1 << int(round(np.log2(max(n, 1))))
    for e in entries:
        if e["n_bucket"] == bucket and e["job"] == job and e["prec"] == prec:
            return e
    return None


def nominal_flops(n):
    return 4.0 * n ** 3 / 3.0 + 2.0 * n ** 3


def workload_name(n, prec):
    spec = "geometric 1..1e-8 random signs" if n <= 8192 else "uniform [-1,1]"
    return (f"n={n} {'FP64' if prec == 'fp64' else 'split-BF16+refinement'} EVD with eigenvectors, "
            f"A=Q Lambda Q^T, Q = 32 seeded Householder reflectors, Lambda {spec}")


def spectrum_for(n, seed):
    from paper_2511_16174_gb300 import inputs
    if n <= 8192:
        return inputs.spectrum_geometric(n, seed)
    return inputs.spectrum_uniform(n, seed)


def load_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def dgemm_peak():
    """The FP64 DGEMM rate measured on this GPU (profiles/fp64_dgemm_peak.json), or None."""
    p = ROOT / "profiles" / "fp64_dgemm_peak.json"
    try:
        return float(json.loads(p.read_text())["tflops"])
    except Exception:
        return None


def committed_traffic(kernel_cat, n, tiles_per_launch=None):
    """DRAM bytes per launch from a committed ncu summary (profiles/traffic.json),
    if the kernel's sources are unchanged since the capture (else None).  An entry
    holds either bytes per launch for one n, or bytes per tile (a tile's traffic
    does not depend on n), scaled here by the tiles one launch processes."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    try:
        d = json.loads(p.read_text())
    except Exception:
        return None
    ent = d.get("kernels", {}).get(kernel_cat)
    if not ent:
        return None
    if "dram_bytes_per_tile" not in ent and ent.get("n") != n:
        return None
    h = hashlib.sha256()
    for f in ent.get("sources", []):
        q = ROOT / f
        if not q.exists():
            return None
        h.update(f.encode())
        h.update(q.read_bytes())
    if h.hexdigest()[:16] != ent.get("src_hash"):
        return None
    if "dram_bytes_per_tile" in ent:
        return None if tiles_per_launch is None else ent["dram_bytes_per_tile"] * tiles_per_launch
    return ent.get("dram_bytes_per_launch")


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGINT)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in Path(self.path).read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def run_oracle_sample(target_s=15.0):
    """Time the CPU oracle (one-stage tridiagonalization + implicit QL with
    vectors) on a bounded sample of the workload: the same construction (A = Q
    Lambda Q^T, Lambda uniform in [-1, 1]) at the size ns that takes about target_s
    seconds.  Returns (tflops, ns, seconds, cores)."""
    import oracle
    from paper_2511_16174_gb300 import inputs
    n0 = 768
    A = inputs.qlq(inputs.spectrum_uniform(n0, 1), 2)
    t = time.perf_counter()
    oracle.eigh(A, want_vectors=True)
    t0 = time.perf_counter() - t
    ns = int(n0 * (target_s / max(t0, 1e-3)) ** (1.0 / 3.0))
    ns = max(512, min(4096, ns // 64 * 64))
    A = inputs.qlq(inputs.spectrum_uniform(ns, 3), 4)
    t = time.perf_counter()
    oracle.eigh(A, want_vectors=True)
    ts = time.perf_counter() - t
    return nominal_flops(ns) / ts / 1e12, ns, ts, oracle.num_threads()


def sample_text(ns, secs):
    return (f"one-stage Householder + implicit QL with vectors on the same construction at n={ns} "
            f"(A = Q Lambda Q^T, Lambda uniform [-1,1]), {secs:.1f} s per solve; flops counted as 4n^3/3+2n^3")


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reference_arm(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return 0
    n = args.n
    vals, times = [], []
    for i in range(args.warmup + args.steps):
        tf, ns, ts, cores = run_oracle_sample(target_s=min(20.0, 120.0 / max(1, args.warmup + args.steps)))
        if i >= args.warmup:
            vals.append(tf)
            times.append(ts)
    v = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(times)) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"CPU oracle on a bounded sample of the n={n} workload: each step one solve at "
                               f"n={ns} of the same construction, TFLOP/s of that sample (not an n={n} solve)",
                   "n": n, "sample_n": ns, "job": "V", "prec": args.prec},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample_text(ns, float(np.mean(times)))},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ours(args):
    import torch
    import torch.distributed as dist

    ws_, rank, local = dist_setup()
    if ws_ > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    # plans created with b = nb = 0 take the autotuner's entry for their size
    os.environ.setdefault("EVD_AUTOTUNE_CACHE", str(AUTOTUNE_FILE))
    from paper_2511_16174_gb300 import evd, inputs

    n = args.n
    seed = inputs.SEED_BASE + (2 if n > 8192 else 1)
    lam = np.sort(spectrum_for(n, seed))
    if n <= 8192:
        A0 = evd.as_colmajor(torch.from_numpy(inputs.qlq(lam, seed)).cuda())
    else:
        A0 = evd.as_colmajor(inputs.qlq_device(lam, seed))
    torch.cuda.synchronize()
    # The step's input lives in pinned host memory; A is symmetric, so the row-major
    # host copy of the column-major device matrix holds the same values.
    Ah = torch.empty((n, n), dtype=torch.float64).pin_memory()
    Ah.copy_(A0.t())
    del A0
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    options = {}
    if args.refine_iters is not None:
        options["refine_iters"] = args.refine_iters
    if args.order is not None:
        options["order"] = args.order
    plan = evd.Plan(n, job="V", prec=args.prec, b=args.b, nb=args.nb, stream=stream, options=options)
    ws = plan.workspace()
    Aw = evd.empty_colmajor(n, n)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    Q = evd.empty_colmajor(n, n)
    wh = torch.empty(n, dtype=torch.float64).pin_memory()
    Qh = torch.empty((n, n), dtype=torch.float64).pin_memory()
    Aw_rm = Aw.t()  # row-major view of the column-major buffer

    def step(ev=None):
        """One step through the public API: host -> device copy of A, the solve,
        device -> host copy of w and Q (the row-major host Qh holds Q^T)."""
        if ev:
            ev[0].record(stream)
        Aw_rm.copy_(Ah, non_blocking=True)
        if ev:
            ev[1].record(stream)
        plan.syevd(Aw, w, Q, ws)
        if ev:
            ev[2].record(stream)
        wh.copy_(w, non_blocking=True)
        Qh.copy_(Q.t(), non_blocking=True)
        if ev:
            ev[3].record(stream)

    for i in range(args.warmup):
        step()
        if i == 0:
            plan.check("warmup solve")
    torch.cuda.synchronize()
    if ws_ > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    evd.stats_reset()
    evd.stats_enable(not args.no_stats)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    if ws_ > 1:
        dist.barrier()
    torch.cuda.nvtx.range_push("timed_steps")  # ncu --nvtx-include "timed_steps/" takes exactly these launches
    for k in range(args.steps):
        step(evs[k])
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws_ > 1:
        dist.barrier()
    evd.stats_enable(False)
    launches = evd.launch_count()
    clk = clocks.stop()
    plan.check("timed solves")
    # value: the solves alone (inputs resident in HBM); e2e: the whole steps
    ms = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    ems = evs[0][0].elapsed_time(evs[-1][3]) / args.steps
    h2d_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    d2h_ms = sum(e[2].elapsed_time(e[3]) for e in evs) / args.steps
    st = evd.stats()
    if ws_ > 1:
        t = torch.tensor([ms, ems], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ems = float(t[0].item()), float(t[1].item())
    value = nominal_flops(n) / (ms / 1e3) / 1e12 * ws_
    e2e = {"value": nominal_flops(n) / (ems / 1e3) / 1e12 * ws_, "unit": "TFLOP/s",
           "h2d_bytes_per_step": 8 * n * n, "d2h_bytes_per_step": 8 * n + 8 * n * n,
           "ms_per_step": ems, "h2d_ms": h2d_ms, "d2h_ms": d2h_ms}

    # ---- accuracy of the last timed result (sampled columns at large n); A is
    # copied back into the solve's input buffer from the host copy
    with torch.no_grad():
        Aw_rm.copy_(Ah)
        A0 = Aw
        lam_t = torch.from_numpy(lam).cuda()
        dlam = float((w - lam_t).abs().max().item())
        gen = torch.Generator(device="cuda")
        gen.manual_seed(n)
        cols = (torch.arange(n, device="cuda") if n <= 8192
                else torch.randperm(n, device="cuda", generator=gen)[:256])
        Qs = Q[:, cols]
        R = A0 @ Qs - Qs * w[cols][None, :]
        O = Q.t() @ Qs
        O[cols, torch.arange(len(cols), device="cuda")] -= 1.0
        normA = float(torch.linalg.matrix_norm(A0).item())
        resid = float(torch.linalg.matrix_norm(R).item()) / (n * normA) * (n / len(cols)) ** 0.5
        orth = float(O.abs().max().item())
        # the host copy of the result is the device result
        host_ok = bool(torch.equal(Qh[cols.cpu()].t().contiguous(), Qs.cpu()) and torch.equal(wh, w.cpu()))
        del R, O, Qs
    U = 2.0 ** -53
    acc = {"dlam": dlam, "dlam_bound": 10 * n * U * float(np.max(np.abs(lam))), "orth_max": orth,
           "orth_bound": 10 * n * U, "resid": resid, "resid_bound": 10 * U,
           "columns_checked": int(len(cols)), "host_copy_matches": host_ok}
    acc["within_bounds"] = bool(acc["dlam"] <= acc["dlam_bound"] and acc["orth_max"] <= acc["orth_bound"]
                                and acc["resid"] <= acc["resid_bound"])

    # ---- roofline of the dominant kernel category
    # Categories are "stage/engine" for products ("/tc_split": tensor-core split
    # product, executed bf16 flops; "/fp64_simt", "/fp64_splitk": FP64 CUDA cores)
    # and plain stage names for the other kernels.  Bulge chasing carries both its
    # FP64 flop count and the byte model 16 b n^2 (+4 n^2 for U).
    peaks, peak_kind = load_peaks()
    # the dominant kernel among the stages on the plan's own streams (in the reordered
    # order D&C runs beside the back transformation on a low-priority stream, and its
    # event times include the waiting for SMs there)
    reordered = plan.option("order") == 1
    main = {k: v for k, v in st.items()
            if not k.endswith("/tc_split_prep") and not (reordered and k.startswith("dc_"))}
    dom = max(main.items(), key=lambda kv: kv[1][0], default=None) if main else None
    roof = None
    if dom:
        cat, (dms, dfl, dby, dca) = dom
        per_launch_ms = dms / max(dca, 1)
        tiles = dby / (16.0 * 127 * 128) / max(dca, 1) if cat.startswith("bc_back_wave") else None
        traffic = committed_traffic(cat, n, tiles)
        secs = dms / 1e3
        if cat.endswith("/tc_split"):
            peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
            roof = {"kernel": cat, "bound": "tensor", "achieved": dfl / secs / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "traffic": traffic,
                    "peak_source": f"{peak_kind} MEASURED_PEAKS.json bf16_tflops_sustained (executed 16-bit "
                                   f"tensor flops of the slice-pair products: bfloat16 slices in the general "
                                   f"product, float16 digits in the fused BC-Back waves, both at the bf16 rate)"}
            # the same work as FP64 flops: slice pairs per FP64 flop (general product: 8
            # slices, 36 pairs, 6 in split precision, 21 pairs; fused waves: 7 digits,
            # 28 pairs, in both precisions)
            if cat.startswith("bc_back_wave"):
                pairs = 28.0
            else:
                pairs = 36.0 if args.prec == "fp64" else 21.0
            roof["fp64_equiv_tflops"] = dfl / pairs / secs / 1e12
            dg = dgemm_peak()
            if dg:
                roof["fp64_dgemm_peak_tflops"] = dg
                roof["frac_of_dgemm_peak"] = roof["fp64_equiv_tflops"] / dg
        else:
            roof = {"kernel": cat, "bound": "alu", "achieved": dfl / secs / 1e12, "peak": FP64_ALU_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "traffic": traffic,
                    "peak_source": "FP64 CUDA-core rate 152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz = 1.26 TFLOP/s"}
            if dby > 0:
                roof["hbm_model_gbs"] = dby / secs / 1e9
                roof["hbm_model_frac"] = roof["hbm_model_gbs"] / peaks.get("hbm_gbs")
        roof["frac"] = roof["achieved"] / roof["peak"] if roof["peak"] else None
        roof["launches"] = int(dca)
        roof["ms_per_launch"] = per_launch_ms
        roof["share_of_step"] = dms / (ms * args.steps) if ms > 0 else None
    breakdown = {k: {"ms": v[0] / args.steps, "calls": v[3] // max(args.steps, 1)} for k, v in st.items()}

    cpu = None
    if rank == 0 and ws_ == 1 and not args.no_cpu:
        tf, ns, ts, cores = run_oracle_sample()
        cpu = {"value": tf, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample_text(ns, ts)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws_, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(n, args.prec), "n": n, "job": "V", "prec": args.prec,
                       "b": plan.b, "nb": plan.nb,
                       "blocking": ("autotuner cache " + os.path.basename(os.environ["EVD_AUTOTUNE_CACHE"])
                                    if args.b == 0 and args.nb == 0
                                    and tuned_entry(n, 1, 0 if args.prec == "fp64" else 2) is not None
                                    and os.path.abspath(os.environ["EVD_AUTOTUNE_CACHE"]) == str(AUTOTUNE_FILE)
                                    else "library default rule" if args.b == 0 and args.nb == 0 else "given"),
                       "seconds_per_solve": ms / 1e3,
                       "paper_tflops_4n3": 4.0 * n ** 3 / (ms / 1e3) / 1e12,
                       "refine_iters": plan.option("refine_iters") if args.prec != "fp64" else 0,
                       "order": "reordered (Sec. 3.3)" if plan.option("order") == 1 else "conventional",
                       "l2": "inputs larger than L2 (A is 8 n^2 bytes)", "parallelism": f"replicas{ws_}"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "accuracy": acc, "stages": breakdown,
        }
        print(json.dumps(line), flush=True)
    if ws_ > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _oracle_values(job):
    """Worker of the batched check: the oracle's eigenvalues of one batch matrix,
    rebuilt from its size and seed (single-threaded)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle
    from paper_2511_16174_gb300 import inputs
    n, seed = job
    w, _ = oracle.eigh(inputs.goe(n, seed), want_vectors=False)
    return np.asarray(w)


def batch_mode(args):
    """The batched configuration: 512 symmetric matrices (G + G^T) / 2, n drawn
    log-uniformly from 64 to 2048, eigenvalues and eigenvectors, one captured graph
    per run, against a loop of single evd_syevd calls on the same buffers.  One JSON
    line (matrices per second); every result is checked on the GPU against the
    acceptance bounds, and every matrix's eigenvalues against the CPU oracle."""
    import torch
    from paper_2511_16174_gb300 import evd, inputs
    torch.cuda.set_device(0)
    count = args.batch
    sizes = [int(x) for x in inputs.batch_sizes(count, inputs.SEED_BASE + 5)]
    batch = evd.Batch(sizes, job="V")
    # host-generated (so that the oracle's workers can rebuild each matrix from its
    # size and seed), then resident on the device
    A0 = [evd.as_colmajor(torch.from_numpy(inputs.goe(n, inputs.SEED_BASE + 1000 + i)).cuda())
          for i, n in enumerate(sizes)]
    stream = torch.cuda.current_stream()

    def refill():
        for a, t in zip(A0, batch.A):
            t.copy_(a)

    def run_batch():
        refill()
        batch.run(stream)

    plans = [evd.Plan(n, job="V", stream=stream) for n in sizes]
    wss = [p.workspace() for p in plans]

    def run_loop():
        refill()
        for p, ws, a, w, q in zip(plans, wss, batch.A, batch.w, batch.Q):
            p.syevd(a, w, q, ws)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, (time.perf_counter() - t0) / args.steps * 1e3

    clocks = ClockSampler(0)
    clocks.start()
    ms_loop, wall_loop = timed(run_loop)
    for p in plans:
        p.check("loop solve")
    ms_batch, wall_batch = timed(run_batch)
    clk = clocks.stop()
    graph = evd.batched_last_graph()
    # accuracy of the last batched run: every matrix on the GPU, a sample against the oracle
    U = 2.0 ** -53
    worst = {"dlam_ratio": 0.0, "orth_ratio": 0.0, "resid_ratio": 0.0}
    with torch.no_grad():
        for a, w, q, n in zip(A0, batch.w, batch.Q, sizes):
            O = q.t() @ q
            O.diagonal().sub_(1.0)
            orth = float(O.abs().max())
            R = a @ q - q * w[None, :]
            resid = float(torch.linalg.matrix_norm(R) / (n * torch.linalg.matrix_norm(a)))
            worst["orth_ratio"] = max(worst["orth_ratio"], orth / (10 * n * U))
            worst["resid_ratio"] = max(worst["resid_ratio"], resid / (10 * U))
    # every matrix's eigenvalues against the CPU oracle, in spawned single-threaded workers
    import multiprocessing as mp
    jobs = [(n, inputs.SEED_BASE + 1000 + i) for i, n in enumerate(sizes)]
    t_or = time.perf_counter()
    with mp.get_context("spawn").Pool(processes=max(1, min(os.cpu_count() or 1, 32))) as pool:
        refs = pool.map(_oracle_values, jobs, chunksize=1)
    t_or = time.perf_counter() - t_or
    for i, w_ref in enumerate(refs):
        dl = float(np.max(np.abs(batch.w[i].cpu().numpy() - w_ref))) if sizes[i] else 0.0
        worst["dlam_ratio"] = max(worst["dlam_ratio"],
                                  dl / (10 * sizes[i] * U * max(float(np.max(np.abs(w_ref))), 1e-300)))
    sample = list(range(count))
    flops = sum(nominal_flops(n) for n in sizes)
    line = {
        "metric": "batched EVD matrices per second (512 matrices, n log-uniform in [64, 2048])",
        "value": count / (ms_batch / 1e3), "unit": "matrices/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{count} x (G+G^T)/2, n log-uniform in [64, 2048] (sum n = {sum(sizes)}), "
                               f"eigenvalues and eigenvectors, FP64",
                   "captured_graph": graph, "tflops_nominal": flops / (ms_batch / 1e3) / 1e12},
        "loop_of_single_solves": {"value": count / (ms_loop / 1e3), "unit": "matrices/s", "ms_per_step": ms_loop,
                                  "host_wall_ms": wall_loop},
        "batched_over_loop": ms_loop / ms_batch, "host_wall_ms": wall_batch,
        "accuracy": {**worst, "oracle_checked": len(sample), "oracle_seconds": t_or,
                     "within_bounds": all(v <= 1.0 for v in worst.values())},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def profile_target(args):
    """A small, untimed run for ncu captures (no JSON line)."""
    import torch
    from paper_2511_16174_gb300 import evd, inputs
    n = args.n
    g = torch.Generator(device="cuda").manual_seed(inputs.SEED_BASE)
    if args.profile == "gemm":
        A = evd.empty_colmajor(n, n)
        B = evd.empty_colmajor(n, n)
        C = evd.empty_colmajor(n, n)
        A.copy_(torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g))
        B.copy_(torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g))
        for _ in range(2):
            evd.dgemm("N", "N", 1.0, A, B, 0.0, C, slices=8 if args.prec == "fp64" else 6)
    else:
        lam = np.sort(spectrum_for(n, inputs.SEED_BASE + 1))
        A = evd.as_colmajor(torch.from_numpy(inputs.qlq(lam, inputs.SEED_BASE + 1)).cuda()) if n <= 8192 else \
            evd.as_colmajor(inputs.qlq_device(lam, inputs.SEED_BASE + 1))
        options = {"order": args.order} if args.order is not None else None
        evd.syevd(A, job="V", prec=args.prec, b=args.b, nb=args.nb, options=options)
    torch.cuda.synchronize()
    print("profile target done", flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=DEFAULT_N)
    ap.add_argument("--prec", choices=["fp64", "split_bf16"], default="fp64")
    ap.add_argument("--b", type=int, default=0)
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--refine-iters", type=int, default=None, help="refinement steps of the split form")
    ap.add_argument("--batch", type=int, default=0,
                    help="the batched configuration with this many matrices (512) instead of the single solve")
    ap.add_argument("--order", type=int, default=None, choices=[0, 1],
                    help="back transformation: 0 conventional, 1 reordered (default: the library's choice)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-stats", action="store_true", help="no per-category event timing in the timed region")
    ap.add_argument("--profile", choices=["gemm", "solve"], default=None,
                    help="untimed target for a profiler: one N^3 split product (N = --n) twice, or one solve")
    args = ap.parse_args()
    if args.profile:
        return profile_target(args)
    if args.batch:
        return batch_mode(args)
    if args.impl == "reference":
        return reference_arm(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
