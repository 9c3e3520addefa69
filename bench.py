#!/usr/bin/env python3
"""FR-ADM throughput on one GB300: solves/s of the 16384 x 16384, r = 64 workload.

One step = one full FR-ADM solve (Algorithm 1 to ||M - L - S||_F / ||M||_F <= 1e-9)
of a seeded 16384 x 16384 rank-64 matrix with 5% outliers in [-50, 50], stored in
bfloat16, on the mixed path (float32 sweep, float64 r x r projectors), through
the libsfr C ABI with inputs resident in HBM.  Inputs (512 MB M, 2 x 1 GB
multiplier buffers) are larger than the 129 MB L2, so no flush is needed.

Printed (rank 0, one JSON line): value = solves/s over all ranks; roofline of the
fused sweep kernel (algorithmic bytes / event-timed duration, against the measured
HBM copy bandwidth); e2e = the same metric through the C ABI with host buffers
(host -> device copy of M and device -> host copy of S inside the timed region);
cpu_baseline = the FP64 CPU oracle on a bounded sample of the same recipe.

--impl reference times that oracle alone (the slow reference program).
Multi-GPU (torchrun): replicas only, each rank solves its own problem; no collective
on the data path (barrier + max of the elapsed time only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="square16384_r64_bf16_mixed", m=16384, n=16384, r=64, storage="bf16", precision="mixed",
                outlier_fraction=0.05, outlier_range=[-50, 50], mu0=0.05, rho=1.5, tol=1e-9, max_iter=300,
                l2="inputs larger than L2 (M 512 MB, multipliers 2 x 512 MB, Delta 512 MB); no flush")
SAMPLE = dict(m=4096, n=4096)          # CPU oracle sample of the same recipe (about 10 s on 16 Arm cores)
REF_SAMPLE = dict(m=2048, n=2048)      # one step of the reference arm (about 2.5 s on 16 Arm cores)
FALLBACK_HBM_GBS = 6800.0


def sweep_traffic(m: int, n: int):
    """DRAM bytes of one sweep launch from the committed ncu summary, scaled by m n.

    The summary records bytes per element and the hashes of the kernel's source (the part of
    its file before `source_until`, which holds the sweep kernel, its constants and helpers) and
    of the shared tensor-core helpers; if either has changed since, the figure no longer applies
    and None is returned.
    """
    import hashlib
    keys = ("traffic_bytes_per_element", "source", "source_until", "source_sha256", "helpers", "helpers_sha256")
    try:
        with open(os.path.join(ROOT, "profiles", "sweep_tc_square8192_r64_bf16.md")) as f:
            kv = dict(line.strip().split(": ", 1) for line in f if line.startswith("    ") and ": " in line
                      and line.strip().split(": ", 1)[0] in keys)
        with open(os.path.join(ROOT, kv["source"]), encoding="utf-8") as f:
            text = f.read()
        region = text[:text.index(kv["source_until"])]
        if hashlib.sha256(region.encode("utf-8")).hexdigest() != kv["source_sha256"]:
            return None
        with open(os.path.join(ROOT, kv["helpers"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != kv["helpers_sha256"]:
                return None
        return float(kv["traffic_bytes_per_element"]) * m * n
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].lower().startswith("active")})
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def make_workload(seed: int):
    from paper_1503_03004_gb300 import synth
    return synth.square_large(WORKLOAD["m"], WORKLOAD["r"], dtype="bf16", seed=seed)  # m = n


def host_cpu():
    """(threads available to this process, CPU model name from lscpu or /proc/cpuinfo)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return cores, model or platform.machine()


def oracle_sample_rate(seed: int = 1001, sample=None):
    """FP64 CPU oracle on a sample of the same recipe (default SAMPLE, 4096 x 4096), scaled to
    full-size solves/s.

    FR-ADM costs O(m n r) per iteration and needs a similar iteration count at both sizes
    (42 at 4096^2, 41 at 16384^2), so the full-size time is taken as the sample's solve time x
    (m n of the workload / m n of the sample).
    """
    sample = sample or SAMPLE
    import numpy as np
    from oracle import fradm as O
    from paper_1503_03004_gb300 import synth
    p = synth.planted(sample["m"], sample["n"], WORKLOAD["r"], p=WORKLOAD["outlier_fraction"], amp=50.0, seed=seed,
                      dtype="bf16")
    M = p.values_f64()
    t0 = time.perf_counter()
    res = O.fr_adm(M, WORKLOAD["r"], rho=WORKLOAD["rho"], mu0=WORKLOAD["mu0"], tol=WORKLOAD["tol"],
                   max_iter=WORKLOAD["max_iter"])
    dt = time.perf_counter() - t0
    scale = (WORKLOAD["m"] * WORKLOAD["n"]) / (sample["m"] * sample["n"])
    cores, model = host_cpu()
    return {"value": 1.0 / (dt * scale), "unit": "solves/s", "cores": cores, "cpu_model": model, "kind": "oracle",
            "sample": (f"one FP64 oracle solve of a {sample['m']}x{sample['n']} r=64 sample of the same recipe "
                       f"({res.iters} iterations, {dt:.1f} s), scaled by m*n ({scale:g}x) to "
                       f"{WORKLOAD['m']}x{WORKLOAD['n']}"),
            "sample_iters": res.iters, "sample_seconds": dt, "scale": scale, "converged": bool(res.converged)}, np


def oracle_sample_error(U, Bm, V, S):
    """Relative error of L = U B V^T and of S at the float64 oracle's sampled positions of the
    16384^2 r = 64 bf16 workload (tests/golden/square16384_r64_bf16_samples.txt, written by
    tests/golden/make_fullsize_samples.py from the oracle alone), or None without that file."""
    import numpy as np
    import torch
    path = os.path.join(ROOT, "tests", "golden", "square16384_r64_bf16_samples.txt")
    if not os.path.exists(path):
        return None
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    a = np.array([[float(x) for x in t] for t in rows if len(t) == 5])
    ii = torch.from_numpy(a[:, 0].astype(np.int64)).to(U.device)
    jj = torch.from_numpy(a[:, 1].astype(np.int64)).to(U.device)
    L = torch.einsum("ka,ab,kb->k", U[ii], Bm, V[jj]).cpu().numpy()
    Sv = S[ii, jj].double().cpu().numpy()
    return {"rel_err_L": float(np.linalg.norm(L - a[:, 2]) / np.linalg.norm(a[:, 2])),
            "rel_err_S": float(np.linalg.norm(Sv - a[:, 3]) / np.linalg.norm(a[:, 3])),
            "bar": 1e-5, "samples": int(len(a)), "against": "float64 oracle (sampled positions)"}


def reduce_max(x: float, device=None) -> float:
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(steps: int, elapsed_ms: float) -> float:
    """Whole-job solves/s: every rank solves `steps` problems; time is the slowest rank's."""
    import torch.distributed as dist
    world = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    return world * steps / (reduce_max(elapsed_ms) / 1000.0)


def relaunch_cmd(argv, nproc: int, port: int):
    """Command that runs this script as `nproc` replica ranks (one process per GPU) under
    torch.distributed.run on this node, rendezvous on 127.0.0.1."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
            "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *argv]


def free_port() -> int:
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _serving_item(q):
    """Stored bfloat16 bits of one serving request's matrix (a pool worker: host work only)."""
    from paper_1503_03004_gb300 import synth
    return synth.planted(q.m, q.n, q.r, p=q.p, amp=50.0, seed=q.seed, dtype="bf16").M


def _serving_oracle(args):
    """Float64 oracle (Algorithm 1) of one serving request: L = U B V^T (a pool worker)."""
    q, kw = args
    from oracle import fradm as O
    from paper_1503_03004_gb300 import synth
    prob = synth.planted(q.m, q.n, q.r, p=q.p, amp=50.0, seed=q.seed, dtype="bf16")
    ref = O.fr_adm(prob.values_f64(), q.r, **kw)
    return ref.L, ref.iters, bool(ref.converged)


def run_serving(args):
    """Serving-stream workload: `--requests` uneven planted requests (default 4096: m in [256, 8192],
    n in [16, 512], r in {3, 5, 10, 25}, outliers 2-15 % in [-50, 50], bf16 storage), three ways:
      * serving: the mixed path through sfr_submit / sfr_poll, all requests queued at once
        (throughput), first through --slots slots (one solve per stream), then through the
        grouped engine (--max-batch problems iterated together, one grouped launch per kernel
        and iteration step), then again with Poisson arrivals at 70 % of the grouped rate
        (latency p50 / p99 from arrival to completion);
      * per-problem float64: sfr_solve one request at a time on the float64 path;
      * per-problem mixed: sfr_solve one request at a time on the mixed path.
    Only requests that end with SFR_OK count as solves; the line carries every outcome's count.
    Accuracy: on `--check` seeded requests (m n <= 2^20) the float64 oracle runs on the host and
    the serving (mixed) and per-problem float64 results are compared with it (relative error of
    L = U B V^T).  Inputs are on the device before timing.  Prints one JSON line (supplementary;
    the main benchmark line is the default mode)."""
    import multiprocessing as mproc
    import numpy as np
    from paper_1503_03004_gb300 import synth
    reqs = synth.request_stream(args.requests, rate_per_s=1000.0)
    kw = dict(rho=1.5, mu0=0.05, tol=1e-9, max_iter=300)
    g = synth.rng(77)
    small = [i for i, q in enumerate(reqs) if q.m * q.n <= (1 << 20)]
    check = sorted(int(i) for i in g.choice(small, size=min(args.check, len(small)), replace=False))
    # host work (inputs, and the oracle on the checked requests) in a spawn pool of single-threaded
    # workers, all before any CUDA call of this process and outside every timed region
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    try:
        with mproc.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            mats = pool.map(_serving_item, reqs, chunksize=16)
            refs = pool.map(_serving_oracle, [(reqs[i], kw) for i in check])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    import torch
    from paper_1503_03004_gb300 import binding as B
    torch.cuda.set_device(0)
    items = []
    for q, bits in zip(reqs, mats):
        Md = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()
        f64 = dict(dtype=torch.float64, device="cuda")
        out = dict(U=torch.empty((q.m, q.r), **f64), B=torch.empty((q.r, q.r), **f64),
                   V=torch.empty((q.n, q.r), **f64), S=torch.empty((q.m, q.n), dtype=torch.float32, device="cuda"))
        items.append((q, Md, out))
    del mats
    torch.cuda.synchronize()

    def mk(q, Md, out, prec):
        p = B.make_problem(m=q.m, n=q.n, r=q.r, M_ptr=Md.data_ptr(), m_dtype=B.BF16, precision=prec, **kw)
        res = B.make_result(U_ptr=out["U"].data_ptr(), B_ptr=out["B"].data_ptr(), V_ptr=out["V"].data_ptr(),
                            S_ptr=out["S"].data_ptr(), s_dtype=B.F32, lds=q.n)
        return p, res

    def rel_errs(refs):
        errs = []
        for k, (Lref, _, _) in zip(check, refs):
            out = items[k][2]
            L = (out["U"] @ out["B"] @ out["V"].T).cpu().numpy()
            errs.append(float(np.linalg.norm(L - Lref) / np.linalg.norm(Lref)))
        return errs

    def sequential(prec):
        counts = {}
        with B.Context(0) as ctx:
            for q, Md, out in items[:8]:  # warm-up: graphs, workspaces, tuned grids
                p, res = mk(q, Md, out, prec)
                ctx.solve(p, res)
            t0 = time.perf_counter()
            for q, Md, out in items:
                p, res = mk(q, Md, out, prec)
                st = ctx.solve(p, res)
                counts[B.STATUS_NAMES.get(st, str(st))] = counts.get(B.STATUS_NAMES.get(st, str(st)), 0) + 1
            wall = time.perf_counter() - t0
        return counts.get("OK", 0) / wall, counts

    def serving(rate, batch):
        with B.Context(0, max_slots=args.slots, hbm_budget_bytes=args.budget_gb << 30, max_batch=batch) as ctx:
            for q, Md, out in items[:max(args.slots, min(batch, 64))]:
                p, res = mk(q, Md, out, B.PREC_MIXED)
                ctx.poll(ctx.submit(p, res), -1)
            keep, pending, done, counts = [], {}, {}, {}

            def reap():
                for t in list(pending):
                    st = ctx.poll(t, 0)
                    if st == B.PENDING:
                        continue
                    k, ts = pending.pop(t)
                    name = B.STATUS_NAMES.get(st, str(st))
                    counts[name] = counts.get(name, 0) + 1
                    if st == B.OK:
                        done[k] = time.perf_counter() - ts

            t0 = time.perf_counter()
            for k, (q, Md, out) in enumerate(items):
                if rate:
                    wait = t0 + q.arrival_s * (1000.0 / rate) - time.perf_counter()
                    if wait > 0:
                        time.sleep(wait)
                p, res = mk(q, Md, out, B.PREC_MIXED)
                keep.append((p, res))
                ts = time.perf_counter()  # arrival (latency counts queueing at the client too)
                while True:
                    try:
                        pending[ctx.submit(p, res)] = (k, ts)
                        break
                    except B.SfrError as e:  # the library's queue is full: wait for completions
                        if e.status != B.E_BUSY:
                            raise
                        reap()
                        time.sleep(1e-4)
                reap()
            while pending:
                reap()
                time.sleep(1e-4)
            wall = time.perf_counter() - t0
            lat = sorted(v * 1000.0 for v in done.values()) or [float("nan")]
            return (counts.get("OK", 0) / wall, lat[len(lat) // 2], lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                    counts)

    thr_slots, _, _, counts_slots = serving(None, 0)
    err_slots = rel_errs(refs)  # results of the throughput run (mixed path, through the slots)
    if args.max_batch > 0:
        thr, _, _, counts = serving(None, args.max_batch)
        err_serving = rel_errs(refs)  # the grouped engine's results
    else:
        thr, counts, err_serving = thr_slots, counts_slots, err_slots
    rate = 0.7 * thr
    _, p50, p99, counts_lat = serving(rate, args.max_batch)
    f64, counts_f64 = sequential(B.PREC_FP64)
    err_f64 = rel_errs(refs)
    mix, counts_mix = sequential(B.PREC_MIXED)
    line = {"metric": "serving solves/s", "requests": len(items), "slots": args.slots,
            "max_batch": args.max_batch, "value": thr, "unit": "solves/s", "status_counts": counts,
            "slots_only": {"value": thr_slots, "status_counts": counts_slots,
                           "max_rel_err_L": max(err_slots)},
            "per_problem_fp64": f64, "per_problem_fp64_status_counts": counts_f64,
            "per_problem_mixed": mix, "per_problem_mixed_status_counts": counts_mix,
            "latency_ms_at_rate": {"rate_per_s": rate, "p50": p50, "p99": p99, "status_counts": counts_lat},
            "accuracy": {"against": "float64 oracle (Algorithm 1) on the host", "requests_checked": check,
                         "oracle_converged": all(c for _, _, c in refs),
                         "serving_mixed_max_rel_err_L": max(err_serving), "mixed_bar": 1e-5,
                         "per_problem_fp64_max_rel_err_L": max(err_f64), "fp64_bar": 1e-9},
            "config": {"workload": "serving_stream", "m": [256, 8192], "n": [16, 512], "r": [3, 5, 10, 25],
                       "outlier_fraction": [0.02, 0.15], "storage": "bf16", "tol": 1e-9,
                       "solves_counted": "status OK only"}}
    print(json.dumps(line), flush=True)
    return 0


def run_opt_full(args):
    """FixedRankOptFull (Algorithm 4) as a truncated-SVD replacement on the benchmark's matrix
    (16384 x 16384 bf16, r = 64): one step = one call of sfr_fixed_rank_opt_full from V_0 = I,
    B_0 = I until ||B_i - B_{i-1}||_F <= 1e-6 ||B_i||_F (mixed path: tensor-core P = M V and
    W = M^T U passes).  Inputs are on the device before timing (M is larger than L2).  Reports
    TSVDs/s, the two passes against the HBM roofline (each reads M once: 2 B per element), the
    float64 oracle's Algorithm 4 on the same matrix, and the same call with host buffers (e2e).
    Prints one JSON line (supplementary; the main benchmark line is the default mode)."""
    import numpy as np
    import torch
    from paper_1503_03004_gb300 import binding as B
    torch.cuda.set_device(0)
    m = n = args.m
    r, tol, cap = WORKLOAD["r"], 1e-6, 50
    prob = make_workload(1001) if m == WORKLOAD["m"] else None
    if prob is None:
        from paper_1503_03004_gb300 import synth
        prob = synth.square_large(m, r, dtype="bf16", seed=1001)
    Md = torch.from_numpy(prob.M.view(np.int16)).view(torch.bfloat16).cuda()
    hbm, src = peaks()
    with B.Context(0, profile=True) as ctx:
        for _ in range(args.warmup):
            B.opt_full_torch(ctx, Md, r, tol=tol, max_iter=cap, precision=B.PREC_MIXED)
        torch.cuda.synchronize()
        ctx.stats(reset=True)
        iters = []
        with ClockSampler(0) as clk:
            t0 = time.perf_counter()
            for _ in range(args.steps):
                sol = B.opt_full_torch(ctx, Md, r, tol=tol, max_iter=cap, precision=B.PREC_MIXED)
                iters.append(sol.iters)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        st = ctx.stats()
        # e2e: the same call with host buffers (H2D of M and D2H of U, B, V inside the timed region)
        Mh = torch.from_numpy(prob.M.view(np.int16)).pin_memory()
        U = torch.empty((m, r), dtype=torch.float64).pin_memory()
        Bh = torch.empty((r, r), dtype=torch.float64).pin_memory()
        V = torch.empty((n, r), dtype=torch.float64).pin_memory()
        hp = B.OptFullProblem(m=m, n=n, ldm=n, r=r, m_dtype=B.BF16, M=Mh.data_ptr(), V0=None, B0=None, tol=tol,
                              max_iter=cap, precision=B.PREC_MIXED, mem=B.MEM_HOST)
        hr = B.OptFullResult(U=U.data_ptr(), B=Bh.data_ptr(), V=V.data_ptr())
        ctx.opt_full(hp, hr)
        t1 = time.perf_counter()
        for _ in range(args.e2e_steps):
            if ctx.opt_full(hp, hr) != B.OK:
                raise RuntimeError(ctx.last_error())
        e2e = args.e2e_steps / (time.perf_counter() - t1)
    pp, wp = st[B.STAT_PPASS], st[B.STAT_WPASS]
    p_ms = pp["total_ms"] / max(1, pp["timed"])
    w_ms = wp["total_ms"] / max(1, wp["timed"])
    achieved = (pp["bytes"] / max(1, pp["timed"])) / (p_ms * 1e-3) / 1e9
    line = {"metric": "TSVDs/s", "value": args.steps / dt, "unit": "TSVDs/s", "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps, "higher_is_better": True,
            "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": f"square{m}_r{r}_bf16_opt_full", "m": m, "n": n, "r": r, "storage": "bf16",
                       "precision": "mixed", "stop": f"||B_i - B_(i-1)||_F <= {tol} ||B_i||_F", "max_iter": cap,
                       "iters_per_step": sorted(set(iters)), "l2": f"M {m * n * 2 >> 20} MB, larger than L2; no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": "P pass (ppass_tc_kernel)", "bytes_per_element": 2.0,
                         "avg_launch_ms": p_ms, "timed_launches": pp["timed"], "peak_source": f"{src} hbm_gbs",
                         "wpass_avg_ms": w_ms, "wpass_frac": (wp["bytes"] / max(1, wp["timed"])) / (w_ms * 1e-3) / 1e9 / hbm,
                         "rxr_avg_ms": st[B.STAT_RXR]["total_ms"] / max(1, st[B.STAT_RXR]["timed"])},
            "clocks": clk.summary(),
            "e2e": {"value": e2e, "unit": "TSVDs/s", "h2d_bytes_per_step": m * n * 2,
                    "d2h_bytes_per_step": 8 * (m * r + r * r + n * r)},
            "gpu_launches": st[B.STAT_ALL]["launches"]}
    if not args.no_cpu_baseline:
        # the oracle's Algorithm 4 on the same full-size matrix (float64 copy of the stored values),
        # for the iteration count the GPU took: a few seconds of BLAS-bound CPU work
        from oracle import fradm as O
        Ms = prob.values_f64()
        k = int(np.median(iters))
        t2 = time.perf_counter()
        O.fixed_rank_opt_full(Ms, None, np.eye(r), np.eye(n, r), k)
        dts = time.perf_counter() - t2
        del Ms
        cores, model = host_cpu()
        line["cpu_baseline"] = {"value": 1.0 / dts, "unit": "TSVDs/s", "cores": cores, "cpu_model": model,
                                "kind": "oracle",
                                "sample": f"one run of the FP64 oracle's Algorithm 4 on the same {m}x{n} matrix, "
                                          f"{k} iterations ({dts:.1f} s)"}
    print(json.dumps(line), flush=True)
    return 0


# The other workloads of the benchmark recipe, one supplementary JSON line each (`--config NAME`).
OTHER_CONFIGS = {
    "square500_r25_f64": "500 x 500, r = 25, 10% outliers in [-50, 50], float64 storage, float64 path",
    "square16384_r64_f32_fp64": "16384 x 16384, r = 64, 5% outliers in [-50, 50], float32 storage, float64 path",
    "photometric_1048576x40_r3": "1024^2 pixels x 40 images, r = 3, float32 storage, mixed path (float32 sweep)",
    "affinity_32768_r20_nys2048": "32768^2 symmetric affinity, 20 clusters, 3% outliers, bfloat16 storage, "
                                  "FR-Nys with l = 2048 sampled columns, mixed path",
}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # SMs x FP64 FMA per clock x 2 flops x max SM clock


def run_config(args):
    """Solves/s of one of the other workloads (device-resident inputs, CUDA events on the
    library stream), the sweep against its roofline (HBM for the float32 / bfloat16 sweeps,
    FP64 ALU for the float64 path), the oracle on a bounded sample, and the host-buffer call."""
    import numpy as np
    import torch
    from paper_1503_03004_gb300 import binding as B, synth
    from oracle import fradm as O
    torch.cuda.set_device(0)
    name = args.config
    nys_l, perm = 0, None
    if name == "square500_r25_f64":
        prob, prec, mu0, s_dtype = synth.square_fp64_500(1000), B.PREC_FP64, 0.05, B.F64
    elif name == "square16384_r64_f32_fp64":
        prob, prec, mu0, s_dtype = synth.square_large(16384, 64, dtype="f32", seed=1001), B.PREC_FP64, 0.05, B.F32
    elif name == "photometric_1048576x40_r3":
        prob, prec, mu0, s_dtype = synth.photometric(seed=1002), B.PREC_MIXED, 1.0, B.F32
    else:
        # the tile-wise generator: the same bits the oracle's samples were computed from
        prob, prec, mu0, s_dtype = synth.affinity(n=32768, k=20, seed=1003, dtype="bf16"), B.PREC_MIXED, 1.0, B.F32
        nys_l = 2048
        perm = torch.from_numpy(synth.row_permutation(32768, 5)).cuda()
    M_dev = (torch.from_numpy(prob.M.view(np.int16)).view(torch.bfloat16) if prob.dtype == "bf16"
             else torch.from_numpy(prob.M)).cuda()
    r = prob.r
    m, n = M_dev.shape
    code = {torch.float64: B.F64, torch.float32: B.F32, torch.bfloat16: B.BF16}[M_dev.dtype]
    stream = torch.cuda.Stream()
    ctx = B.Context(0, stream=stream.cuda_stream, profile=True)
    f64 = dict(dtype=torch.float64, device="cuda")
    U, Bm, V = (None, None, None) if nys_l else (torch.empty((m, r), **f64), torch.empty((r, r), **f64),
                                                  torch.empty((n, r), **f64))
    sd = torch.float64 if s_dtype == B.F64 else torch.float32
    S = torch.empty((m, n), dtype=sd, device="cuda")
    kw = dict(m=m, n=n, r=r, m_dtype=code, mu0=mu0, rho=1.5, tol=1e-9, max_iter=300, precision=prec, nys_l=nys_l)
    p = B.make_problem(M_ptr=M_dev.data_ptr(), nys_perm_ptr=perm.data_ptr() if perm is not None else 0, **kw)
    res = B.make_result(U_ptr=U.data_ptr() if U is not None else 0, B_ptr=Bm.data_ptr() if Bm is not None else 0,
                        V_ptr=V.data_ptr() if V is not None else 0, S_ptr=S.data_ptr(), s_dtype=s_dtype, lds=n)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        if ctx.solve(p, res) != B.OK:
            raise RuntimeError(ctx.last_error())
    iters = res.iters
    ctx.stats(reset=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            if ctx.solve(p, res) != B.OK:
                raise RuntimeError(ctx.last_error())
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    st = ctx.stats(reset=True)
    sw = st[B.STAT_SWEEP]
    hbm, src = peaks()
    avg = sw["total_ms"] / max(1, sw["timed"])
    if prec == B.PREC_FP64:
        # float64 sweep: L rebuild (2 r) and (L + Delta) V (2 r) flops per element of the sweep
        achieved = 4 * pad_rank(r) * m * n / (avg * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "fused sweep (SIMT, float64)",
                "flops_per_element": 4 * pad_rank(r), "avg_launch_ms": avg, "timed_launches": sw["timed"],
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2.07 GHz"}
    else:
        achieved = sw["bytes"] / max(1, sw["timed"]) / (avg * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": "fused sweep", "bytes_per_launch": sw["bytes"] / max(1, sw["timed"]),
                "avg_launch_ms": avg, "timed_launches": sw["timed"], "peak_source": f"{src} hbm_gbs"}
    roof["wpass_avg_ms"] = st[B.STAT_WPASS]["total_ms"] / max(1, st[B.STAT_WPASS]["timed"])
    roof["rxr_avg_ms"] = st[B.STAT_RXR]["total_ms"] / max(1, st[B.STAT_RXR]["timed"])
    # e2e: host buffers (H2D of M and D2H of S and the factors inside the timed region)
    Mh = M_dev.cpu().pin_memory()
    Sh = torch.empty((m, n), dtype=sd).pin_memory()
    Uh, Bh, Vh = (np.empty((m, r)), np.empty((r, r)), np.empty((n, r))) if not nys_l else (None, None, None)
    permh = perm.cpu() if perm is not None else None
    ph = B.make_problem(M_ptr=Mh.data_ptr(), mem=B.MEM_HOST, nys_perm_ptr=permh.data_ptr() if permh is not None else 0,
                        **kw)
    rh = B.make_result(U_ptr=Uh.ctypes.data if Uh is not None else 0, B_ptr=Bh.ctypes.data if Bh is not None else 0,
                       V_ptr=Vh.ctypes.data if Vh is not None else 0, S_ptr=Sh.data_ptr(), s_dtype=s_dtype, lds=n)
    ctx.solve(ph, rh)
    t1 = time.perf_counter()
    for _ in range(args.e2e_steps):
        if ctx.solve(ph, rh) != B.OK:
            raise RuntimeError(ctx.last_error())
    e2e = args.e2e_steps / (time.perf_counter() - t1)
    ctx.close()
    line = {"metric": "solves/s", "value": 1000.0 / ms, "unit": "solves/s", "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f64" if prec == B.PREC_FP64 else "f32/f64", "data": "synthetic",
            "config": {"workload": name, "recipe": OTHER_CONFIGS[name], "m": m, "n": n, "r": r, "nys_l": nys_l,
                       "mu0": mu0, "rho": 1.5, "tol": 1e-9, "iters_per_solve": iters},
            "roofline": roof, "clocks": clk.summary(),
            "e2e": {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": Mh.numel() * Mh.element_size(),
                    "d2h_bytes_per_step": Sh.numel() * Sh.element_size() + (0 if nys_l else 8 * (m + n + r) * r)},
            "gpu_launches": st[B.STAT_ALL]["launches"]}
    if not args.no_cpu_baseline:
        # the float64 oracle on a bounded sample of the same recipe, scaled to the full size by
        # the element count (every step of both methods is O(elements) per iteration)
        if name == "square500_r25_f64":
            sp, scale, what = prob, 1.0, "the full 500x500 problem"
            ref = lambda Ms: O.fr_adm(Ms, r, rho=1.5, mu0=mu0, tol=1e-9, max_iter=300)
        elif name == "square16384_r64_f32_fp64":
            sp = synth.planted(2048, 2048, 64, p=0.05, amp=50.0, seed=1001, dtype="f32")
            scale, what = (m * n) / 2048 ** 2, "a 2048x2048 r=64 sample, scaled by m*n"
            ref = lambda Ms: O.fr_adm(Ms, r, rho=1.5, mu0=mu0, tol=1e-9, max_iter=300)
        elif name == "photometric_1048576x40_r3":
            sp = synth.photometric(side=256, seed=1002)
            scale, what = m / 256 ** 2, "a 256^2-pixel x 40 sample of the recipe, scaled by m"
            ref = lambda Ms: O.fr_adm(Ms, r, rho=1.5, mu0=mu0, tol=1e-9, max_iter=300)
        else:
            sp = synth.affinity(n=4096, k=20, seed=1003, dtype="bf16")
            scale, what = (m / 4096) ** 2, "n=4096, l=256 (the same l/n), scaled by n^2"
            sperm = synth.row_permutation(4096, 5)
            ref = lambda Ms: O.fr_nys(Ms, r, 256, sperm, rho=1.5, mu0=mu0, tol=1e-9, max_iter=300)
        Ms = sp.values_f64()
        t2 = time.perf_counter()
        ref(Ms)
        dts = time.perf_counter() - t2
        cores, model = host_cpu()
        line["cpu_baseline"] = {"value": 1.0 / (dts * scale), "unit": "solves/s", "cores": cores, "cpu_model": model,
                                "kind": "oracle",
                                "sample": f"one FP64 oracle solve of {what} ({dts:.1f} s)"}
    print(json.dumps(line), flush=True)
    return 0


def pad_rank(r: int) -> int:
    return 8 if r <= 8 else 16 if r <= 16 else 32 if r <= 32 else 64


def run_paper_tables(args):
    """The scale experiment of Sec. 5.1 (Tables 1 and 2) on the GPU: M = A B^T + S, A, B ~ N(0, 1),
    10 % outliers with magnitudes in [-1, 1], m = n from 500 to 8000 at r = 10 (Table 1) and at
    r = 0.1 m while r <= 64 (Table 2; the library's rank limit), solved by FR-ADM (float64 and
    mixed paths) and FR-Nys (l = 10 r sampled columns, k = 10 as in Algorithm 2), rho = 1.5,
    tol 1e-9, with mu0 = 1 (Algorithm 1) and with mu0 = 1.25 / ||M||_2.  Reports per case the wall time of one device-resident solve (after a
    warm-up solve of the same shape), the iterations, and Err.L = ||L - L0|| / ||L0||,
    Err.S = ||S - S0|| / ||S0|| against the planted matrices.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_1503_03004_gb300 import binding as B, synth
    torch.cuda.set_device(0)
    cases = [(m, 10) for m in (500, 1000, 2000, 4000, 8000)] + [(500, 50), (640, 64)]
    rows = []
    with B.Context(0) as ctx:
        for m, r in cases:
            prob = synth.paper_table1(m, r=r, seed=7)
            Md = torch.from_numpy(prob.M).cuda()
            L0 = torch.from_numpy(prob.U0 @ prob.V0.T).cuda()
            S0 = Md - L0
            nl0, ns0 = float(torch.linalg.norm(L0)), float(torch.linalg.norm(S0))
            perm = torch.from_numpy(synth.row_permutation(m, 5)).cuda()
            # two readings of mu_0: Algorithm 1's literal 1, and the 1.25 / ||M||_2 of the inexact
            # ALM the paper builds on (scale-aware; ||M||_2 computed here, outside the timing)
            mu_alm = 1.25 / float(torch.linalg.matrix_norm(Md, ord=2))
            variants = []
            for mu0, tag in ((1.0, "1"), (mu_alm, "1.25/||M||_2")):
                variants += [("FR-ADM", B.PREC_FP64, 0, mu0, tag), ("FR-ADM", B.PREC_MIXED, 0, mu0, tag)]
                if 10 * r <= m:
                    variants += [("FR-Nys", B.PREC_FP64, 10 * r, mu0, tag), ("FR-Nys", B.PREC_MIXED, 10 * r, mu0, tag)]
            for method, prec, l, mu0, tag in variants:
                kw = dict(rho=1.5, mu0=mu0, tol=1e-9, max_iter=500, precision=prec, s_dtype=B.F64, check=False)
                if l:
                    kw.update(nys_l=l, nys_perm=perm, want_L=True)
                B.solve_torch(ctx, Md, r, **kw)  # warm-up: workspace, graphs, tuned grid
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sol = B.solve_torch(ctx, Md, r, **kw)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                L = sol.L if l else sol.U @ sol.B @ sol.V.T
                rows.append({"m": m, "r": r, "method": method, "precision": "fp64" if prec == B.PREC_FP64 else "mixed",
                             "mu0": tag, "nys_l": l, "status": B.STATUS_NAMES.get(sol.status, sol.status),
                             "iters": sol.iters,
                             "seconds": dt, "err_L": float(torch.linalg.norm(L - L0)) / nl0,
                             "err_S": float(torch.linalg.norm(sol.S - S0)) / ns0})
    line = {"metric": "paper Sec. 5.1 scale experiment (Tables 1-2 recipe)", "unit": "s per solve",
            "higher_is_better": False, "data": "synthetic",
            "config": {"recipe": "L = A B^T, A, B ~ N(0,1); 10% outliers uniform in [-1, 1]; seed 7",
                       "mu0": ["1", "1.25/||M||_2"], "rho": 1.5, "tol": 1e-9, "nys_l": "10 r"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_phase(args):
    """The phase-transition experiment of Fig. 2 for FR-ADM on the GPU: m = n = 800, rank fraction
    r / 800 in {0.01, 0.02, 0.04, 0.06, 0.08} (the library's r <= 64 caps it there), outlier
    fraction 0.05 .. 0.50, the Sec. 5.1 entries (A, B ~ N(0, 1), outliers in [-1, 1]), `--reps`
    repetitions per cell.  All problems go through sfr_submit / sfr_poll (8 slots, mixed path;
    mu0 = 1.25 / ||M||_2, the scale-aware start of the inexact ALM the paper builds on, rho = 1.5,
    tol 1e-9).  Per cell: the paper's error
    measure (1 / K) sum_z sum_ij psi_eps(S_z - S*_z) / (m n), psi_eps(s) = |s| if |s| > eps else 0,
    eps = 1e-3, and Err.L; plus the batch's throughput.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_1503_03004_gb300 import binding as B, synth
    torch.cuda.set_device(0)
    m = 800
    fr = [0.01, 0.02, 0.04, 0.06, 0.08]
    po = [0.05, 0.10, 0.15, 0.20, 0.25, 0.30, 0.35, 0.40, 0.45, 0.50]
    eps = 1e-3
    items = []
    for ri, f in enumerate(fr):
        r = max(1, int(round(f * m)))
        for pi, p in enumerate(po):
            for z in range(args.reps):
                prob = synth.planted(m, m, r, p=p, amp=1.0, seed=9000 + 1000 * ri + 10 * pi + z, dtype="f64")
                Md = torch.from_numpy(prob.M).cuda()
                L0 = torch.from_numpy(prob.U0 @ prob.V0.T).cuda()
                mu0 = 1.25 / float(torch.linalg.matrix_norm(Md, ord=2))
                f64 = dict(dtype=torch.float64, device="cuda")
                out = dict(U=torch.empty((m, r), **f64), B=torch.empty((r, r), **f64), V=torch.empty((m, r), **f64),
                           S=torch.empty((m, m), **f64))
                q = B.make_problem(m=m, n=m, r=r, M_ptr=Md.data_ptr(), m_dtype=B.F64, mu0=mu0, rho=1.5, tol=1e-9,
                                   max_iter=500, precision=B.PREC_MIXED)
                res = B.make_result(U_ptr=out["U"].data_ptr(), B_ptr=out["B"].data_ptr(), V_ptr=out["V"].data_ptr(),
                                    S_ptr=out["S"].data_ptr(), s_dtype=B.F64, lds=m)
                items.append(((f, p, r), Md, L0, out, q, res))
    torch.cuda.synchronize()
    with B.Context(0, max_slots=8) as ctx:
        t0 = time.perf_counter()
        tickets = [ctx.submit(it[4], it[5]) for it in items]
        status = [ctx.poll(t, -1) for t in tickets]
        wall = time.perf_counter() - t0
    cells = {}
    for (key, Md, L0, out, q, res), st in zip(items, status):
        S0 = Md - L0
        d = (out["S"] - S0).abs()
        psi = float(torch.where(d > eps, d, torch.zeros_like(d)).sum()) / (m * m)
        L = out["U"] @ out["B"] @ out["V"].T
        errl = float(torch.linalg.norm(L - L0) / torch.linalg.norm(L0))
        c = cells.setdefault(key, {"rank_fraction": key[0], "outlier_fraction": key[1], "r": key[2], "psi": 0.0,
                                   "err_L": 0.0, "iters": 0, "ok": 0, "count": 0})
        c["psi"] += psi / args.reps
        c["err_L"] = max(c["err_L"], errl)
        c["iters"] += res.iters
        c["ok"] += int(st == B.OK)
        c["count"] += 1
    line = {"metric": "Fig. 2 phase transition, FR-ADM (batched through the serving slots)",
            "value": len(items) / wall, "unit": "solves/s", "problems": len(items), "slots": 8,
            "config": {"m": m, "n": m, "rank_fractions": fr, "outlier_fractions": po, "reps": args.reps,
                       "outliers": "uniform in [-1, 1]", "mu0": "1.25/||M||_2", "rho": 1.5, "tol": 1e-9,
                       "eps": eps, "precision": "mixed", "storage": "f64"},
            "cells": list(cells.values())}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    """The reference arm: the float64 oracle (the slow reference program) on the host cores.

    Each step is one oracle solve of a REF_SAMPLE-sized sample of the workload's recipe (a
    bounded sample, so that the run ends within a few minutes); `ms_per_step` is that measured
    wall time, and `value` is the full workload's rate it implies (sample rate / scale, scale =
    the ratio of element counts, since the method is O(m n r) per iteration)."""
    rank, world, _ = dist_setup()
    if rank != 0:
        return 0
    times, info = [], None
    for i in range(args.warmup + args.steps):
        info, _ = oracle_sample_rate(sample=REF_SAMPLE)
        if i >= args.warmup:
            times.append(info["sample_seconds"])
    per_step = sum(times) / len(times)
    value = 1.0 / (per_step * info["scale"])
    line = {"impl": "reference", "metric": "solves/s", "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": WORKLOAD | {"scaled": (f"each step solves a {REF_SAMPLE['m']}x{REF_SAMPLE['n']} sample of "
                                             f"the recipe; value = its rate / {info['scale']:g} (element count)"),
                                  "sample_m": REF_SAMPLE["m"], "sample_n": REF_SAMPLE["n"]},
            "sample_ms_per_step": 1000.0 * per_step, "scale_to_workload": info["scale"],
            "cpu_baseline": {k: info[k] for k in ("kind", "cores", "cpu_model", "sample")} | {"value": value,
                                                                                          "unit": "solves/s"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true",
                    help="do not time kernels with events (no roofline; for measuring the profiling cost)")
    ap.add_argument("--serving", action="store_true",
                    help="supplementary: the serving-stream workload (submit/poll slots vs per-problem solves)")
    ap.add_argument("--opt-full", action="store_true",
                    help="supplementary: FixedRankOptFull (Algorithm 4) as a TSVD of the benchmark matrix")
    ap.add_argument("--config", choices=sorted(OTHER_CONFIGS),
                    help="supplementary: one of the other workloads of the recipe")
    ap.add_argument("--paper-tables", action="store_true",
                    help="supplementary: the Sec. 5.1 scale experiment (Tables 1-2 recipe) on the GPU")
    ap.add_argument("--phase", action="store_true",
                    help="supplementary: the Fig. 2 phase transition for FR-ADM, batched through the serving slots")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--requests", type=int, default=4096)
    ap.add_argument("--check", type=int, default=8, help="serving: requests checked against the float64 oracle")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--max-batch", type=int, default=256,
                    help="serving: problems the grouped engine iterates together (0: slots only)")
    ap.add_argument("--budget-gb", type=int, default=64)
    ap.add_argument("--m", type=int, default=WORKLOAD["m"],
                    help="square size of the same recipe (smaller sizes are for profiler captures)")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # --gpus N outside torchrun: start N replica ranks (each solves its own problem on its own
        # GPU; barrier and max-time reduction only)
        return subprocess.call(relaunch_cmd(sys.argv[1:], args.gpus, free_port()))
    if args.m != WORKLOAD["m"]:
        mb = args.m * args.m * 2 // (1 << 20)
        WORKLOAD.update(m=args.m, n=args.m, workload=f"square{args.m}_r64_bf16_mixed",
                        l2=f"M {mb} MB, multipliers 2 x {mb} MB, Delta {mb} MB; no flush")
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)
    if args.opt_full:
        return run_opt_full(args)
    if args.config:
        return run_config(args)
    if args.paper_tables:
        return run_paper_tables(args)
    if args.phase:
        return run_phase(args)

    import numpy as np
    import torch
    from paper_1503_03004_gb300 import binding as B

    rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        # gloo carries the two scalar reductions (barrier, max time); the data path has no collective
        dist.init_process_group("gloo")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_base, _ = oracle_sample_rate()  # before any CUDA work of the library (host cores only)

    prob = make_workload(seed=1001 + rank)
    m, n, r = WORKLOAD["m"], WORKLOAD["n"], WORKLOAD["r"]
    M_dev = torch.from_numpy(prob.M.view(np.int16)).view(torch.bfloat16).cuda()
    U = torch.empty((m, r), dtype=torch.float64, device="cuda")
    Bm = torch.empty((r, r), dtype=torch.float64, device="cuda")
    V = torch.empty((n, r), dtype=torch.float64, device="cuda")
    S = torch.empty((m, n), dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()           # the library and the timing events share this stream
    # inside the timed region only the sweep is timed with events (event records between the other
    # kernels of the iteration would cost time and split the programmatic launch chain)
    ctx = B.Context(local, stream=stream.cuda_stream, profile=0 if args.no_profile else 2)
    kw = dict(m=m, n=n, r=r, m_dtype=B.BF16, mu0=WORKLOAD["mu0"], rho=WORKLOAD["rho"], tol=WORKLOAD["tol"],
              max_iter=WORKLOAD["max_iter"], precision=B.PREC_MIXED)
    p = B.make_problem(M_ptr=M_dev.data_ptr(), **kw)
    res = B.make_result(U_ptr=U.data_ptr(), B_ptr=Bm.data_ptr(), V_ptr=V.data_ptr(), S_ptr=S.data_ptr(),
                        s_dtype=B.F32, lds=n)
    torch.cuda.synchronize()

    def one_solve():
        st = ctx.solve(p, res)
        if st != B.OK:
            raise RuntimeError(f"solve failed: {B.STATUS_NAMES.get(st)} {ctx.last_error()}")
        return res.iters

    for _ in range(args.warmup):
        one_solve()
    iters_seen = res.iters
    ctx.stats(reset=True)

    # ---- timed region: K device-resident solves
    barrier()
    torch.cuda.synchronize()
    lat = []
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):
            a = time.perf_counter()
            one_solve()  # synchronous: the library waits for its stream before returning
            lat.append(time.perf_counter() - a)
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    stats = ctx.stats(reset=True)
    value = aggregate(args.steps, elapsed_ms)
    elapsed_ms = reduce_max(elapsed_ms)
    clocks = clk.summary()

    # per-kernel breakdown (W pass, r x r projector) from one more solve outside the timed region,
    # with every kernel class timed
    breakdown = {}
    if not args.no_profile:
        with B.Context(local, stream=stream.cuda_stream, profile=1) as pctx:
            if pctx.solve(p, res) != B.OK:
                raise RuntimeError(pctx.last_error())
            pst = pctx.stats()
        breakdown = {"wpass_avg_ms": pst[B.STAT_WPASS]["total_ms"] / max(1, pst[B.STAT_WPASS]["timed"]),
                     "rxr_avg_ms": pst[B.STAT_RXR]["total_ms"] / max(1, pst[B.STAT_RXR]["timed"]),
                     "breakdown_from": "one untimed solve with every kernel class event-timed"}

    # roofline of the fused sweep kernel: algorithmic bytes per launch / event-timed duration
    sw = stats[B.STAT_SWEEP]
    peak, peak_kind = peaks()
    roofline = None
    if sw["timed"] > 0:
        # algorithmic bytes per launch as the library accounts them: M, Y_k read, Y_{k+1}, Delta written
        alg_bytes = sw["bytes"] / sw["timed"]
        avg_ms = sw["total_ms"] / sw["timed"]
        achieved = alg_bytes / (avg_ms / 1000.0) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": sweep_traffic(m, n), "kernel": "fused sweep", "bytes_per_launch": alg_bytes,
                    "bytes_per_element": alg_bytes / (m * n), "avg_launch_ms": avg_ms, "timed_launches": sw["timed"],
                    "peak_source": peak_kind + " hbm_gbs"} | breakdown

    # ---- e2e: the same solve through the C ABI with pinned host buffers (copies inside the region)
    M_host = torch.from_numpy(prob.M.view(np.int16)).pin_memory()
    S_host = torch.empty((m, n), dtype=torch.float32).pin_memory()
    U_h = np.empty((m, r)); B_h = np.empty((r, r)); V_h = np.empty((n, r))
    ph = B.make_problem(M_ptr=M_host.data_ptr(), mem=B.MEM_HOST, **kw)
    rh = B.make_result(U_ptr=U_h.ctypes.data, B_ptr=B_h.ctypes.data, V_ptr=V_h.ctypes.data, S_ptr=S_host.data_ptr(),
                       s_dtype=B.F32, lds=n)
    if ctx.solve(ph, rh) != B.OK:
        raise RuntimeError(ctx.last_error())
    barrier()
    a = time.perf_counter()
    for _ in range(args.e2e_steps):
        if ctx.solve(ph, rh) != B.OK:
            raise RuntimeError(ctx.last_error())
    e2e_s = reduce_max(time.perf_counter() - a)
    e2e = {"value": world * args.e2e_steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 2 * m * n,
           "d2h_bytes_per_step": 4 * m * n + 8 * (m * r + r * r + n * r)}

    # accuracy of the timed solves against the float64 oracle: its L_ij and S_ij at the 4096 seeded
    # positions stored by tests/golden/make_fullsize_samples.py (oracle and generators only)
    accuracy = oracle_sample_error(U, Bm, V, S) if (m, n, r) == (16384, 16384, 64) and rank == 0 else None

    lat_ms = sorted(x * 1000.0 for x in lat)
    line = {"metric": "solves/s", "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": WORKLOAD | {"parallelism": f"replicas x{world}", "iters_per_solve": iters_seen},
            "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1,
                                                                                int(0.99 * len(lat_ms)))]},
            "roofline": roofline, "clocks": clocks, "e2e": e2e,
            "gpu_launches": stats[B.STAT_ALL]["launches"],
            "cpu_baseline": cpu_base and {k: cpu_base[k] for k in ("value", "unit", "cores", "cpu_model", "kind",
                                                                   "sample")},
            "accuracy": accuracy}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
