#!/usr/bin/env python
"""Benchmark: k smallest eigenpairs of the s-FairSC operator + embedding + k-means
(Algorithm 3 end to end) on a synthetic m-SBM workload, one solve per step.

Default workload: msbm_n1m_k50_h10 (n = 1,000,000, k = 50 Dirichlet(5)-sized
clusters, h = 10 Zipf(1) groups, mean degree 32 split 50/25/15/10, BF16 0/1
weights, seed 2), mixed precision, Krylov block 4, residual tol 1e-6 * sigma.
A step = sfairsc_create (setup) + sfairsc_solve (eigensolve, embedding,
k-means) on device-resident inputs.  value = seconds per solve (job level).

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank solves its own replica (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

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

METRIC = "fused fair-operator HBM GB/s; k-eigpair solve s, mixed/batched vs plain FP64 @1e-6"
VDT_BYTES = {"f64": 8, "f32": 4, "bf16": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="msbm_n1m_k50_h10")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--block", type=int, default=4)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 / operator / e2e / CPU side measurements")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-graph batched measurement")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink n of the workload (profiling runs only)")
    ap.add_argument("--cpu-child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--only", default=None, choices=["operator", "solve"],
                    help="profiling runs: time the standalone operator (--nvec, --reps), or run one solve")
    ap.add_argument("--nvec", type=int, default=1)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--window", type=int, default=0, help="spmv_window option of the context (0 or 1)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def load_workload(name, scale=1.0):
    from msbm import configs

    c = configs.BUILDERS[name](scale=scale)
    if "graphs" in c:
        raise SystemExit("batched workload: use the batched bench entry")
    return c


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline arithmetic
def operator_bytes(n, nnz, s_v, s_x, b):
    """Algorithmic bytes of one fused operator launch on b vectors.

    row_ptr 4(n+1) + col 4 nnz + values s_v nnz (read once), the b input and
    b output vectors (s_x each), the uint8 labels and D^{-1/2} (s_x) per row.
    """
    return 4 * (n + 1) + nnz * (4 + s_v) + n * (2 * b * s_x + 1 + s_x)


def orth_bytes(n, sum_cols, launches, sweeps, s_x, b):
    """Algorithmic bytes of the Gram-Schmidt launches: V[:, 0:J] is read once
    per sweep (2 sweeps: coefficients, then the update fused with the second
    coefficients and the Gram matrix; 3 when the DGKS test asks for the second
    projection), the new block is read once and written once.  sweeps / launches
    is the measured mean number of sweeps per launch."""
    return (sweeps / max(1, launches)) * n * s_x * sum_cols + launches * 2 * n * b * s_x


def recorded_traffic(summary: str, sources: list[str]):
    """DRAM bytes per launch from a committed ncu summary (profiles/), or None if
    any of the kernel's source files changed since the counters were taken."""
    import hashlib
    import re

    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    if not m:
        return None
    for src in sources:
        h = re.search(r"source_sha256 " + re.escape(os.path.basename(src)) + r":\s*([0-9a-f]{64})", text)
        with open(os.path.join(ROOT, src), "rb") as f:
            cur = hashlib.sha256(f.read()).hexdigest()
        if not h or h.group(1) != cur:
            return None
    return int(m.group(1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def batched_basis(n, k):
    """Basis size m and thick-restart size K of one graph of the batched solver."""
    m = max(2 * k + 8, 20)
    m = (m + 3) // 4 * 4
    m = min(m, min(60, (n // 4) * 4 - 4))
    K = k + (m - k) // 2
    K = max(K // 4 * 4, (k + 3) // 4 * 4)
    K = min(K, m - 4)
    return m, K


def batched_bytes(n, nnz, k, matvecs, restarts):
    """Algorithmic HBM bytes of one graph's batched solve (FP32 vectors, FP32 weights).

    Per block step (4 operator applications): the CSR once (4(n+1) + 8 nnz),
    the input panel, the output block, D^{-1/2} and the labels (n (16 + 16 + 4
    + 1)); classical Gram-Schmidt at its minimum, V[:, 0:J] read twice (8 n J)
    plus the new panel written (16 n), J averaged over a restart cycle.  Per
    restart the basis is read once and the kept columns written once."""
    m, K = batched_basis(n, k)
    steps = matvecs // 4
    jbar = (K + m) / 2 + 2
    per_step = 4 * (n + 1) + 8 * nnz + n * 37 + 8 * n * jbar + 16 * n
    per_restart = 4 * n * (m + K)
    return steps * per_step + restarts * per_restart


def batched_extra(dev, peak, scale=1.0, sequential=True, seq_sample=None):
    """The batched form on the 256-graph workload: one persistent launch per
    solve, default schedule and autotuned, against sequential solves of the
    same graphs through the single-graph API (FP64 block 1, and mixed block 4)."""
    import numpy as np
    import torch

    from msbm import configs
    from paper_2210_16435_gb300.solver import FairSC, FairSCBatch

    t0 = time.perf_counter()
    c = configs.msbm_batch256(scale=scale)
    gen_s = time.perf_counter() - t0
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    ents = [{"row_ptr": T(x["graph"].row_ptr, torch.int32), "col_idx": T(x["graph"].col_idx, torch.int32),
             "values": T(x["graph"].values, torch.float32), "groups": T(x["graph"].groups, torch.int32),
             "k": x["k"], "h": x["h"]} for x in c["graphs"]]
    b = FairSCBatch(ents)
    b.solve()
    reps = 3
    ms_def = [b.solve()[1]["ms_solve"] for _ in range(reps)]
    st, info_def = b.solve()
    t0 = time.perf_counter()
    from paper_2210_16435_gb300 import binding as B

    B.sfairsc_batch_autotune(b.handle)
    tune_s = time.perf_counter() - t0
    ms_at = [b.solve()[1]["ms_solve"] for _ in range(reps)]
    st, info = b.solve()
    restarts, matvecs, resid = b.stats()
    b.close()
    tot_bytes = sum(batched_bytes(x["graph"].n, x["graph"].nnz, x["k"], mv, rs)
                    for x, mv, rs in zip(c["graphs"], matvecs, restarts))
    ms = min(ms_at)
    gbs = tot_bytes / (ms * 1e6)
    # sequential solves through the single-graph API (every graph, or a sample scaled up)
    idx = list(range(len(ents))) if seq_sample is None else seq_sample
    seq = {}
    for prec, blk in ((("fp64", 1), ("mixed", 4)) if sequential else ()):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        nconv = 0
        for i in idx:
            e = ents[i]
            s = FairSC(e["row_ptr"], e["col_idx"], e["values"], e["groups"], k=e["k"], h=e["h"], prec=prec, block=blk)
            _, _, _, inf = s.solve(want_labels=False, allow_not_converged=True)
            nconv += s.status == 0
            s.close()
        torch.cuda.synchronize()
        el = (time.perf_counter() - t1) * len(ents) / len(idx)
        seq[f"sequential_{prec}_block{blk}_s"] = el
        seq[f"sequential_{prec}_converged"] = f"{nconv}/{len(idx)}"
    return {
        "workload": "msbm_batch256 (256 m-SBM graphs, n log-uniform 1k-64k, k 3-10, h 2-6, degree 16-64, FP32 weights)",
        "graphs": len(ents), "sum_n": int(sum(x["graph"].n for x in c["graphs"])),
        "sum_nnz": int(sum(x["graph"].nnz for x in c["graphs"])),
        "solve_s": ms / 1e3, "solve_s_default_schedule": min(ms_def) / 1e3, "autotune_s": tune_s,
        "converged": info["converged"], "max_resid": info["max_resid"], "restarts": info["restarts"],
        "matvecs": info["matvecs"], "schedule": {"ctas_per_sm": info["ctas_per_sm"], "max_team": info["max_team"],
                                                  "split": info["split"], "teams_1_2_4_8_16": info["teams"],
                                                  "grid": info["grid"]},
        "cuda_graph": info["cuda_graph"], "gpu_launches_per_solve": 1,
        "roofline": {"kernel": "batched_kernel (persistent, all graphs)", "bound": "hbm", "achieved": gbs,
                     "peak": peak, "unit": "GB/s", "frac": gbs / peak, "traffic": None,
                     "bytes_per_launch": tot_bytes, "ms_per_launch": ms},
        **seq, "speedup_vs_sequential_fp64": (seq["sequential_fp64_block1_s"] / (ms / 1e3)) if seq else None,
        "generate_s": gen_s,
    }


def run_batched_main(args):
    """--workload msbm_batch256: the batched solve alone (one launch per step), e.g. for profiling."""
    import torch

    torch.cuda.set_device(0)
    from paper_2210_16435_gb300 import buildlib

    buildlib.build()
    peak, _ = measured_peaks()
    r = batched_extra(torch.device("cuda", 0), peak, scale=args.scale, sequential=not args.no_extras)
    print(json.dumps({"metric": "batched k-eigenpair solve (256 graphs, one launch)", "value": r["solve_s"],
                      "unit": "s/batch", "higher_is_better": False, "batched": r}), flush=True)


# ---------------------------------------------------------------- oracle on the host cores
class _StopCycles(Exception):
    pass


def oracle_solve_timed(g, k, tol=1e-6, max_cycles=None, on_cycle=None):
    """The CPU oracle's eigensolve (Algorithm 3 steps 1-3) on the full graph, timed.

    Setup (operator_from_graph: degrees, L_n, C, the C^T C factor, sigma) and
    the oracle's own thick-restart Lanczos (m = max(2k, 20), two classical
    Gram-Schmidt passes per step, FP64) to ||A x - lambda x|| <= tol sigma.
    Cycle i's time runs from the end of cycle i-1's steps to the end of its
    own (so it includes the previous restart).  max_cycles stops the solve
    early (a bounded sample).  Returns a dict of times and counts, and the
    operator and vectors when the solve finished.
    """
    from oracle.lanczos import thick_restart_lanczos
    from oracle.sfairsc import operator_from_graph

    t0 = time.perf_counter()
    op = operator_from_graph(g)
    t_setup = time.perf_counter() - t0
    marks = [time.perf_counter()]
    mv = [0]

    def cb(cycle, matvecs):
        marks.append(time.perf_counter())
        mv[0] = matvecs
        if on_cycle is not None:
            on_cycle(cycle, marks[-1] - marks[-2])
        if max_cycles is not None and cycle + 1 >= max_cycles:
            raise _StopCycles()

    done, lam, X, info = True, None, None, {}
    try:
        lam, X, info = thick_restart_lanczos(op.apply, g.n, k, tol=tol, anorm=op.sigma, seed=0, on_cycle=cb)
    except _StopCycles:
        done = False
    t_end = time.perf_counter()
    cycles = [b - a for a, b in zip(marks[:-1], marks[1:])]
    return {"op": op, "lam": lam, "X": X, "done": done, "setup_s": t_setup, "cycle_s": cycles,
            "tail_s": t_end - marks[-1], "solve_s": t_end - marks[0], "matvecs": info.get("matvecs", mv[0]),
            "restarts": info.get("restarts", len(cycles) - 1)}


def oracle_kmeans_timed(H, k, full=True, sample_iters=3, iters_total=None):
    """The oracle's seeded k-means (Algorithm 3 step 4) on the rows of H: k-means++
    seeding and Lloyd assignments to convergence (full), or the seeding and
    sample_iters assignments timed and scaled to iters_total assignments."""
    import numpy as np

    from oracle.kmeans import kmeanspp, lloyd

    X32 = np.ascontiguousarray(np.asarray(H, dtype=np.float64).astype(np.float32))
    t0 = time.perf_counter()
    seeds = kmeanspp(X32, k, 0, 0)
    t_seed = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, _, iters = lloyd(X32, X32[seeds].astype(np.float64), 100 if full else sample_iters)
    t_lloyd = time.perf_counter() - t0
    if full:
        return t_seed + t_lloyd, iters, f"seeding {t_seed:.1f}s + {iters} Lloyd assignments {t_lloyd:.1f}s"
    per = t_lloyd / iters
    est = t_seed + per * iters_total
    return est, iters_total, (f"seeding {t_seed:.1f}s + {iters} Lloyd assignments timed ({per:.2f}s each), "
                              f"x {iters_total} assignments (the count of the same algorithm on the same H)")


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_single_thread_child(args):
    """--cpu-child FILE: the oracle's setup and first two Lanczos cycles on one thread
    (BLAS threads pinned to 1 by the parent's environment) on the graph saved in FILE;
    prints one JSON line."""
    import numpy as np

    from msbm import Graph

    d = np.load(args.cpu_child)
    g = Graph(d["row_ptr"], d["col_idx"], d["values"], d["groups"], d["groups"] * 0, int(d["h"]), int(d["k"]))
    r = oracle_solve_timed(g, int(d["k"]), tol=1e-6, max_cycles=2)
    print(json.dumps({"setup_s": r["setup_s"], "cycle_s": r["cycle_s"]}), flush=True)


def oracle_single_thread(g, k, cycles_total):
    """Seconds per solve of the oracle on one host thread: setup and the first two cycles
    timed in a child process with OMP/OPENBLAS/MKL threads = 1, the remaining cycles
    at the second cycle's time (every later cycle does the same m - K steps)."""
    import tempfile

    import numpy as np

    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "graph.npz")
        np.savez(path, row_ptr=g.row_ptr, col_idx=g.col_idx, values=g.values, groups=g.groups, h=g.h, k=k)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child", path],
                           capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return None, f"single-thread child failed: {r.stderr[-300:]}"
    d = json.loads(r.stdout.strip().splitlines()[-1])
    cyc = d["cycle_s"]
    later = cyc[1] if len(cyc) > 1 else cyc[0]
    est = d["setup_s"] + cyc[0] + later * max(0, cycles_total - 1)
    return est, (f"one thread: setup {d['setup_s']:.1f}s, cycle 1 {cyc[0]:.1f}s, cycle 2 {later:.1f}s timed; "
                 f"x {cycles_total} cycles of the all-core solve of the same graph")


# ---------------------------------------------------------------- arms
def run_reference(args):
    """The CPU oracle on the host cores, on the same workload (no GPU).

    A step is one restart cycle of the oracle's thick-restart Lanczos on the
    full graph (a bounded sample of a few seconds).  Solves run back to back
    cycle by cycle: W warm-up cycles, then K timed cycles; a solve that is
    still running then continues to convergence, so at least one complete
    solve is measured.  value = setup + every cycle of one complete solve +
    embedding + the oracle's k-means to convergence on its H: a measured
    time, nothing extrapolated."""
    import numpy as np

    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle.sfairsc import embed

    c = load_workload(args.workload)
    g, k, h = c["graph"], c["k"], c["h"]
    timed = []
    state = {"cycle": 0}

    def on_cycle(cycle, dt):
        state["cycle"] += 1
        if state["cycle"] > args.warmup and len(timed) < args.steps:
            timed.append(dt)

    solves = []
    while True:
        r = oracle_solve_timed(g, k, tol=1e-6, on_cycle=on_cycle)
        solves.append(r)
        if len(timed) >= args.steps:
            break
    first = solves[0]
    t0 = time.perf_counter()
    H = embed(first["op"], first["X"])
    t_embed = time.perf_counter() - t0
    t_km, iters, km_text = oracle_kmeans_timed(H, k, full=True)
    solve_s = statistics.median(x["setup_s"] + x["solve_s"] for x in solves)
    value = solve_s + t_embed + t_km
    cores = host_threads()
    sample = (f"oracle (FP64 NumPy/SciPy) on the full graph, {cores} host threads: {len(solves)} complete "
              f"solve(s) to 1e-6 sigma, setup {first['setup_s']:.1f}s + {len(first['cycle_s'])} Lanczos cycles "
              f"{first['solve_s']:.1f}s ({first['matvecs']} matvecs, {first['restarts']} restarts); embedding "
              f"{t_embed:.2f}s; k-means: {km_text}; a step = one Lanczos cycle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(timed) * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": g.n, "nnz": g.nnz, "k": k, "h": h, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "s/solve", "cores": cores, "kind": "oracle", "sample": sample,
                         "matvecs": first["matvecs"], "restarts": first["restarts"]},
        "e2e": {"value": value, "unit": "s/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_operator(B, s, dev, stream, g, s_v, s_x, nvecs, peak, reps=50):
    """Median-free mean device time of back-to-back sfairsc_apply_operator calls (CUDA
    events on the launching stream, 5 untimed first), and its algorithmic GB/s."""
    import torch

    out = {}
    for nv in nvecs:
        Wc = torch.randn(nv, g.n, device=dev, dtype=s.vec_dtype)
        O = torch.empty_like(Wc)
        for _ in range(5):
            B.sfairsc_apply_operator(s.ctx, Wc.data_ptr(), O.data_ptr(), nv)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record(stream)
        for _ in range(reps):
            B.sfairsc_apply_operator(s.ctx, Wc.data_ptr(), O.data_ptr(), nv)
        a1.record(stream)
        torch.cuda.synchronize()
        oms = a0.elapsed_time(a1) / reps
        ob = operator_bytes(g.n, g.nnz, s_v, s_x, nv)
        out[f"nvec{nv}"] = {"us": oms * 1e3, "achieved_gbs": ob / (oms * 1e6), "frac": ob / (oms * 1e6) / peak,
                            "bytes": ob}
    return out


def h_sweep(FairSC, B, dev, stream, g, rp, ci, v, k, h, args, s_v, s_x, peak):
    """Solve time of the same graph with its h groups merged to fewer (h = 1 is plain SC)."""
    import torch

    out = []
    for hh in (1, 2, 5, h):
        grp = torch.as_tensor((g.groups % hh) if hh > 1 else g.groups * 0, dtype=torch.int32, device=dev)
        s = FairSC(rp, ci, v, grp, k=k, h=hh, prec=args.prec, block=args.block, profile=1)
        s.solve(want_labels=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, _, inf = s.solve(want_labels=False)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        op = time_operator(B, s, dev, stream, g, s_v, s_x, (args.block,), peak, reps=20)[f"nvec{args.block}"]
        s.close()
        out.append({"h": hh, "solve_s": t, "matvecs": inf["matvecs"], "restarts": inf["restarts"],
                    "ms_operator_total": inf["ms_operator"], "ms_orth_total": inf["ms_orth"],
                    "operator_us": op["us"], "max_resid": inf["max_resid"]})
    base = out[0]["solve_s"]
    for r in out:
        r["vs_sc"] = r["solve_s"] / base
    return {"graph": "msbm_n1m_k50_h10 edges; groups merged as g mod h (h = 1: plain SC)", "prec": args.prec,
            "block": args.block, "rows": out}


def backward_bench(dev, peak):
    """The differentiation form on the n = 200,000, k = 10, h = 4 Gaussian-weight workload: forward
    solve time (MIXED) and the SDDMM backward (weights and bandwidth) time and algorithmic GB/s."""
    import numpy as np
    import torch

    from msbm import configs
    from paper_2210_16435_gb300.solver import FairSC

    c = configs.msbm_n200k_k10_h4_gauss()
    g, k, h, bw = c["graph"], c["k"], c["h"], c["bandwidth"]
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    rp, ci, v, gr = T(g.row_ptr, torch.int32), T(g.col_idx, torch.int32), T(g.values, torch.float32), \
        T(g.groups, torch.int32)
    s = FairSC(rp, ci, v, gr, k=k, h=h, prec="mixed")
    s.solve(want_labels=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, _, _, inf = s.solve(want_labels=False)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    gl = torch.ones(k, dtype=torch.float64, device=dev)
    for _ in range(3):
        s.backward(gl, bw)
    stream = torch.cuda.current_stream()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    torch.cuda.synchronize()
    a0.record(stream)
    for _ in range(reps):
        s.backward(gl, bw)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1) / reps
    s.close()
    # the eigenvector-level backward (a loss on H): k conjugate-gradient solves on the FP64 operator + SDDMM,
    # deflated with the eigenvectors of an FP64 solve at 1e-12 sigma (the solves need them that accurate)
    s = FairSC(rp, ci, v, gr, k=k, h=h, prec="fp64", tol=1e-12)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.solve(want_labels=False)
    torch.cuda.synchronize()
    t_fwd64 = time.perf_counter() - t0
    Gh = torch.randn(g.n, k, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    s.backward_vectors(Gh, gl, bw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, cg_it, cg_rr = s.backward_vectors(Gh, gl, bw)
    torch.cuda.synchronize()
    vec_s = time.perf_counter() - t0
    s.close()
    # stored entries: column index + FP32 weight read, FP64 gradient written; H rows read once per row
    bytes_ = g.nnz * (4 + 4) + g.n * k * 8 + g.nnz * 8 + 4 * (g.n + 1)
    gbs = bytes_ / (ms * 1e6)
    return {"workload": "msbm_n200k_k10_h4_gauss", "n": g.n, "nnz": g.nnz, "k": k, "forward_solve_s": t_fwd,
            "forward_restarts": inf["restarts"], "backward_ms": ms, "backward_bytes": bytes_,
            "achieved_gbs": gbs, "frac": gbs / peak, "vector_forward_fp64_s": t_fwd64, "vector_backward_s": vec_s,
            "vector_backward_cg_iterations": cg_it,
            "vector_backward_cg_rel_resid": cg_rr,
            "fd_check": "tests/test_gpu_backward.py::test_differentiation_workload_full_size"}


def _timed_solve(FairSC, args, kw, reps=3):
    """Median wall time of create + solve (labels included) after one untimed run."""
    import torch

    def once():
        s = FairSC(*args, **kw)
        out = s.solve()
        s.close()
        return out

    once()
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = once()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts), out


def random_laplacian_bench(dev):
    """Exp. 4: random sparse W (mean degree 100, weights U(0, 1]) and a random dense F (h = 5), n from
    5,000 to 10,000, k in {5, 8, 10}: time of s-FairSC (dense-constraint context) and of SC (no
    constraint) on the GPU, FP64, residual 1e-6 sigma."""
    import numpy as np
    import torch

    from msbm import configs
    from paper_2210_16435_gb300.solver import FairSC

    rows = []
    for n in (5000, 7500, 10000):
        c = configs.random_laplacian(n, 5, seed=1)
        g, F = c["graph"], c["F"]
        T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        args = (T(g.row_ptr, torch.int32), T(g.col_idx, torch.int32), T(g.values, torch.float64))
        zero = torch.zeros(g.n, dtype=torch.int32, device=dev)
        Ft = T(F, torch.float64)
        for k in (5, 8, 10):
            t_fair, (_, _, _, inf) = _timed_solve(FairSC, args + (None,), dict(k=k, prec="fp64", F=Ft))
            t_sc, (_, _, _, inf0) = _timed_solve(FairSC, args + (zero,), dict(k=k, h=1, prec="fp64"))
            rows.append({"n": n, "k": k, "nnz": g.nnz, "sfairsc_s": t_fair, "sc_s": t_sc, "ratio": t_fair / t_sc,
                         "sfairsc_matvecs": inf["matvecs"], "sc_matvecs": inf0["matvecs"],
                         "fairness_err": inf["fairness_err"]})
    return {"workload": "random Laplacian (mean degree 100), random dense F with h = 5 (Exp. 4)", "rows": rows}


def paper_msbm_bench(dev, sizes=(1000, 2000, 4000, 10000), fairsc_max_n=2000):
    """Exp. 1 / App. C: m-SBM with k = 5, h in {2, 5, 10}, probabilities (10, 7, 4, 1) (log n / n)^(2/3):
    error rate (eq. err) and average balance (eq. avebal) of s-FairSC and SC on the GPU (FP64,
    k-means with 10 replicates) and of the oracle's dense FairSC (Algorithm 2) on the host up to
    n = fairsc_max_n, with the times of each."""
    import numpy as np
    import torch

    from msbm import configs
    from oracle import fairsc
    from oracle.kmeans import kmeans as oracle_kmeans
    from oracle.metrics import average_balance, error_rate
    from paper_2210_16435_gb300.solver import FairSC

    rows = []
    for h in (2, 5, 10):
        for n in sizes:
            c = configs.paper_msbm(n, h)
            g, k = c["graph"], c["k"]
            T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
            args = (T(g.row_ptr, torch.int32), T(g.col_idx, torch.int32), T(g.values, torch.float64))
            kw = dict(k=k, prec="fp64", kmeans_n_init=10, kmeans_max_iter=300)
            t_fair, (_, _, lab, _) = _timed_solve(FairSC, args + (T(g.groups, torch.int32),), dict(kw, h=h))
            t_sc, (_, _, lab_sc, _) = _timed_solve(FairSC, args + (T(g.groups * 0, torch.int32),), dict(kw, h=1))
            lab, lab_sc = lab.cpu().numpy(), lab_sc.cpu().numpy()
            row = {"n": n, "h": h, "nnz": g.nnz, "sfairsc_gpu_s": t_fair, "sc_gpu_s": t_sc,
                   "err_sfairsc": error_rate(lab, g.clusters, k), "err_sc": error_rate(lab_sc, g.clusters, k),
                   "bal_sfairsc": average_balance(lab, g.groups, k, h),
                   "bal_sc": average_balance(lab_sc, g.groups, k, h)}
            if n <= fairsc_max_n:
                t0 = time.perf_counter()
                _, Hf = fairsc.fairsc_dense(g.to_scipy(), g.groups, h, k)
                lf, _, _ = oracle_kmeans(Hf, k, seed=0, n_init=10, max_iter=300)
                row["fairsc_host_s"] = time.perf_counter() - t0
                row["err_fairsc"] = error_rate(lf, g.clusters, k)
                row["bal_fairsc"] = average_balance(lf, g.groups, k, h)
            rows.append(row)
    return {"workload": "m-SBM k = 5, h in {2, 5, 10}, (a, b, c, d) = (10, 7, 4, 1) (log n / n)^(2/3)", "rows": rows}


def step_breakdown(FairSC, inputs, outs, kw):
    """Wall-clock milliseconds of create, solve and close for one step (synchronised between the
    calls), with the solve's own CUDA-event times of the eigensolve and the k-means."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = FairSC(*inputs, **kw)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    _, _, _, info = s.solve(out=outs) if outs is not None else s.solve()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    s.close()
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    return {"create_ms": (t1 - t0) * 1e3, "solve_call_ms": (t2 - t1) * 1e3, "close_ms": (t3 - t2) * 1e3,
            "solve_events_ms": info["ms_solve"], "kmeans_events_ms": info["ms_kmeans"]}


def cpu_baseline(args, c, FairSC, rp, ci, v, gr, kw):
    """The oracle on the host cores at the bench workload: setup + its own Lanczos to
    1e-6 sigma (complete, timed, all threads) + embedding + k-means (seeding and three
    Lloyd assignments timed on the library's H, scaled to the assignment count of the
    identical k-means on that H); and the same on one thread (first two cycles timed)."""
    from oracle.sfairsc import embed

    g, k = c["graph"], c["k"]
    cores = host_threads()
    r = oracle_solve_timed(g, k, tol=1e-6)
    t0 = time.perf_counter()
    embed(r["op"], r["X"])
    t_embed = time.perf_counter() - t0
    s = FairSC(rp, ci, v, gr, **dict(kw, profile=0))
    _, H, _, inf = s.solve()
    s.close()
    t_km, _, km_text = oracle_kmeans_timed(H.cpu().numpy(), k, full=False, sample_iters=3,
                                           iters_total=max(1, inf["kmeans_iters"]))
    value = r["setup_s"] + r["solve_s"] + t_embed + t_km
    out = {"value": value, "unit": "s/solve", "cores": cores, "kind": "oracle",
           "sample": (f"complete oracle solve of the full graph on {cores} host threads: setup {r['setup_s']:.1f}s, "
                      f"{len(r['cycle_s'])} Lanczos cycles {r['solve_s']:.1f}s ({r['matvecs']} matvecs, "
                      f"{r['restarts']} restarts) to 1e-6 sigma; embedding {t_embed:.2f}s; k-means: {km_text}"),
           "matvecs": r["matvecs"], "restarts": r["restarts"], "setup_s": r["setup_s"], "solve_s": r["solve_s"],
           "kmeans_s": t_km}
    st, st_text = oracle_single_thread(g, k, len(r["cycle_s"]))
    if st is not None:
        out["single_thread"] = {"value": st + t_embed + t_km, "unit": "s/solve", "cores": 1, "kind": "oracle",
                                "sample": st_text + "; embedding and k-means as above (single-threaded NumPy)"}
    return out


def fairsc_c1(FairSC, dev):
    """Context for the paper's FairSC-vs-s-FairSC comparison (Exp. 1) at n = 2,000, k = 5, h = 2:
    dense FairSC (Algorithm 2) and the sparse s-FairSC oracle on the host, and the library's
    FP64 solve on the GPU."""
    import numpy as np
    import torch

    from msbm import configs
    from oracle import fairsc
    from oracle.sfairsc import operator_from_graph, smallest_eigenpairs

    c = configs.msbm_n2000_k5_h2()
    g, k, h = c["graph"], c["k"], c["h"]
    W = g.to_scipy()
    t0 = time.perf_counter()
    fairsc.fairsc_dense(W, g.groups, h, k)
    t_dense = time.perf_counter() - t0
    t0 = time.perf_counter()
    op = operator_from_graph(g)
    smallest_eigenpairs(op, k, tol=1e-6, method="lanczos")
    t_sparse = time.perf_counter() - t0
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    args = (T(g.row_ptr, torch.int32), T(g.col_idx, torch.int32), T(g.values, torch.float64), T(g.groups, torch.int32))
    FairSC(*args, k=k, h=h, prec="fp64").close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = FairSC(*args, k=k, h=h, prec="fp64")
    s.solve(want_labels=False)
    s.close()
    torch.cuda.synchronize()
    t_gpu = time.perf_counter() - t0
    return {"workload": "msbm_n2000_k5_h2", "fairsc_dense_host_s": t_dense, "sfairsc_oracle_host_s": t_sparse,
            "sfairsc_gpu_fp64_s": t_gpu, "host_threads": host_threads()}


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2210_16435_gb300 import buildlib

    buildlib.build()
    from paper_2210_16435_gb300 import binding as B
    from paper_2210_16435_gb300.solver import FairSC

    c = load_workload(args.workload, args.scale)
    g, k, h = c["graph"], c["k"], c["h"]
    vdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[c["value_dtype"]]
    dev = torch.device("cuda", torch.cuda.current_device())
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    rp, ci, v, gr = T(g.row_ptr, torch.int32), T(g.col_idx, torch.int32), T(g.values, vdt), T(g.groups, torch.int32)
    kw = dict(k=k, h=h, prec=args.prec, block=args.block, profile=1)

    def step():
        s = FairSC(rp, ci, v, gr, **kw)
        lam, H, lab, info = s.solve()
        s.close()
        return info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        infos.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = ms / 1e3 / world  # seconds per solve at the job level (world replicas per step)

    s_x = 8 if args.prec == "fp64" else 4
    s_v = VDT_BYTES[c["value_dtype"]] if not (args.prec == "mixed" and c["value_dtype"] == "f64") else 4
    inf = infos[-1]
    b = inf["block"]
    op_avg_ms = sum(i["ms_operator"] for i in infos) / max(1, sum(i["n_operator"] for i in infos))
    orth_avg_ms = sum(i["ms_orth"] for i in infos) / max(1, sum(i["n_orth"] for i in infos))
    op_bytes = operator_bytes(g.n, g.nnz, s_v, s_x, b)
    orth_b = orth_bytes(g.n, inf["orth_cols"], inf["n_orth"], inf["orth_sweeps"], s_x, b) / max(1, inf["n_orth"])
    peak, peak_kind = measured_peaks()
    op_gbs = op_bytes / (op_avg_ms * 1e6)
    orth_gbs = orth_b / (orth_avg_ms * 1e6)
    t_op = sum(i["ms_operator"] for i in infos)
    t_orth = sum(i["ms_orth"] for i in infos)
    if t_orth >= t_op:
        traffic = None
        if args.workload == "msbm_n1m_k50_h10" and args.scale == 1.0 and args.prec == "mixed" and args.block == 4:
            traffic = recorded_traffic("orth_kernel_msbm_n1m_k50_h10.md",
                                       ["paper_2210_16435_gb300/csrc/orth.cu", "paper_2210_16435_gb300/csrc/common.cuh"])
        roof = {"kernel": "orth_kernel (CGS2 + CholQR)", "bound": "hbm", "achieved": orth_gbs, "peak": peak,
                "unit": "GB/s", "frac": orth_gbs / peak, "traffic": traffic,
                "bytes_per_launch": orth_b, "ms_per_launch": orth_avg_ms}
    else:
        roof = {"kernel": "fused_operator_kernel", "bound": "hbm", "achieved": op_gbs, "peak": peak, "unit": "GB/s",
                "frac": op_gbs / peak, "traffic": None, "bytes_per_launch": op_bytes, "ms_per_launch": op_avg_ms}
    roof["peak_kind"] = f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind
    launches = sum(i["n_launches"] for i in infos) + 5 * args.steps  # + create: validate, degrees, sigma, partition, (convert)

    line = {
        "metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.prec == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": args.workload if args.scale == 1.0 else f"{args.workload}@scale{args.scale}",
                   "n": g.n, "nnz": g.nnz, "k": k, "h": h, "prec": args.prec,
                   "block": b, "basis": inf["basis"], "tol": 1e-6, "values": c["value_dtype"],
                   "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (CSR 192 MB, basis 400+ MB)"},
        "roofline": roof, "clocks": clk, "gpu_launches": launches,
        "solve": {"restarts": inf["restarts"], "matvecs": inf["matvecs"], "max_resid": inf["max_resid"],
                  "fairness_err": inf["fairness_err"], "dorth_err": inf["dorth_err"],
                  "ms_solve": inf["ms_solve"], "ms_kmeans": inf["ms_kmeans"], "kmeans_iters": inf["kmeans_iters"],
                  "ms_operator_total": inf["ms_operator"], "ms_orth_total": inf["ms_orth"],
                  "ms_restart_total": inf["ms_restart"], "ms_host_eig_total": inf["ms_host_eig"],
                  "ms_final": inf["ms_final"], "orth_sweeps": inf["orth_sweeps"], "n_orth": inf["n_orth"]},
        "operator_in_solve": {"achieved_gbs": op_gbs, "frac": op_gbs / peak, "ms_per_launch": op_avg_ms,
                              "bytes_per_launch": op_bytes},
    }
    if rank == 0 and not args.no_extras:
        # standalone fused operator on the workload (the metric's operator GB/s), b = 1 and 4
        s = FairSC(rp, ci, v, gr, k=k, h=h, prec=args.prec, block=args.block)
        opx = time_operator(B, s, dev, stream, g, s_v, s_x, (1, 4), peak)
        s.close()
        # the same with shared-memory windows of the input vector (static row ranges), for comparison
        s = FairSC(rp, ci, v, gr, k=k, h=h, prec=args.prec, block=args.block, spmv_window=1)
        line["operator_windows"] = time_operator(B, s, dev, stream, g, s_v, s_x, (1, 4), peak)
        s.close()
        line["operator"] = opx
        # plain FP64 GPU path on the same graph, block 1 and block 4 (block 4 isolates the precision effect)
        for blk in (1, 4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = FairSC(rp, ci, v, gr, k=k, h=h, prec="fp64", block=blk)
            _, _, _, i64 = s.solve()
            torch.cuda.synchronize()
            line[f"fp64_block{blk}_solve_s"] = time.perf_counter() - t0
            line[f"fp64_block{blk}_info"] = {"restarts": i64["restarts"], "matvecs": i64["matvecs"],
                                             "max_resid": i64["max_resid"], "ms_final": i64["ms_final"]}
            s.close()
        # the FP64 operator alone (the final residual check and the plain FP64 path use it)
        s = FairSC(rp, ci, v, gr, k=k, h=h, prec="fp64", block=4)
        line["operator_fp64"] = time_operator(B, s, dev, stream, g, VDT_BYTES[c["value_dtype"]], 8, (1, 4), peak)
        s.close()
        # s-FairSC against plain SC on the same graph (the paper's overhead question, Exp. 1/4, App. C):
        # the same W with its groups merged to h = 5, 2 and 1 (h = 1: no fairness constraint, Algorithm 1)
        line["h_sweep"] = h_sweep(FairSC, B, dev, stream, g, rp, ci, v, k, h, args, s_v, s_x, peak)
        # differentiation form: gradient of the sum of the 10 smallest eigenvalues at n = 200,000
        line["backward"] = backward_bench(dev, peak)
        # Exp. 4: random Laplacian with a random dense F, s-FairSC against SC on the GPU
        line["random_laplacian"] = random_laplacian_bench(dev)
        # Exp. 1 / App. C: the experiments' m-SBM, s-FairSC and SC on the GPU, FairSC on the host
        line["paper_msbm"] = paper_msbm_bench(dev)
        # end to end through the C ABI with host buffers: copies inside the timed region
        hp = [torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
              for a, dt in ((g.row_ptr, torch.int32), (g.col_idx, torch.int32), (g.values, vdt),
                            (g.groups, torch.int32))]
        # pinned output buffers owned by the caller, allocated once (as a serving loop would)
        outs = (torch.empty(k, dtype=torch.float64).pin_memory(), torch.empty(g.n, k, dtype=torch.float64).pin_memory(),
                torch.empty(g.n, dtype=torch.int32).pin_memory())
        ne = max(1, min(3, args.steps))
        s = FairSC(*hp, k=k, h=h, prec=args.prec, block=args.block)  # untimed warm-up of the host path
        s.solve(out=outs)
        s.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ne):
            s = FairSC(*hp, k=k, h=h, prec=args.prec, block=args.block)
            lam, H, lab, _ = s.solve(out=outs)
            s.close()
        torch.cuda.synchronize()
        e2e = (time.perf_counter() - t0) / ne
        h2d = 4 * (g.n + 1) + 4 * g.nnz + VDT_BYTES[c["value_dtype"]] * g.nnz + 4 * g.n
        d2h = 8 * k + 8 * g.n * k + 4 * g.n
        line["e2e"] = {"value": e2e, "unit": "s/solve", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        # untimed: one step on each path split into its calls, the device synchronised between them
        # (where the end-to-end time above the device-resident value goes)
        try:
            kw_e2e = dict(k=k, h=h, prec=args.prec, block=args.block)
            line["e2e_breakdown"] = {"device_inputs": step_breakdown(FairSC, (rp, ci, v, gr), None, kw_e2e),
                                     "host_inputs": step_breakdown(FairSC, hp, outs, kw_e2e)}
        except Exception as ex:  # a diagnostic: it never costs the bench line
            line["e2e_breakdown"] = {"error": repr(ex)}
        # batched form (256 graphs, one launch) against sequential single-graph solves
        if not args.no_batched:
            line["batched"] = batched_extra(dev, peak)
        # the CPU oracle on the host cores: a complete, timed solve of the same graph
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(args, c, FairSC, rp, ci, v, gr, kw)
            line["fairsc_c1"] = fairsc_c1(FairSC, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_only(args):
    """--only operator: the standalone fused operator on the workload (nvec vectors, reps calls timed
    with CUDA events after 3 untimed ones); --only solve: one create + solve with per-phase timing."""
    import numpy as np
    import torch

    torch.cuda.set_device(0)
    from paper_2210_16435_gb300 import binding as B
    from paper_2210_16435_gb300 import buildlib

    buildlib.build()
    from paper_2210_16435_gb300.solver import FairSC

    c = load_workload(args.workload, args.scale)
    g, k, h = c["graph"], c["k"], c["h"]
    vdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[c["value_dtype"]]
    T = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    s = FairSC(T(g.row_ptr, torch.int32), T(g.col_idx, torch.int32), T(g.values, vdt), T(g.groups, torch.int32),
               k=k, h=h, prec=args.prec, block=args.block, spmv_window=args.window, profile=1)
    if args.only == "operator":
        W = torch.randn(args.nvec, g.n, device="cuda", dtype=s.vec_dtype)
        O = torch.empty_like(W)
        for _ in range(3):
            B.sfairsc_apply_operator(s.ctx, W.data_ptr(), O.data_ptr(), args.nvec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            B.sfairsc_apply_operator(s.ctx, W.data_ptr(), O.data_ptr(), args.nvec)
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / args.reps * 1e3
        s_x = 8 if args.prec == "fp64" else 4
        ob = operator_bytes(g.n, g.nnz, VDT_BYTES[c["value_dtype"]], s_x, args.nvec)
        print(json.dumps({"only": "operator", "workload": args.workload, "nvec": args.nvec, "prec": args.prec,
                          "window": args.window, "us": us, "gbs": ob / (us * 1e3)}), flush=True)
    else:
        _, _, _, inf = s.solve(want_labels=False)
        print(json.dumps({"only": "solve", "workload": args.workload, **inf}), flush=True)
    s.close()


def main():
    args = parse()
    if args.cpu_child:
        oracle_single_thread_child(args)
        return
    if args.only:
        run_only(args)
        return
    if args.workload == "msbm_batch256" and args.impl != "reference":
        run_batched_main(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
