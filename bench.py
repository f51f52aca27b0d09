#!/usr/bin/env python3
"""Throughput of the GaBP SVM solver on one GB300 (or N independent replicas).

A step is one complete solve of the n=20000, m=128 FP32 mixture workload
(gamma = 1/128, C = 10, Q stored FP32, 100 synchronous rounds): input
staging, Q formation with the weighted diagonal, 100 broadcast-GaBP rounds
(pair sweep + per-node finalize each), and the final FP64 residual, dual
objective and alpha.  `value` is synchronous rounds ("sweeps") per second over
all ranks, with the inputs resident on the device; `e2e` is the same through
the C ABI with pinned host buffers (H2D of X and y, D2H of alpha inside the
timed region).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank solves its own instance (no collective): weak
scaling, `value` = all ranks' sweeps / max elapsed over ranks.
`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_0810_1648_gb300 import workloads  # noqa: E402

METRIC = "GaBP sweeps/sec (n² edge updates/s, % HBM roofline); solves/s + p50/p99 vs plain"
UNIT = "sweeps/s"
ROUNDS = 100
PROFILE_STRIDE = 4   # sweeps timed by events: every 4th round of the timed solves
WORKLOAD = {
    "workload": "plain GaBP SVM, n=20000, m=128 FP32 two-class 3-component Gaussian mixture "
                "(means N(0,1), sigma 0.7), RBF gamma=1/128, C=10, Q stored FP32 upper triangle, "
                "100 synchronous sweeps per solve, seed 1",
    "n": 20000, "m": 128, "sweeps_per_step": ROUNDS, "q_mode": "f32",
    "l2": "no flush: every sweep streams 3.3 GB of messages + 0.8 GB of Q, far above the 129 MB L2",
}
PRECISION_WORKLOAD = {
    "workload": "precision form, n=100000, m=64 FP32 3-component mixture (seed 2), RBF gamma=0.5/64, C=1, "
                "100 synchronous sweeps per solve, Q as selected by q_mode",
    "n": 100000, "m": 64, "sweeps_per_step": ROUNDS,
    "l2": "no flush: every sweep streams 80 GB of messages, far above the 129 MB L2",
}
# Stored bytes of one Q entry per unordered pair, by Q mode.
Q_BYTES = {"f32": 4, "bf16": 2, "recompute": 0}
Q_MODES = {"f32": 0, "bf16": 1, "recompute": 2}
T_TILE = 128   # tile edge of the stored upper triangle
TASKS = {"svm": 0, "krr": 1}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _job_rate(units, ms, ws, device):
    """Whole-job rate over all ranks: the units every rank processed, summed,
    over the slowest rank's elapsed time (max over ranks).  Returns (rate per
    second, max ms)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return float(u.item()) / (ms_max / 1e3), ms_max


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# The sources the pair sweep is compiled from: sweep.cu and the headers it
# includes.  The profile summaries record the SHA-256 of their concatenation.
SWEEP_SOURCES = ("sweep.cu", "common.cuh", "ptx.cuh", "qtile_epi.cuh")


def sweep_source_sha() -> str:
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_0810_1648_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic_from_profile():
    """DRAM bytes per launch of the pair sweep from the committed ncu summary,
    or None when the kernel sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "k_sweep_plain_large.txt")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m_sha = re.search(r"^source_sha256:\s*([0-9a-f]+)", txt, re.M)
    m_b = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt, re.M)
    if not (m_sha and m_b):
        return None
    return float(m_b.group(1)) if sweep_source_sha() == m_sha.group(1) else None


def _peak_gbs() -> float:
    """Measured HBM copy bandwidth of the GB300s, else the fallback."""
    peaks = _peaks()
    return float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6800.0


def _oracle_sample(p, sweeps: int, single: bool = False):
    """Times the FP64 oracle: Q formation for the whole set + `sweeps` rounds.
    Returns (t_q, t_per_sweep, threads[, t_per_sweep with one thread])."""
    import oracle
    X = p.X.astype(np.float64)
    y = p.y.astype(np.float64)
    t0 = time.perf_counter()
    Q = oracle.build_q(X, y, p.gamma, p.C)
    t1 = time.perf_counter()
    oracle.gabp(Q, np.ones(p.n), iters=sweeps, tol=0.0)
    t2 = time.perf_counter()
    th = oracle.threads()
    if not single:
        del Q
        return t1 - t0, (t2 - t1) / max(sweeps, 1), th
    oracle.set_threads(1)
    try:
        t3 = time.perf_counter()
        oracle.gabp(Q, np.ones(p.n), iters=1, tol=0.0)
        t4 = time.perf_counter()
    finally:
        oracle.set_threads(th)
    del Q
    return t1 - t0, (t2 - t1) / max(sweeps, 1), th, t4 - t3


def _host_mem_gb():
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def _cpu_baseline(p, sweeps: int):
    need_gb = 3 * 8 * p.n * p.n / 1e9 + 1
    if _host_mem_gb() < need_gb * 1.3:
        return {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                "sample": f"skipped: the FP64 oracle needs {need_gb:.0f} GB of host memory"}
    tq, ts, th, t1 = _oracle_sample(p, sweeps, single=True)
    v = ROUNDS / (tq + ROUNDS * ts)
    return {"value": v, "unit": UNIT, "cores": th, "kind": "oracle",
            "sample": f"FP64 oracle on the same workload: Q formation for all n=20000 points "
                      f"({tq:.1f} s) + {sweeps} synchronous rounds ({ts:.2f} s each), "
                      f"scaled to one {ROUNDS}-round solve",
            "single_thread_s_per_sweep": t1}


def run_reference(args):
    """The FP64 oracle on the same workload.  A step is `--ref-sweeps`
    synchronous rounds (one by default) over all n=20000 points, timed as
    run; Q is formed once before the timed region (its time is reported
    beside the rate, and a 100-round solve with formation is extrapolated
    under its own key)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    p = workloads.plain_large()
    sweeps = max(1, args.ref_sweeps)
    X = p.X.astype(np.float64)
    y = p.y.astype(np.float64)
    t0 = time.perf_counter()
    Q = oracle.build_q(X, y, p.gamma, p.C)
    t_form = time.perf_counter() - t0
    b = np.ones(p.n)
    for _ in range(args.warmup):
        oracle.gabp(Q, b, iters=sweeps, tol=0.0)
    secs = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.gabp(Q, b, iters=sweeps, tol=0.0)
        secs.append(time.perf_counter() - t0)
    th = oracle.threads()
    del Q
    total = float(np.sum(secs))
    v = args.steps * sweeps / total
    per_sweep = total / (args.steps * sweeps)
    sample = (f"FP64 oracle ({th} threads): {sweeps} synchronous round(s) over all n=20000 points per step, "
              f"Q formed once before the timed steps ({t_form:.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, parallelism=f"replicas{ws}"),
            "sweeps_per_timed_step": sweeps,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "formation_s": t_form,
            "extrapolated_ms_per_solve": {"value": 1e3 * (t_form + ROUNDS * per_sweep),
                                          "note": f"Q formation + {ROUNDS} rounds at the measured rate "
                                                  "(extrapolated, not timed)"}}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_small(args):
    """One short solve on a smaller set (n=6144 by default, --profile-n; 8
    rounds, so that the last rounds run with frozen P messages) for ncu
    captures: the message state (0.3 GB at n=6144) is still above L2, the
    device footprint small."""
    import torch

    from paper_0810_1648_gb300 import build as gbuild
    from paper_0810_1648_gb300 import gabp
    if not os.path.exists(gabp.LIB_PATH):
        gbuild.build()
    n = args.profile_n
    p = workloads.mixture(n, 128, seed=1, gamma=1.0 / 128, C=10.0)
    h = gabp.svm_create(p.X, p.y, p.gamma, p.C, gabp.opts_default(chunk=8, q_mode=Q_MODES[args.q_mode],
                                                                 msg_bf16=1 if args.msg_bf16 else 0))
    alpha = np.empty(p.n, dtype=np.float32)
    rinf, k = gabp.svm_solve(h, 8, 0.0, alpha)
    gabp.svm_destroy(h)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": f"n={n} m=128 mixture, 8 rounds, q_mode {args.q_mode}", "rounds": k,
                      "residual_inf": rinf}), flush=True)
    return 0


def run_batch(args):
    """512 uneven instances (32 data sets x C in {0.1,1,10,100} x gamma in
    {0.1,0.5,1,2}/m, n log-uniform in [200, 4000], m in {8,32,128,256}) solved
    together to ||r||_inf < 1e-6 or 200 rounds: plain FP32 vs the BF16
    tensor-core form with refinement to the same tolerance.  Metric: solves/s."""
    import torch

    from paper_0810_1648_gb300 import build as gbuild
    from paper_0810_1648_gb300 import gabp
    if not os.path.exists(gabp.LIB_PATH):
        gbuild.build()
    probs = workloads.batch_grid()
    # inputs resident in device memory for the timed solves (device pointer
    # mode); the grid points of a data set pass the same device arrays, as a
    # parameter search would, so the solver forms their Gram tiles once
    dev = {}
    for p in probs:
        if id(p.X) not in dev:
            dev[id(p.X)] = (torch.from_numpy(p.X).cuda(), torch.from_numpy(p.y).cuda())
    dprobs = [workloads.Problem(*dev[id(p.X)], p.gamma, p.C) for p in probs]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    out = {}
    st = args.stages if args.stages > 1 else 4
    all_modes = (("f32", dict(q_mode=0)), ("bf16q_refined", dict(q_mode=1, refine=8)),
                 ("bf16_refined", dict(q_mode=1, refine=8, msg_bf16=1)),
                 ("f32_staged", dict(q_mode=0, stages=st)),
                 ("bf16_refined_staged", dict(q_mode=1, refine=8, msg_bf16=1, stages=st)))
    chosen = args.batch_modes.split(",") if args.batch_modes else [m for m, _ in all_modes]
    for mode, kw in all_modes:
        if mode not in chosen:
            continue
        for _ in range(args.warmup):
            gabp.batch_solve(dprobs, 200, 1e-6, chunk=0, stream=stream.cuda_stream, **kw)
        times, last = [], None
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            alphas, res, rc = gabp.batch_solve(dprobs, 200, 1e-6, chunk=0, stream=stream.cuda_stream, **kw)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            last = res
        conv = sum(r["converged"] for r in last)
        ph = gabp.batch_last_phases()
        # algorithmic bytes of all the rounds run, per pair and round: Q once,
        # the message state read once and written once while P changes, only
        # H written after the exact P-freeze (a few rounds in): the two give a
        # range, since the freeze round of each instance is not reported
        qb = 2 if kw.get("q_mode", 0) == 1 else 4
        ms = 4 if kw.get("msg_bf16") else 8
        b_live, b_frozen = qb + 4 * ms, qb + 3 * ms
        pair_rounds = sum(r["iters_done"] * p.n * (p.n - 1) / 2 for p, r in zip(probs, last))
        rs = ph["rounds_ms"] / 1e3
        out[mode] = {"solves_per_s": len(probs) / float(np.median(times)), "ms_per_batch": 1e3 * float(np.median(times)),
                     "phases_ms": ph,
                     "converged": conv, "max_residual": max(r["residual_inf"] for r in last),
                     "mean_rounds": float(np.mean([r["iters_done"] for r in last])),
                     "rounds_hbm": {"pair_rounds": pair_rounds, "bytes_per_pair_round": [b_frozen, b_live],
                                    "GBps_over_rounds_phase": [pair_rounds * b / rs / 1e9 for b in (b_frozen, b_live)],
                                    "frac_of_measured_peak": [pair_rounds * b / rs / 1e9 / _peak_gbs()
                                                              for b in (b_frozen, b_live)]}}
    # end to end: host (numpy) inputs, their copies inside the timed solves
    e2e_t = []
    kw_e2e = dict(q_mode=1, refine=8, msg_bf16=1)
    if "bf16_refined" in out:
        gabp.batch_solve(probs, 200, 1e-6, chunk=0, stream=stream.cuda_stream, **kw_e2e)
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gabp.batch_solve(probs, 200, 1e-6, chunk=0, stream=stream.cuda_stream, **kw_e2e)
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t0)

    def ratio(a, b):
        return out[a]["solves_per_s"] / out[b]["solves_per_s"] if a in out and b in out else None
    h2d = int(sum(p.X.nbytes + p.y.nbytes for p in probs))
    n2 = sum(p.n * p.n for p in probs)
    head = "bf16_refined" if "bf16_refined" in out else next(iter(out))
    line = {"metric": METRIC, "value": out[head]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
            "config": {"workload": "batched form: 512 instances, 32 mixture data sets x C {0.1,1,10,100} x "
                                   "gamma {0.1,0.5,1,2}/m, n log-uniform [200,4000], m in {8,32,128,256}, "
                                   "tol 1e-6 or 200 rounds, one persistent launch per round, autotuned schedule; "
                                   "modes: plain FP32; BF16 Q + refinement; BF16 Q and BF16 messages + refinement "
                                   "(all to ||1 - Q mu||_inf < 1e-6 with the FP32-Gram Q), under the synchronous "
                                   f"schedule and the {st}-stage block Gauss-Seidel schedule",
                       "instances": len(probs), "sum_n2": n2, "stages": st},
            "value_mode": head, "modes": out, "bf16_over_f32": ratio("bf16_refined", "f32"),
            "e2e": ({"value": len(probs) / float(np.median(e2e_t)), "unit": "solves/s", "mode": "bf16_refined",
                     "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(sum(4 * p.n for p in probs))}
                    if e2e_t else None),
            "bf16_over_f32_staged": ratio("bf16_refined_staged", "f32_staged"),
            "staged_over_synchronous": {"f32": ratio("f32_staged", "f32"),
                                        "bf16": ratio("bf16_refined_staged", "bf16_refined")}}
    print(json.dumps(line), flush=True)
    return 0


def run_sparse(args):
    """Tile-sparse kernel on clustered data.  Default (--sparse-n 20000):
    n=20000, m=64 mixture with rows grouped by component, gamma=0.15, C=1,
    tau=1e-3, against the dense solve of the same data.  --sparse-n 200000:
    six tight clusters (sigma 0.5), gamma=0.3, tau=5e-5, a size whose dense
    message state (8 n^2 bytes) exceeds the device, so no dense solve beside
    it.  Reports sweeps/s of 100 synchronous rounds (inputs resident on the
    device, CUDA events), the HBM fraction of the sparse sweep for the pairs
    of its kept tiles, the device memory held, the time to ||r||_inf < 1e-6
    and the stated error bound."""
    import torch

    from paper_0810_1648_gb300 import build as gbuild
    from paper_0810_1648_gb300 import gabp
    if not os.path.exists(gabp.LIB_PATH):
        gbuild.build()
    gabp.load()
    big = args.sparse_n > 20000
    if big:
        tau = 5e-5
        comps = args.sparse_comps
        p = workloads.clustered_mixture(args.sparse_n, 64, seed=5, gamma=0.3, C=1.0, comps=comps, sigma=0.5)
        names = (("tile_sparse", tau),)
        desc = (f"tile-sparse kernel: n={p.n}, m=64 mixture ({comps} components per class, sigma 0.5, seed 5) with "
                f"rows grouped by component, RBF gamma=0.3, C=1, tiles with max |Q_ij| <= {tau} dropped; "
                "100 synchronous sweeps per step; the dense message state (8 n^2 bytes) exceeds the device")
    else:
        tau = 1e-3
        p = workloads.clustered_mixture(args.sparse_n, 64, seed=5, gamma=0.15, C=1.0)
        names = (("dense", 0.0), ("tile_sparse", tau))
        desc = (f"tile-sparse kernel: n={p.n}, m=64 mixture (3 components per class, sigma 0.7, seed 5) with "
                f"rows grouped by component, RBF gamma=0.15, C=1, tiles with max |Q_ij| <= {tau} dropped; "
                "100 synchronous sweeps per step; dense solve of the same data beside it")
    Xd, yd = torch.from_numpy(p.X).cuda(), torch.from_numpy(p.y).cuda()
    stream = torch.cuda.Stream()
    alpha = torch.empty(p.n, dtype=torch.float32, device="cuda")
    out, answers = {}, {}
    for name, st in names:
        opts = gabp.opts_default(stream=stream.cuda_stream, chunk=ROUNDS, sparse_tau=st)
        h = gabp.svm_create(Xd, yd, p.gamma, p.C, opts)
        gabp.svm_set_profiling(h, PROFILE_STRIDE)
        for _ in range(args.warmup):
            gabp.svm_refit(h, Xd, yd, p.gamma, p.C)
            gabp.svm_solve(h, ROUNDS, 0.0, alpha)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gabp.svm_get_profile(h, reset=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            gabp.svm_refit(h, Xd, yd, p.gamma, p.C)
            gabp.svm_solve(h, ROUNDS, 0.0, alpha)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = float(e0.elapsed_time(e1))
        prof = gabp.svm_get_profile(h)
        stt = gabp.svm_get_stats(h)
        kept, total = int(stt["tiles_kept"]), int(stt["tiles_total"])
        nt = (p.n + T_TILE - 1) // T_TILE
        pairs = (kept - nt) * T_TILE * T_TILE + nt * T_TILE * (T_TILE - 1) // 2   # full-tile count, diagonal halves
        bytes_frozen = 28 * pairs
        sweep_ms = prof["sweep_ms"] / max(prof["sweep_launches"], 1)
        dev_bytes = int(stt["device_bytes"])
        gabp.svm_destroy(h)
        # to tolerance
        opts2 = gabp.opts_default(stream=stream.cuda_stream, chunk=8, sparse_tau=st)
        h2 = gabp.svm_create(Xd, yd, p.gamma, p.C, opts2)
        for rep in range(2):
            torch.cuda.synchronize()
            e0.record(stream)
            gabp.svm_refit(h2, Xd, yd, p.gamma, p.C)
            rinf, k = gabp.svm_solve(h2, 400, 1e-6, alpha)
            e1.record(stream)
            torch.cuda.synchronize()
        st2 = gabp.svm_get_stats(h2)
        answers[name] = alpha.cpu().numpy().copy()
        out[name] = {"sweeps_per_s": args.steps * ROUNDS / (ms / 1e3), "tiles_kept": kept, "tiles_total": total,
                     "device_bytes": dev_bytes, "dense_message_state_bytes": 8 * p.n * p.n,
                     "avg_sweep_ms": sweep_ms, "hbm_frac_frozen_bytes": bytes_frozen / (sweep_ms / 1e3) / 1e9 / _peak_gbs(),
                     "to_tolerance": {"ms": float(e0.elapsed_time(e1)), "rounds": int(k), "residual_inf": float(rinf),
                                      "converged": int(st2["converged"]), "err_bound_over_C": st2["err_bound"] / p.C,
                                      "margin": st2["margin"]}}
        gabp.svm_destroy(h2)
    line = {"metric": METRIC, "value": out["tile_sparse"]["sweeps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "n": p.n, "m": 64, "sparse_tau": tau},
            "modes": out}
    if not big:
        line["speedup_sweeps"] = out["tile_sparse"]["sweeps_per_s"] / out["dense"]["sweeps_per_s"]
        line["speedup_to_tolerance"] = out["dense"]["to_tolerance"]["ms"] / out["tile_sparse"]["to_tolerance"]["ms"]
        line["max_alpha_difference_over_C"] = float(np.max(np.abs(answers["dense"] - answers["tile_sparse"]))) / p.C
    print(json.dumps(line), flush=True)
    return 0


# Shapes (n x m) of the data sets the paper times in Section 5 (Tables 2 and 3),
# with the paper's run time in seconds and its hardware: context only (other
# machines, other data).  The bench fills them with the seeded mixture.
PAPER_SHAPES = (
    ("table2_6238x617", 6238, 617, 228.0, "5 x 3.5 GHz Pentium, MPICH2"),
    ("table2_20000x16", 20000, 16, 468.0, "5 x 3.5 GHz Pentium, MPICH2"),
    ("table2_8124x117", 8124, 117, 226.0, "5 x 3.5 GHz Pentium, MPICH2"),
    ("table2_12960x25", 12960, 25, 221.0, "5 x 3.5 GHz Pentium, MPICH2"),
    ("table2_5473x10", 5473, 10, 26.0, "5 x 3.5 GHz Pentium, MPICH2"),
    ("table2_7494x16", 7494, 16, 45.0, "5 x 3.5 GHz Pentium, MPICH2"),
    ("table2_4601x57", 4601, 57, 49.0, "5 x 3.5 GHz Pentium, MPICH2"),
    ("table3_150000x54", 150000, 54, 468.0, "1024 CPUs of an IBM Blue Gene"),
    ("table3_60000x784", 60000, 784, 756.0, "1024 CPUs of an IBM Blue Gene"),
)


def run_paper_shapes(args):
    """Whole solves (formation + rounds to ||r||_inf < 1e-6, at most 200) on
    seeded mixtures with the shapes of the data sets Section 5 times, gamma =
    1/m, C = 1, plain FP32 and BF16 refined, inputs resident on the device,
    CUDA events around each solve (after one warm-up solve).  The paper's run
    times are quoted beside them as context: they were measured on CPU
    clusters, on the real data sets, for the whole training."""
    import torch

    from paper_0810_1648_gb300 import build as gbuild
    from paper_0810_1648_gb300 import gabp
    if not os.path.exists(gabp.LIB_PATH):
        gbuild.build()
    gabp.load()
    stream = torch.cuda.Stream()
    out = {}
    for k, (name, n, m, paper_s, hw) in enumerate(PAPER_SHAPES):
        p = workloads.mixture(n, m, seed=300 + k, gamma=1.0 / m, C=1.0)
        Xd, yd = torch.from_numpy(p.X).cuda(), torch.from_numpy(p.y).cuda()
        alpha = torch.empty(n, dtype=torch.float32, device="cuda")
        res = {"n": n, "m": m, "paper_run_time_s": paper_s, "paper_hardware": hw}
        for form, kw in (("f32", dict(q_mode=0)), ("bf16_refined", dict(q_mode=1, refine=10, msg_bf16=1))):
            h = gabp.svm_create(Xd, yd, p.gamma, p.C, gabp.opts_default(stream=stream.cuda_stream, chunk=8, **kw))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for rep in range(2):
                torch.cuda.synchronize()
                e0.record(stream)
                gabp.svm_refit(h, Xd, yd, p.gamma, p.C)
                rinf, it = gabp.svm_solve(h, 200, 1e-6, alpha)
                e1.record(stream)
                torch.cuda.synchronize()
            st = gabp.svm_get_stats(h)
            res[form] = {"ms": float(e0.elapsed_time(e1)), "rounds": int(it), "residual_inf": float(rinf),
                         "converged": int(st["converged"]), "err_bound_over_C": st["err_bound"] / p.C,
                         "support_vectors": int((alpha > 0).sum().item())}
            gabp.svm_destroy(h)
        out[name] = res
        del Xd, yd, alpha
        torch.cuda.empty_cache()
    line = {"metric": METRIC, "value": None, "unit": "ms per whole solve", "n_gpus": 1, "steps": 1, "warmup": 1,
            "higher_is_better": False, "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "seeded mixtures (3 components per class, sigma 0.7) with the shapes of the data "
                                   "sets of the paper's Tables 2 and 3, gamma = 1/m, C = 1, to ||r||_inf < 1e-6 "
                                   "(at most 200 rounds), formation included"},
            "shapes": out}
    print(json.dumps(line), flush=True)
    return 0


def _serve_run(gabp, rate, duration, q_mode, msg_bf16, stages, max_members):
    """Replays the seeded Poisson stream (rate/s for `duration` s) in real time
    through the continuous-batching server; returns latency percentiles,
    solves/s over the wall time, and the largest stated error bound."""
    reqs = workloads.poisson_requests(rate=rate, duration=duration, seed=7)
    # request data: row/column slices of one seeded mixture pool (labels from it)
    pool = workloads.mixture(50000, 512, seed=7)
    rng = np.random.default_rng(8)
    starts = [int(rng.integers(0, 50000 - r.n + 1)) for r in reqs]
    srv = gabp.Server(iters=200, tol=1e-6, max_members=max_members, q_mode=Q_MODES[q_mode],
                      refine=8 if q_mode != "f32" else 0, msg_bf16=1 if msg_bf16 else 0, chunk=4,
                      stages=stages)
    t0 = time.perf_counter()
    sub, lat, nxt = {}, [], 0
    rounds, passes, conv, errb, resid = [], [], 0, [], []
    done_n = 0
    while done_n < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt].t_arrive <= now:
            r = reqs[nxt]
            X = np.ascontiguousarray(pool.X[starts[nxt]:starts[nxt] + r.n, :r.m])
            y = pool.y[starts[nxt]:starts[nxt] + r.n]
            if abs(float(y.sum())) == r.n:          # need both classes
                y = y.copy(); y[0] = -y[0]
            t = srv.submit(X, y, 1.0 / r.m, r.C)
            sub[t] = (r.t_arrive, r.C)
            nxt += 1
        active, queued, completed = srv.step()
        for t in srv.completed():
            res = srv.poll(t)
            if res is not None:
                t_arr, C = sub.pop(t)
                lat.append(time.perf_counter() - t0 - t_arr)
                rounds.append(res[1]["iters_done"])
                passes.append(res[1]["refine_passes"])
                conv += res[1]["converged"]
                errb.append(res[1]["err_bound"] / C)
                resid.append(res[1]["residual_inf"])
                done_n += 1
        if active == 0 and queued == 0 and nxt < len(reqs):
            time.sleep(max(0.0, min(0.01, reqs[nxt].t_arrive - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    phases = srv.phases()
    srv.close()
    lat = np.array(lat)
    return {"requests": len(reqs), "offered_per_s": rate, "duration_s": duration, "wall_s": wall,
            "solves_per_s": len(reqs) / wall,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
            "converged": int(conv), "max_residual": float(max(resid)),
            "max_err_bound_over_C": float(max(errb)),
            "mean_rounds": float(np.mean(rounds)), "mean_refine_passes": float(np.mean(passes)),
            "server_phases_ms": phases}


def run_serve(args):
    """Poisson stream of SVM-training requests replayed in real time through
    the continuous-batching server; reports p50/p99 latency and solves/s."""
    from paper_0810_1648_gb300 import build as gbuild
    from paper_0810_1648_gb300 import gabp
    if not os.path.exists(gabp.LIB_PATH):
        gbuild.build()
    r = _serve_run(gabp, args.rate, args.duration, args.q_mode, args.msg_bf16, args.stages, args.max_members)
    line = {"metric": METRIC, "value": r["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": 1,
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.q_mode == "f32" else "bf16+f32", "data": "synthetic",
            "config": {"workload": f"serving form: Poisson arrivals rate {args.rate}/s for {args.duration} s, "
                                   "n log-uniform [500,50000], m log-uniform [16,512], C log-uniform [0.1,100], "
                                   "gamma 1/m, tol 1e-6 or 200 rounds, admission by device memory",
                       "requests": r["requests"], "q_mode": args.q_mode, "max_members": args.max_members,
                       "stages": max(args.stages, 1)},
            "latency_s": r["latency_s"], "wall_s": r["wall_s"], "offered_per_s": args.rate,
            "server_phases_ms": r["server_phases_ms"], "mean_rounds": r["mean_rounds"],
            "mean_refine_passes": r["mean_refine_passes"], "converged": r["converged"],
            "max_err_bound_over_C": r["max_err_bound_over_C"]}
    print(json.dumps(line), flush=True)
    return 0


def _extra_batch(gabp, torch, warmup, steps):
    """The batched workload (512 instances, to ||r||_inf < 1e-6 or 200 rounds)
    in plain FP32 and in the BF16 form (BF16 Q + BF16 messages + refinement),
    under the synchronous and the 4-stage schedules: solves/s (median of
    `steps` timed batches, inputs resident on the device), and each form's
    stated error: the largest Varah bound residual / margin over the 512
    results, relative to C."""
    probs = workloads.batch_grid()
    dev = {}
    for p in probs:
        if id(p.X) not in dev:
            dev[id(p.X)] = (torch.from_numpy(p.X).cuda(), torch.from_numpy(p.y).cuda())
    dprobs = [workloads.Problem(*dev[id(p.X)], p.gamma, p.C) for p in probs]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    modes = (("f32", dict(q_mode=0)), ("bf16_refined", dict(q_mode=1, refine=8, msg_bf16=1)),
             ("f32_staged4", dict(q_mode=0, stages=4)),
             ("bf16_refined_staged4", dict(q_mode=1, refine=8, msg_bf16=1, stages=4)))
    out = {}
    for name, kw in modes:
        for _ in range(max(1, warmup)):
            gabp.batch_solve(dprobs, 200, 1e-6, chunk=0, stream=stream.cuda_stream, **kw)
        times, res = [], None
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, res, rc = gabp.batch_solve(dprobs, 200, 1e-6, chunk=0, stream=stream.cuda_stream, **kw)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        out[name] = {"solves_per_s": len(probs) / float(np.median(times)),
                     "ms_per_batch": 1e3 * float(np.median(times)),
                     "converged": int(sum(r["converged"] for r in res)),
                     "max_residual": float(max(r["residual_inf"] for r in res)),
                     "max_err_bound_over_C": float(max(r["err_bound"] / p.C for r, p in zip(res, probs))),
                     "mean_rounds": float(np.mean([r["iters_done"] for r in res]))}
    gabp.batch_release()
    out["instances"] = len(probs)
    out["workload"] = ("512 instances: 32 mixture data sets x C {0.1,1,10,100} x gamma {0.1,0.5,1,2}/m, "
                       "n log-uniform [200,4000], m in {8,32,128,256}, tol 1e-6 or 200 rounds, device inputs")
    out["bf16_over_f32"] = out["bf16_refined"]["solves_per_s"] / out["f32"]["solves_per_s"]
    out["bf16_over_f32_staged4"] = (out["bf16_refined_staged4"]["solves_per_s"]
                                    / out["f32_staged4"]["solves_per_s"])
    out["error_note"] = ("max_err_bound_over_C: max over the instances of ||mu - Q^-1 1||_inf / C bounded by "
                         "Varah: residual / min_i(Q_ii - R_i) of the FP32-Gram matrix, as each result states it")
    return out


def _extra_precision(gabp, torch, peak):
    """The precision workload (n=100000, m=64, gamma=0.5/64, C=1): sweeps/s of
    100 synchronous rounds (one warm-up solve, two timed, CUDA events) and the
    HBM fraction of the pair sweep (every 4th round bracketed) for FP32 Q,
    BF16 Q + BF16 messages and Q recomputed per sweep + BF16 messages; then
    each form to ||r||_inf < 1e-6 (FP32, or refinement on the FP32-Gram
    residual) with its time, rounds and stated error bound."""
    p = workloads.precision_large()
    n = p.n
    pairs = n * (n - 1) // 2
    Xd, yd = torch.from_numpy(p.X).cuda(), torch.from_numpy(p.y).cuda()
    stream = torch.cuda.Stream()
    alpha = torch.empty(n, dtype=torch.float32, device="cuda")
    modes = (("f32", 0, 0), ("bf16", 1, 1), ("recompute", 2, 1))
    out = {}
    for name, qm, mb16 in modes:
        qb = Q_BYTES[name]
        mb = 4 if mb16 else 8
        h = gabp.svm_create(Xd, yd, p.gamma, p.C, gabp.opts_default(stream=stream.cuda_stream, chunk=ROUNDS,
                                                                    q_mode=qm, msg_bf16=mb16))
        gabp.svm_set_profiling(h, PROFILE_STRIDE)
        gabp.svm_solve(h, ROUNDS, 0.0, alpha)
        gabp.svm_get_profile(h, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(2):
            gabp.svm_refit(h, Xd, yd, p.gamma, p.C)
            gabp.svm_solve(h, ROUNDS, 0.0, alpha)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = float(e0.elapsed_time(e1))
        prof = gabp.svm_get_profile(h)
        gabp.svm_destroy(h)
        nz, nf, nl = prof["sweep_launches_zero_state"], prof["sweep_launches_p_frozen"], prof["sweep_launches"]
        alg = pairs * ((4 * mb + qb) * (nl - nz - nf) + (3 * mb + qb) * nf + (2 * mb + qb) * nz)
        achieved = alg / (prof["sweep_ms"] / 1e3) / 1e9 if prof["sweep_ms"] > 0 else None
        entry = {"sweeps_per_s": 2 * ROUNDS / (ms / 1e3),
                 "sweep_hbm": {"achieved_GBps": achieved, "frac_of_measured_peak": achieved / peak if achieved else None,
                               "avg_launch_ms": prof["sweep_ms"] / max(nl, 1), "launches_timed": nl,
                               "bytes_per_pair": {"p_live": 4 * mb + qb, "p_frozen": 3 * mb + qb}}}
        # to tolerance: refinement removes the BF16 error (FP32-Gram residual, FP64 sums)
        opts = gabp.opts_default(stream=stream.cuda_stream, chunk=8, q_mode=qm, msg_bf16=mb16,
                                 refine=10 if qm else 0)
        h = gabp.svm_create(Xd, yd, p.gamma, p.C, opts)
        for _ in range(2):
            torch.cuda.synchronize()
            e0.record(stream)
            gabp.svm_refit(h, Xd, yd, p.gamma, p.C)
            rinf, k = gabp.svm_solve(h, 400, 1e-6, alpha)
            e1.record(stream)
            torch.cuda.synchronize()
        st = gabp.svm_get_stats(h)
        gabp.svm_destroy(h)
        entry["to_tolerance"] = {"ms": float(e0.elapsed_time(e1)), "rounds": int(k), "residual_inf": float(rinf),
                                 "converged": int(st["converged"]), "refine_passes": int(st["refine_passes"]),
                                 "err_bound": float(st["err_bound"]), "err_bound_over_C": float(st["err_bound"] / p.C),
                                 "margin": float(st["margin"])}
        out[name] = entry
    out["workload"] = ("precision form: n=100000, m=64 mixture (seed 2), gamma=0.5/64, C=1; 100 synchronous "
                       "rounds per timed solve; FP32 Q / BF16 Q + BF16 messages / Q recomputed per sweep on the "
                       "tensor cores + BF16 messages")
    out["bf16_over_f32_sweeps"] = out["bf16"]["sweeps_per_s"] / out["f32"]["sweeps_per_s"]
    out["bf16_over_f32_to_tolerance"] = out["f32"]["to_tolerance"]["ms"] / out["bf16"]["to_tolerance"]["ms"]
    return out


def _extra_serve(gabp):
    """The serving form, both forms: the first 3 s of the configured stream
    (200 requests/s: more than one GB300 clears, so solves/s is the
    sustainable rate) and a sub-saturating 15 requests/s for 8 s (latency)."""
    out = {}
    for name, qm, mb16 in (("f32", "f32", False), ("bf16_refined", "bf16", True)):
        out[name] = {"saturating": _serve_run(gabp, 200.0, 3.0, qm, mb16, 4, 64),
                     "sub_saturating": _serve_run(gabp, 15.0, 8.0, qm, mb16, 4, 64)}
        for k in ("saturating", "sub_saturating"):
            out[name][k].pop("server_phases_ms", None)
    out["bf16_over_f32_saturating"] = (out["bf16_refined"]["saturating"]["solves_per_s"]
                                       / out["f32"]["saturating"]["solves_per_s"])
    out["workload"] = ("serving form: Poisson stream (seed 7), n log-uniform [500,50000], m log-uniform [16,512], "
                       "C log-uniform [0.1,100], gamma 1/m, tol 1e-6 or 200 rounds, 4-stage schedule, chunk 4, "
                       "up to 64 members; replayed in real time")
    return out


def run_ours(args):
    import torch

    from paper_0810_1648_gb300 import build as gbuild
    from paper_0810_1648_gb300 import gabp

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(gabp.LIB_PATH):
        gbuild.build()
    gabp.load()

    if args.workload == "precision_large":
        p = workloads.mixture(100000, 64, seed=2 + rank, gamma=0.5 / 64, C=1.0)
        wl = dict(PRECISION_WORKLOAD, q_mode=args.q_mode)
    else:
        p = workloads.mixture(20000, 128, seed=1 + rank, gamma=1.0 / 128, C=10.0)
        wl = dict(WORKLOAD, q_mode=args.q_mode)
    if args.task == "krr":
        # kernel ridge regression on the same features: real targets, ridge 1
        p = workloads.Problem(p.X, workloads.krr_targets(p, 11 + rank), p.gamma, 1.0, name="krr")
        wl = dict(wl, task="krr", workload="kernel ridge regression (Section 1.2) on the same features: targets "
                  "sin(<w, x>) + 0.1 N(0, 1) (w ~ N(0, I/m), seed 11), ridge 1, dominant diagonal; " + wl["workload"])
    qb = Q_BYTES[args.q_mode]
    mb = 4 if args.msg_bf16 else 8     # bytes of one stored message pair
    n = p.n
    stream = torch.cuda.Stream(device=dev)
    Xd = torch.from_numpy(p.X).to(dev)
    yd = torch.from_numpy(p.y).to(dev)
    alpha_d = torch.empty(n, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    opts = gabp.opts_default(stream=stream.cuda_stream, chunk=ROUNDS, q_mode=Q_MODES[args.q_mode],
                             msg_bf16=1 if args.msg_bf16 else 0, task=TASKS[args.task])
    h = gabp.svm_create(Xd, yd, p.gamma, p.C, opts)
    # the pair sweep of every PROFILE_STRIDE-th round is bracketed by events
    # (each bracket costs the captured graph a few microseconds)
    gabp.svm_set_profiling(h, PROFILE_STRIDE)

    def step():
        gabp.svm_refit(h, Xd, yd, p.gamma, p.C)
        gabp.svm_solve(h, ROUNDS, 0.0, alpha_d)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    gabp.svm_get_profile(h, reset=True)
    launches0 = gabp.svm_get_profile(h)["kernel_launches"]
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = gabp.svm_get_profile(h)
    launches = prof["kernel_launches"] - launches0
    st = gabp.svm_get_stats(h)
    value, ms_max = _job_rate(ROUNDS * args.steps, ms, ws, dev)

    # roofline of the dominant kernel (the pair sweep), timed live by events
    pairs = n * (n - 1) // 2
    nz = prof["sweep_launches_zero_state"]
    nf = prof["sweep_launches_p_frozen"]
    nl = prof["sweep_launches"]
    # per pair: round 0 writes P and H (16 B); later rounds read and write
    # both (32 B) until the P messages reach their fixed point, then read P and
    # H and write H (24 B); every round reads the stored Q entry (qb B)
    alg_bytes = pairs * ((4 * mb + qb) * (nl - nz - nf) + (3 * mb + qb) * nf + (2 * mb + qb) * nz)
    sweep_s = prof["sweep_ms"] / 1e3
    achieved = alg_bytes / sweep_s / 1e9 if sweep_s > 0 else None
    peaks = _peaks()
    if peaks and "hbm_gbs" in peaks:
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    traffic = _traffic_from_profile()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic if (args.workload == "plain_large" and args.q_mode == "f32") else None,
            "traffic_note": "ncu dram read+write of one frozen-P launch of this workload "
                            "(profiles/k_sweep_plain_large.txt); null if the kernel source changed since",
            "kernel": {"f32": "k_sweep<float>", "bf16": "k_sweep<bf16>", "recompute": "k_sweep_rc"}[args.q_mode]
                      + " (pair sweep)", "peak_source": peak_src,
            "bytes_per_pair": {"round0": 2 * mb + qb, "p_live": 4 * mb + qb, "p_frozen": 3 * mb + qb},
            "launches_p_frozen": nf,
            "algorithmic_bytes_per_launch": alg_bytes / max(nl, 1),
            "avg_launch_ms": prof["sweep_ms"] / max(nl, 1), "launches_timed": nl,
            "launch_sampling": f"every {PROFILE_STRIDE}th round's sweep bracketed by CUDA events on its stream",
            "share_of_step": (prof["sweep_ms"] / max(nl, 1) * ROUNDS * args.steps / ms) if ms > 0 else None}

    gabp.svm_destroy(h)
    to_tol = None if args.no_to_tol else _to_tolerance(args, Xd, yd, p, stream, gabp, torch)
    e2e = None
    if not args.no_e2e:
        e2e = _e2e(args, p, stream, dev, ws, gabp, torch)
    extras = {}
    if rank == 0 and ws == 1 and not args.no_extras and args.workload == "plain_large" and args.task == "svm":
        # the other forms of the method, measured in the same run (outside the timed region)
        extras["batch"] = _extra_batch(gabp, torch, 1, 3)
        extras["precision"] = _extra_precision(gabp, torch, peak)
        extras["serve"] = _extra_serve(gabp)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        if args.workload != "plain_large":
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                   "sample": "skipped: the FP64 oracle of n=100000 needs 240 GB of host memory"}
        elif args.task != "svm":
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                   "sample": "skipped: the regression task runs the same oracle arithmetic as the default line"}
        else:
            cpu = _cpu_baseline(p, args.cpu_sweeps)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.q_mode == "f32" else "bf16+f32",
                "data": "synthetic", "config": dict(wl, parallelism=f"replicas{ws}"),
                "edge_updates_per_s": value * n * (n - 1),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk, "solve_to_tolerance": to_tol,
                "result": {"residual_inf": st["residual_inf"], "dual_objective": st["dual_objective"],
                           "n_support": st["n_support"]}}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _to_tolerance(args, Xd, yd, p, stream, gabp, torch):
    """Outside the timed region: one whole solve of the same workload to
    ||r||_inf < 1e-6 (formation included; refinement in the precision forms)
    under the synchronous and the 4-stage block Gauss-Seidel schedules, timed
    with CUDA events on the solver's stream after one warm-up solve."""
    out = {}
    refine = 0 if args.q_mode == "f32" else 10
    for name, stages in (("synchronous", 0), ("staged4", 4)):
        opts = gabp.opts_default(stream=stream.cuda_stream, chunk=8, q_mode=Q_MODES[args.q_mode], refine=refine,
                                 msg_bf16=1 if args.msg_bf16 else 0, task=TASKS[args.task], stages=stages)
        h = gabp.svm_create(Xd, yd, p.gamma, p.C, opts)
        alpha = torch.empty(p.n, dtype=torch.float32, device=Xd.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(2):
            torch.cuda.synchronize()
            e0.record(stream)
            gabp.svm_refit(h, Xd, yd, p.gamma, p.C)
            rinf, k = gabp.svm_solve(h, 400, 1e-6, alpha)
            e1.record(stream)
            torch.cuda.synchronize()
        st = gabp.svm_get_stats(h)
        out[name] = {"ms": float(e0.elapsed_time(e1)), "rounds": int(k), "residual_inf": float(rinf),
                     "converged": int(st["converged"]), "refine_passes": int(st["refine_passes"])}
        gabp.svm_destroy(h)
    out["staged_speedup"] = out["synchronous"]["ms"] / out["staged4"]["ms"]
    return out


def _e2e(args, p, stream, dev, ws, gabp, torch):
    """Same solve through the C ABI from pinned host buffers: H2D of X and y and
    D2H of alpha inside the timed region."""
    n = p.n
    Xh = torch.from_numpy(p.X).pin_memory()
    yh = torch.from_numpy(p.y).pin_memory()
    ah = torch.empty(n, dtype=torch.float32).pin_memory()
    opts2 = gabp.opts_default(stream=stream.cuda_stream, chunk=ROUNDS, q_mode=Q_MODES[args.q_mode],
                              task=TASKS[args.task],
                              msg_bf16=1 if args.msg_bf16 else 0)
    h2 = gabp.svm_create(Xh, yh, p.gamma, p.C, opts2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def step_e2e():
        gabp.svm_refit(h2, Xh, yh, p.gamma, p.C)
        gabp.svm_solve(h2, ROUNDS, 0.0, ah)

    for _ in range(max(1, args.warmup)):
        step_e2e()
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step_e2e()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_value, _ = _job_rate(ROUNDS * args.steps, e0.elapsed_time(e1), ws, dev)
    gabp.svm_destroy(h2)
    return {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(p.X.nbytes + p.y.nbytes),
            "d2h_bytes_per_step": int(4 * n)}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sweeps", type=int, default=2)
    ap.add_argument("--ref-sweeps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-to-tol", action="store_true", help="skip the solve-to-tolerance extra measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, precision and serving measurements added to the default line")
    ap.add_argument("--workload", default="plain_large",
                    choices=["plain_large", "precision_large", "batch_grid", "serve", "sparse_large",
                             "paper_shapes"])
    ap.add_argument("--batch-modes", default="",
                    help="batch_grid: comma-separated subset of f32, bf16q_refined, bf16_refined, f32_staged, "
                         "bf16_refined_staged (default all)")
    ap.add_argument("--sparse-n", type=int, default=20000,
                    help="sparse_large: n of the clustered set (20000, or e.g. 200000 beyond dense memory)")
    ap.add_argument("--sparse-comps", type=int, default=3,
                    help="sparse_large beyond 20000: mixture components per class (3; more components keep "
                         "fewer tiles, e.g. 12 at n=500000)")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--max-members", type=int, default=64)
    ap.add_argument("--msg-bf16", action="store_true", help="precision forms: BF16 message storage")
    ap.add_argument("--stages", type=int, default=0,
                    help="message schedule: 0/1 synchronous (default), S > 1 block Gauss-Seidel in S stages "
                         "(serve; the batch workload always adds S-stage modes, S = 4 by default)")
    ap.add_argument("--task", default="svm", choices=list(TASKS),
                    help="svm (default) or krr: kernel ridge regression on the same features and sweep")
    ap.add_argument("--q-mode", default=None, choices=list(Q_MODES))
    ap.add_argument("--profile-small", action="store_true",
                    help="one 8-round solve at n=--profile-n (for ncu captures), no JSON bench line")
    ap.add_argument("--profile-n", type=int, default=6144, help="n of the --profile-small case")
    args = ap.parse_args()
    if args.q_mode is None:
        args.q_mode = "f32" if args.workload == "plain_large" else "bf16"
    if args.profile_small:
        return run_profile_small(args)
    if args.workload == "batch_grid":
        return run_batch(args)
    if args.workload == "sparse_large":
        return run_sparse(args)
    if args.workload == "paper_shapes":
        return run_paper_shapes(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
