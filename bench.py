"""Benchmark of the MACGIC-iQUAPI per-step path update on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--precision fp64|c64]

Workload (default): the structured-bath spin-boson model with memory 16 and
the 10-point MACGIC mask, filter 1e-9 (workloads.SPIN_BOSON_STRUCTURED_DK16).
The trajectory is propagated to t = T0 (steady path count), then W untimed
steps, then K timed steps.  One benchmark step = one propagation step
(pre-merge, extension, influence, filter, rho) over the whole stored set.
Between timed steps the L2 cache is flushed (a 512 MB write on the same
stream, outside the timed events).  Metric: extended paths per second =
sum over timed steps of (groups * M^2) / sum of the steps' CUDA-event times.

--impl reference times the FP64 CPU oracle (the deliberately plain
reference) on the same workload, steps and metric on all host cores
(independent replicas in spawned processes).
Multi-GPU (torchrun): independent replicas of the workload, one per rank.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOADS = {
    "spin_boson_structured_dk16": W.SPIN_BOSON_STRUCTURED_DK16,
    "spin_boson_ohmic_dk8": W.SPIN_BOSON_OHMIC_DK8,
    "chain3_structured_dk12": W.CHAIN3_STRUCTURED_DK12,
    "tls_ohmic_full_dk14": W.TLS_OHMIC_FULL_DK14,
    "tls_ohmic_full_dk12": W.tls_ohmic_full(12),
    "tls_ohmic_full_dk13": W.tls_ohmic_full(13),
    "tls_ohmic_full_dk15": W.tls_ohmic_full(15),
    "tls_ohmic_full_dk16": W.tls_ohmic_full(16),
}
METRIC = "extended paths/s"
T0_DEFAULT = 100


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index
        self.on = False

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            if self.on:
                self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for n, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def code_hash(path):
    """sha256 prefix (16 hex digits) of a C++/CUDA source's code: comments
    removed (string and character literals kept whole) and white space
    collapsed, so that DRAM counters, which depend on the code only, stay
    tied to it across edits of its comments."""
    import hashlib
    with open(path, encoding="utf-8") as f:
        src = f.read()
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return hashlib.sha256(" ".join("".join(out).split()).encode()).hexdigest()[:16]


def ncu_traffic(workload, regular, n_in):
    """DRAM bytes per step of the stream kernels from one ncu capture
    (profiles/traffic.txt), or None when none matches the current kernel
    code.  The regular kernel's capture is scaled by stored paths."""
    try:
        sha = code_hash(os.path.join(ROOT, "paper_2506_03127_gb300", "csrc", "qp.cu"))
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    for w, k, src, b, n in rows:
        if src != sha:
            continue
        if regular and k == "stream_regular" and workload.startswith("tls_ohmic_full") and int(n) > 0:
            return float(b) / int(n) * n_in
        if not regular and k == "stream_tile" and w == workload:
            return float(b)
    return None


def algorithmic_bytes(stats_rows, M, amp_bytes, merge, engine="hash"):
    """Per-kernel algorithmic DRAM bytes for a list of steps: stored path =
    8 B key + amp_bytes; merge-table slot 32 B + 8 B key.  The stream engine
    reads the stored set once and writes the survivors (N_in E + N_out E);
    the merge-table kernels read the stored set and the slots they touch."""
    E = 8 + amp_bytes
    ins = tie = exp = 0
    for (t, groups, extended, kept, *_), n_in in stats_rows:
        if engine == "stream":
            exp += n_in * E + kept * E
        elif merge(t):
            ins += n_in * (E + 4) + groups * 32
            tie += n_in * (E + 4) + groups * 16
            exp += groups * (4 + 8 + 32 + 40) + kept * E
        else:
            exp += n_in * E + kept * E
    return np.array([ins, tie, exp, 0.0])


def run_ours(args, rank, world, precision):
    import torch
    from paper_2506_03127_gb300 import Propagator

    w = WORKLOADS[args.workload]
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    amp_bytes = 16 if precision == "fp64" else 8
    p = Propagator.from_workload(w, precision=precision, engine=args.engine, max_paths=args.max_paths)
    p.step(args.t0)
    p.sync()
    # the library's autotuner picks the launch shape (tile size, blocks per
    # SM) on the running propagation; it advances it by a few steps.  A shape
    # given on the command line is used as is (profiling runs pin it: the
    # autotuner's timings are not meaningful under a profiler)
    if getattr(args, "stream_tile", None) or getattr(args, "blocks_per_sm", None):
        kw = {}
        if args.stream_tile:
            kw["stream_tile"] = args.stream_tile
        if args.blocks_per_sm:
            kw["expand_blocks_per_sm"] = args.blocks_per_sm
        p.set_tuning(**kw)
        tuning = p.tuning()
    else:
        p.autotune(trial_steps=8, use_cache=True)
        tuning = p.tuning()   # as applied, with the propagation's engine
    p.sync()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    for _ in range(args.warmup):
        p.step(1)
        with torch.cuda.stream(p.stream):
            flush.zero_()
    p.sync()
    t_first = p.current()[0] + 1
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_id = vis.split(",")[dev] if vis else str(dev)
    clocks = ClockSampler(smi_id)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.on = True
    wall0 = time.perf_counter()
    for k in range(args.steps):
        starts[k].record(p.stream)
        p.step(1)
        ends[k].record(p.stream)
        with torch.cuda.stream(p.stream):
            flush.zero_()
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    if wall1 - wall0 < 1.0:
        time.sleep(1.0 - (wall1 - wall0))
    clocks.on = False
    clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    stats = p.stats(t_first, args.steps)
    prev = p.stats(t_first - 1, args.steps)
    n_in = [r[3] for r in prev]
    extended = float(sum(r[2] for r in stats))
    t_ms = float(step_ms.sum())
    # roofline: per-kernel CUDA-event times over a further run of steps
    nprof = min(args.steps, 200)
    prof_first = p.current()[0] + 1
    kern_ms = p.profile(nprof)
    pstats = p.stats(prof_first, nprof)
    pprev = p.stats(prof_first - 1, nprof)
    t_end = p.current()[0]
    rho_hist = p.rho(1, t_end)
    merge = (lambda t: t >= w.dkmax)
    tun = p.tuning()
    engine = "stream" if tun.engine == 2 else "hash"
    abytes = algorithmic_bytes(list(zip(pstats, [r[3] for r in pprev])), w.M, amp_bytes, merge, engine)
    names = ["premerge_insert", "premerge_tiebreak", "expand_influence_filter_rho", "finalize"]
    peak, peak_src = peaks()
    regular_cfg = engine == "stream" and w.theta == 0.0 and w.M == 2
    if engine == "stream":
        # one step = the regular map kernel (launched where regular steps are
        # possible: M = 2, no filter) and the tile kernel, one of which does
        # the step; both are timed together as the step's kernel
        names = ["stream_regular", "-", "stream_tile", "-"]
        step_ms = kern_ms[0] + kern_ms[2]
        kname = "stream_step (regular map + tile kernel)" if regular_cfg else "stream_step (tile kernel)"
        achieved = abytes[2] / (step_ms / 1e3) / 1e9 if step_ms > 0 else 0.0
    else:
        dom = int(np.argmax(kern_ms))
        kname = names[dom]
        achieved = abytes[dom] / (kern_ms[dom] / 1e3) / 1e9 if kern_ms[dom] > 0 else 0.0
    traffic = None
    if engine == "stream" and precision == "c64":
        tr = ncu_traffic(args.workload, regular_cfg, float(np.mean([r[3] for r in pprev])))
        traffic = None if tr is None else round(tr)
    roof = {"bound": "hbm", "kernel": kname, "engine": engine, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_src,
            "kernel_share": {n: round(float(m / kern_ms.sum()), 4) for n, m in zip(names, kern_ms) if n != "-"},
            "kernel_avg_us": {n: round(float(m / nprof * 1e3), 2) for n, m in zip(names, kern_ms) if n != "-"}}

    # end to end through the public API, from host inputs.  (a) The whole
    # trajectory: eta, mask and rho(0) set from host arrays, then per step
    # qp_step and qp_read_rho_async of rho(t) into pinned host memory
    # (stream-ordered; one qp_sync at the end).  (b) The same steps as the
    # timed region: set-up and the first steps untimed, then the timed steps
    # each with qp_step and the read of rho(t); the stored set, the step's
    # input, stays on the device, so the per-step host->device bytes are 0.
    e2e_steps = args.t0 + args.warmup + args.steps
    from paper_2506_03127_gb300 import eta_from_bath
    eta_h = eta_from_bath(w.bath, w.dt, w.dkmax)
    rho_pinned = torch.empty((e2e_steps, w.M, w.M), dtype=torch.complex128, pin_memory=True)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    p.set_eta(eta_h)
    p.set_mask(w.mask)
    p.set_rho0(w.rho0_array())
    for s in range(e2e_steps):
        p.step(1)
        p.rho_async(s + 1, rho_pinned[s])   # rho(t) to pinned host memory every step
    p.sync()
    e1 = time.perf_counter()
    e_stats = p.stats(1, e2e_steps)
    e2e_traj = float(sum(r[2] for r in e_stats)) / (e1 - e0)
    setup_h2d = eta_h.size * 16 + len(w.mask_list()) * 4 + w.M * w.M * 16
    d2h = w.M * w.M * 16
    # the rows read during the run are the propagation's rho history (the
    # last 4000 steps, which the history ring still holds)
    n_chk = min(e2e_steps, 4000)
    e2e_hist = p.rho(e2e_steps - n_chk + 1, n_chk)
    assert np.array_equal(rho_pinned.numpy()[e2e_steps - n_chk:], e2e_hist), "asynchronous rho reads differ from the history"
    # (b): the timed steps start where the device-timed ones started
    t_start = t_first - 1
    p.set_eta(eta_h)
    p.set_mask(w.mask)
    p.set_rho0(w.rho0_array())
    p.step(t_start)
    p.sync()
    rows = torch.empty((args.steps, w.M, w.M), dtype=torch.complex128, pin_memory=True)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for k in range(args.steps):
        p.step(1)
        p.rho_async(t_start + k + 1, rows[k])
    p.sync()
    e1 = time.perf_counter()
    e2e_same = float(sum(r[2] for r in p.stats(t_start + 1, args.steps))) / (e1 - e0)
    assert np.array_equal(rows.numpy(), p.rho(t_start + 1, args.steps)), "asynchronous rho reads differ from the history"
    p.close()

    res = dict(ext=extended, t_ms=t_ms, wall=wall1 - wall0, e2e=e2e_same, e2e_traj=e2e_traj, roof=roof,
               tuning=tuning.as_dict(), clocks=clocks.summary(), setup_h2d=setup_h2d, d2h=d2h, step_ms=step_ms,
               stats=stats, kernels_per_step=(2 if regular_cfg else 1) if engine == "stream" else 4, rho=rho_hist,
               t_first=t_first)
    return res


def run_batched_sweep(n_inst=64, reps=3):
    """The coupling sweep (n_inst instances of the 8-step model whose path
    counts differ by more than 2x) as one batched context in complex64 on
    the stream engine, autotuned (graph launches per step or one persistent
    launch per call), each trajectory (all steps) one timed qp_step call
    after an L2 flush; the other launch mode and the merge-table engine's
    batch timed the same way; against the plain FP64 path running the
    instances one after another.  Returns the summary object."""
    import torch
    from paper_2506_03127_gb300 import Propagator, abi, batch_from_workloads

    ws = W.coupling_sweep(n_inst)
    w0 = ws[0]
    T = w0.steps
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def trajectory_ms(p):
        times = []
        for _ in range(reps):
            p.set_rho0(w0.rho0_array())
            with torch.cuda.stream(p.stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(p.stream)
            p.step(T)
            e1.record(p.stream)
            p.sync()
            times.append(e0.elapsed_time(e1))
        return float(np.median(times))

    def launch_name(t):
        return "persistent kernel (one launch per call)" if t.mode == abi.QP_LAUNCH_PERSISTENT else \
            "CUDA graphs of %d steps" % t.graph_steps

    p = batch_from_workloads(ws, precision="c64", max_paths=1 << 23, rho_history=max(4096, T + 1))
    engine = "stream" if p.tuning().engine == abi.QP_ENGINE_STREAM else "merge-table"
    p.step(w0.dkmax + 2)
    p.autotune(trial_steps=4, use_cache=False)
    best = p.tuning()   # as applied, with the propagation's engine
    t_b = trajectory_ms(p)
    ext = float(sum(r[2] for r in p.stats(1, T)))
    rho_b = p.rho(0, T + 1)
    counts = p.instance_counts(T)
    # the other launch mode, same tile size
    if best.mode == abi.QP_LAUNCH_PERSISTENT:
        p.set_tuning(mode=abi.QP_LAUNCH_GRAPH, expand_blocks_per_sm=2)
    else:
        p.set_tuning(mode=abi.QP_LAUNCH_PERSISTENT, persistent_blocks=2 * torch.cuda.get_device_properties(0).multi_processor_count)
    other = p.tuning()
    t_other = trajectory_ms(p)
    p.close()
    # the merge-table engine's batch (the same instances)
    h = batch_from_workloads(ws, precision="c64", max_paths=1 << 23, rho_history=max(4096, T + 1), engine="hash")
    h.step(w0.dkmax + 2)
    h.autotune(trial_steps=4, use_cache=False)
    t_h = trajectory_ms(h)
    h.close()
    # plain FP64 path, one instance at a time
    t_s, ext_s, err = 0.0, 0.0, 0.0
    for i, w in enumerate(ws):
        q = Propagator.from_workload(w, precision="fp64", max_paths=1 << 18)
        with torch.cuda.stream(q.stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(q.stream)
        q.step(T)
        e1.record(q.stream)
        q.sync()
        t_s += e0.elapsed_time(e1)
        ext_s += float(sum(r[2] for r in q.stats(1, T)))
        err = max(err, float(np.abs(q.rho(0, T + 1) - rho_b[:, i]).max()))
        q.close()
    return {"workload": f"coupling_sweep{n_inst}", "instances": n_inst, "steps": T, "theta": w0.theta,
            "value": ext / (t_b / 1e3), "unit": "paths/s", "ms_per_trajectory": t_b, "precision": "c64",
            "engine": engine, "launch": launch_name(best) + " (autotuned)", "tuning": best.as_dict(),
            "other_launch": {"launch": launch_name(other), "ms_per_trajectory": t_other},
            "merge_table_batch_ms_per_trajectory": t_h,
            "l2": "flushed before each timed trajectory",
            "kept_per_instance": {"min": int(counts.min()), "max": int(counts.max()),
                                  "max_over_min": float(counts.max() / max(1, counts.min())),
                                  "all": [int(c) for c in counts]},
            "fp64_one_by_one": {"value": ext_s / (t_s / 1e3), "ms_total": t_s},
            "speedup_vs_fp64_one_by_one": (ext / (t_b / 1e3)) / (ext_s / (t_s / 1e3)),
            "rho_max_abs_err_vs_fp64": err}


def run_wide(steps=30, tail=10):
    """The reaction-coordinate model of Sec. 4.3 (M = 8, Delta k_max = 12:
    keys of 96 bits, the qp_wide context) at the paper's converged settings
    (Delta k_eff = 10, theta = 1e-9), complex64 and FP64 over the same first
    `steps` steps (the window fills at t = 12; the set then holds ~3e8
    paths); time per step over the last `tail` steps (CUDA events, one
    qp_wide_step call each), stored and extended paths, and rho of the two
    precisions compared.  The paper's run of this model: ~32 h on 96 cores
    (Sec. 4.3), 2.5e8 paths on average."""
    import torch
    from paper_2506_03127_gb300 import WidePropagator, eta_from_bath

    w = W.reaction_coordinate()
    eta = eta_from_bath(w.bath, w.dt, w.dkmax)
    out = {"workload": w.name, "M": w.M, "dkmax": w.dkmax, "mask": list(w.mask), "theta": w.theta, "dt": w.dt,
           "steps": steps, "key_bits": 8 * w.dkmax}
    rhos = {}
    for prec, mp in (("c64", 1 << 30), ("fp64", 1 << 30)):
        p = WidePropagator(w.M, w.dkmax, w.dt, w.q, w.hs_array(), w.theta, prec, max_paths=mp, max_groups=mp // 4)
        p.set_eta(eta)
        p.set_mask(w.mask)
        p.set_rho0(w.rho0_array())
        ms = []
        for k in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(p.stream)
            p.step(1)
            e1.record(p.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        t, n = p.current()
        st = p.stats(t - tail + 1, tail)
        ext = float(sum(r[2] for r in st))
        t_tail = float(sum(ms[-tail:]))
        rhos[prec] = p.rho(0, t + 1)
        out[prec] = {"ms_per_step": t_tail / tail, "stored_paths_last": int(n),
                     "extended_paths_per_s": ext / (t_tail / 1e3), "workspace_gb": p.nbytes / 1e9,
                     "trace_last": float(np.trace(rhos[prec][-1]).real)}
        p.close()
        del p
        torch.cuda.empty_cache()
    out["rho_max_abs_diff_c64_vs_fp64"] = float(np.abs(rhos["c64"] - rhos["fp64"]).max())
    out["note"] = ("keys beyond 64 bits; parity with the oracle on smaller cases of the same key width "
                   "(tests/test_wide_gpu.py); the paper: ~32 h on 96 cores for the converged run of this model")
    return out


def run_surrogate(T_train=100, T_long=1000, L=32, epochs=2000):
    """The learned surrogate: train (libqp kernels) on 100-step trajectories of
    48 sweep instances, roll 16 held-out instances out to t = 1000 and check
    them against the plain path at checkpoints; times of both."""
    import torch
    from paper_2506_03127_gb300 import batch_from_workloads
    from paper_2506_03127_gb300.surrogate import Surrogate, bath_features, checkpoint_errors, truncated_memory_baselines

    ws = W.resonance_sweep(64)
    p = batch_from_workloads(ws, precision="c64", max_paths=1 << 23)
    p.step(T_train)
    rho = p.rho(0, T_train + 1)
    p.close()
    par = bath_features(ws)
    s = Surrogate(L=L)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = s.fit(rho, par, train=(0, 48), epochs=epochs, lr=2e-3, log_every=epochs - 1)
    t_fit = time.perf_counter() - t0
    q = batch_from_workloads(ws[48:], precision="c64", max_paths=1 << 22)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q.step(T_long - 1)
    q.sync()
    t_plain = time.perf_counter() - t0
    rp = q.rho(0, T_long)
    q.close()
    t0 = time.perf_counter()
    rs = s.rollout(rp[:L].transpose(1, 0, 2, 3), par[48:], T_long)
    t_sur = time.perf_counter() - t0
    errs, raw, fb = checkpoint_errors(rs, rp, (200, 400, 600, 800, 999))
    # the path update's own cheaper settings on the same instances: shorter
    # memory (1 = the Markov map) at the same filter, against the full path
    base = truncated_memory_baselines(ws[48:], T_long, rp, (200, 400, 600, 800, 999))
    err_s = max(raw.values())
    us_s = 1e6 * t_sur / (T_long - L)
    faster = [dk for dk, b in base.items() if b["us_per_step"] <= us_s]
    as_accurate = [dk for dk, b in base.items() if b["err_max"] <= err_s]
    outcome = (f"surrogate {us_s:.1f} us/step at max error {err_s:.3f}; "
               + (f"memory <= {max(faster)} is as fast but its error is >= "
                  f"{min(base[d]['err_max'] for d in faster):.3f}; " if faster else "no shorter memory is as fast; ")
               + (f"memory {min(as_accurate)} is as accurate at {base[min(as_accurate)]['us_per_step']:.1f} us/step"
                  if as_accurate else f"no memory up to {max(base)} is as accurate "
                                      f"(best {min(b['err_max'] for b in base.values()):.3f}); the full memory 8 "
                                      f"takes {1e6 * t_plain / (T_long - 1):.1f} us/step"))
    return {"network": "MLP %d-256-256-8, tanh, BF16 weights/activations, FP32 accumulation" % (8 * L + 2),
            "train": {"instances": 48, "steps": T_train, "windows": 48 * (T_train + 1 - L), "epochs": epochs,
                      "seconds": round(t_fit, 3), "loss_first": hist[0][1], "loss_last": hist[-1][1]},
            "rollout": {"instances": 16, "from_step": L, "to_step": T_long, "seconds": round(t_sur, 4),
                        "us_per_step": round(1e6 * t_sur / (T_long - L), 2)},
            "plain_c64_path": {"seconds": round(t_plain, 4), "us_per_step": round(1e6 * t_plain / (T_long - 1), 2)},
            "speedup_vs_plain": round(t_plain / (t_sur + fb.mean() * t_plain), 2),
            "speedup_note": "fallback instances are charged the plain path's time",
            "rho_max_abs_err_at_checkpoints": {str(k): round(v, 5) for k, v in errs.items()},
            "rho_max_abs_err_raw_surrogate": {str(k): round(v, 5) for k, v in raw.items()},
            "fallback_instances": int(fb.sum()),
            "plain_shorter_memory": {str(dk): {"us_per_step": round(b["us_per_step"], 1), "err_max": round(b["err_max"], 4)}
                                     for dk, b in base.items()},
            "matched_comparison": outcome}


def run_pre_vs_post(t0=100, steps=20, precisions=("fp64", "c64")):
    """The paper's comparison of the pre-merging order (Sec. 3.1) with the
    original post-merging order (Sec. 2.1; Sec. 4.1, Fig. performance), on
    the structured spin-boson model (memory 16) for masks of 4, 6, 10 and
    16 positions and two filter thresholds: per setting the time per step
    (CUDA events, L2 flushed between steps), the paths each order extends,
    its largest set (pre: the stored children; post: the unmerged set) and
    the rho difference between the two orders at the last step."""
    import torch
    from dataclasses import replace
    from paper_2506_03127_gb300 import Propagator
    base = W.SPIN_BOSON_STRUCTURED_DK16
    masks = {4: (0, 1, 2, 3), 6: (0, 1, 2, 3, 4, 8), 10: base.mask, 16: None}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = []
    for prec in precisions:
        for theta in (1e-6, 1e-9):
            for keff, mask in masks.items():
                w = replace(base, mask=mask, theta=theta)
                row = {"precision": prec, "theta": theta, "dk_eff": keff}
                rhos = {}
                for scheme in ("pre", "post"):
                    p = Propagator.from_workload(w, precision=prec, max_paths=1 << 24, scheme=scheme)
                    p.step(t0)
                    p.sync()
                    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                          for _ in range(steps)]
                    t_first = p.current()[0] + 1
                    for a, b in ev:
                        with torch.cuda.stream(p.stream):
                            flush.zero_()
                        a.record(p.stream)
                        p.step(1)
                        b.record(p.stream)
                    p.sync()
                    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
                    st = p.stats(t_first, steps)
                    rhos[scheme] = p.rho(t_first + steps - 1, 1)[0]
                    row[scheme] = {"ms_per_step": round(ms, 4), "paths_extended": int(np.mean([r[1] for r in st])),
                                   "largest_set": int(np.mean([r[4] for r in st])),
                                   "stored": int(np.mean([r[3] for r in st]))}
                    p.close()
                row["pre_over_post_time"] = round(row["pre"]["ms_per_step"] / row["post"]["ms_per_step"], 3)
                row["post_over_pre_largest_set"] = round(row["post"]["largest_set"] / max(1, row["pre"]["largest_set"]), 3)
                row["rho_diff_post_vs_pre"] = float(np.abs(rhos["post"] - rhos["pre"]).max())
                out.append(row)
    return {"workload": base.name + " with masks of 4, 6, 10, 16 positions", "t0": t0, "steps": steps,
            "engines": "pre: stream engine (order-preserving, segmented sums); post: sort engine (radix sort, "
                       "reduce by key)", "rows": out}


def aggregate_over_ranks(t_ms, units):
    """Whole-job figures of independent replicas (one per rank, no data
    exchange): the slowest rank's timed-region time (max over ranks) and the
    units all ranks processed (sum).  Uses the default process group: NCCL
    with CUDA tensors on GPUs, gloo with CPU tensors otherwise."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(t_ms), float(units)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


GOLDEN = {   # oracle trajectories (tests/golden/, written by make_golden.py from oracle/ only)
    "spin_boson_structured_dk16": "spin_boson_structured_dk16_rho200.txt",
    "spin_boson_ohmic_dk8": "spin_boson_ohmic_dk8_rho.txt",
    "chain3_structured_dk12": "chain3_structured_dk12_rho10.txt",
    # the first 10 steps do not depend on the memory length (window filling)
    "tls_ohmic_full_dk13": "tls_ohmic_full_dk14_rho10.txt",
    "tls_ohmic_full_dk14": "tls_ohmic_full_dk14_rho10.txt",
}


def oracle_error(name, rho_hist):
    """max_t max_ab |rho(t) - rho_oracle(t)| over the steps t = 1 .. n the
    stored oracle trajectory covers (rho_hist[k] = rho(k + 1)); (err, n)."""
    fname = GOLDEN.get(name)
    if fname is None:
        return None, 0
    rows = np.loadtxt(os.path.join(ROOT, "tests", "golden", fname), comments="#")
    v = rows[:, 2:]
    rho_o = (v[:, 0::2] + 1j * v[:, 1::2]).reshape(len(rows), rho_hist.shape[-1], rho_hist.shape[-1])
    n = min(len(rows) - 1, len(rho_hist))
    return float(np.abs(rho_hist[:n] - rho_o[1:n + 1]).max()), n


def run_config(name, t0, steps, max_paths, warmup=3, engine="auto", precisions=("c64", "fp64")):
    """Another workload of the benchmark set, measured like the headline
    (autotuned, L2 flushed between timed steps) in each precision on the
    same trajectory; the first precision is the configuration's own, the
    others are compared with it (speed, rho)."""
    a = argparse.Namespace(workload=name, t0=t0, steps=steps, warmup=warmup, max_paths=max_paths, engine=engine,
                           stream_tile=None, blocks_per_sm=None)
    w = WORKLOADS[name]
    runs = {pr: run_ours(a, 0, 1, pr) for pr in precisions}
    out = {"workload": name, "M": w.M, "dkmax": w.dkmax, "mask": w.mask_list(), "theta": w.theta, "t0": t0,
           "steps": steps, "engine": engine, "max_paths": max_paths}
    for pr, r in runs.items():
        e_or, n_or = oracle_error(name, r["rho"])
        out[pr] = {"value": r["ext"] / (r["t_ms"] / 1e3), "unit": "paths/s", "ms_per_step": r["t_ms"] / steps,
                   "paths_kept_last": int(r["stats"][-1][3]), "roofline": r["roof"], "tuning": r["tuning"],
                   "clocks": r["clocks"], "e2e": r["e2e"], "rho_max_abs_err_vs_oracle": e_or, "oracle_steps": n_or}
    if "fp64" in runs and "c64" in runs:
        n = min(len(runs["c64"]["rho"]), len(runs["fp64"]["rho"]))
        out["c64"]["rho_max_abs_err_vs_fp64"] = float(np.abs(runs["c64"]["rho"][:n] - runs["fp64"]["rho"][:n]).max())
        out["c64"]["rho_err_steps"] = n
        out["c64"]["speedup_vs_fp64_gpu"] = out["c64"]["value"] / out["fp64"]["value"]
    out["precision"] = precisions[0]
    return out


def compact(cfg):
    """One configuration in a few numbers (the end of the bench line)."""
    pr = cfg["precision"]
    r = cfg[pr]
    g = lambda x: None if x is None else float(f"{x:.3g}")   # noqa: E731
    d = {"prec": pr, "paths_s": g(r["value"]), "ms_step": g(r["ms_per_step"]), "frac": r["roofline"]["frac"],
         "err_oracle": g(r["rho_max_abs_err_vs_oracle"]), "oracle_t": r["oracle_steps"]}
    other = "fp64" if pr == "c64" else "c64"
    if other in cfg:
        o = cfg[other]
        d[other] = {"paths_s": g(o["value"]), "ms_step": g(o["ms_per_step"]), "frac": o["roofline"]["frac"],
                    "err_oracle": g(o["rho_max_abs_err_vs_oracle"])}
        d["err_c64_vs_fp64"] = g(cfg["c64"].get("rho_max_abs_err_vs_fp64"))
    return d


def _oracle_sample(job):
    """One replica of the oracle on a bounded sample of a workload: the steps
    1 .. t_end, with t_from .. t_end timed.  Returns (extended paths, seconds
    of the timed steps).  Runs in a spawned process."""
    name, t_from, t_end = job
    sys.path.insert(0, ROOT)
    import workloads as W_  # noqa: F401
    from oracle import bath, iquapi
    w = WORKLOADS[name]
    eta = bath.eta_coefficients(w.bath, w.dt, w.dkmax)
    P = iquapi.check_mask(w.mask_list(), w.dkmax)
    Pp = iquapi.premerge_positions(P, w.dkmax)
    U = iquapi.short_time_propagator(w.hs_array(), w.dt)
    q = np.asarray(w.q)
    paths = iquapi.initial_paths(w.rho0_array())
    ext, sec = 0, 0.0
    for t in range(1, t_end + 1):
        a = time.perf_counter()
        paths, rho, st = iquapi.step(paths, t, U, q, eta, w.dkmax, Pp, w.theta, w.M)
        b = time.perf_counter()
        if t >= t_from:
            ext += st.extended
            sec += b - a
    return ext, sec


def oracle_on_host_cores(name, t_from, t_end, procs=None):
    """The oracle as it stands (one thread per process) on every host core:
    independent replicas of the same bounded sample, started together in
    spawned processes; the value is the sum of the replicas' rates.  Also
    one replica alone first (single-core figure).  Returns a dict."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        e1, s1 = pool.apply(_oracle_sample, ((name, t_from, t_end),))
        res = pool.map(_oracle_sample, [(name, t_from, t_end)] * procs)
    ext = sum(r[0] for r in res)
    return {"value": float(sum(e / s for e, s in res)), "unit": "paths/s", "cores": procs, "kind": "oracle",
            "single_core": float(e1 / s1), "seconds_per_replica": float(max(s for _, s in res)),
            "extended_total": int(ext),
            "sample": f"{procs} replicas (one per host core) of oracle steps 1..{t_end} of {name}, "
                      f"steps {t_from}..{t_end} timed; value = sum of the replicas' rates"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="spin_boson_structured_dk16", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="c64", choices=["fp64", "c64"])
    ap.add_argument("--engine", default="auto", choices=["auto", "hash", "stream"])
    ap.add_argument("--t0", type=int, default=T0_DEFAULT)
    ap.add_argument("--max-paths", type=int, default=1 << 21)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-sweep measurement")
    ap.add_argument("--block", default=None, choices=["batched", "surrogate", "pre_vs_post", "wide"],
                    help="run one detail block alone and print its JSON (no contract line)")
    ap.add_argument("--no-more-configs", action="store_true",
                    help="skip the three-level chain and full-memory TLS measurements")
    ap.add_argument("--paper-scale", action="store_true",
                    help="also the full-memory TLS model at memory 15 and 16 (1.1e9 and 4.3e9 stored paths, c64)")
    ap.add_argument("--stream-tile", type=int, default=None, help="pin the stream tile (skips the autotuner)")
    ap.add_argument("--blocks-per-sm", type=int, default=None, help="pin the blocks per SM (skips the autotuner)")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    w = WORKLOADS[args.workload]
    cfg = {"workload": w.name, "M": w.M, "dkmax": w.dkmax, "mask": w.mask_list(), "theta": w.theta,
           "dt": w.dt, "t0": args.t0, "precision": args.precision, "engine": f"{args.engine} (used: in roofline)",
           "amplitudes": "complex64, FP32 influence exponent (Kahan), FP32 error-free (TwoSum) group sums, FP64 eta/rho"
           if args.precision == "c64" else "complex128, FP64 throughout",
           "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas{args.gpus}"}

    if args.impl == "reference":
        if rank != 0:
            return
        # the oracle as it stands, on every host core (independent replicas,
        # spawned processes), over the same steps the GPU arm times
        t_from = args.t0 + args.warmup + 1
        t_end = t_from + args.steps - 1
        cb = oracle_on_host_cores(args.workload, t_from, t_end)
        v = cb["value"]
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "paths/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cb["seconds_per_replica"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": dict(cfg, precision="fp64", engine="oracle",
                                                     amplitudes="complex128, FP64 throughout (the CPU oracle)",
                                                     l2="not applicable (host cores)",
                                                     parallelism=f"{cb['cores']} host processes (replicas)"),
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.block:   # one detail block alone (profiling, quick looks)
        from paper_2506_03127_gb300 import build
        build.build()
        fn = {"batched": run_batched_sweep, "surrogate": run_surrogate, "pre_vs_post": run_pre_vs_post,
              "wide": run_wide}[args.block]
        print(json.dumps({args.block: fn()}))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    from paper_2506_03127_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    # the chosen form (complex64 amplitudes) is the headline; the plain FP64
    # path runs the same trajectory for the comparison at a stated rho error
    res = run_ours(args, rank, world, args.precision)
    ref = run_ours(args, rank, world, "fp64") if args.precision != "fp64" else res
    t_ms, ext = aggregate_over_ranks(res["t_ms"], res["ext"])
    if rank != 0:
        return
    value = ext / (t_ms / 1e3)
    n = min(len(res["rho"]), len(ref["rho"]))
    rho_err = float(np.abs(res["rho"][:n] - ref["rho"][:n]).max())
    fp64_value = ref["ext"] / (ref["t_ms"] / 1e3)
    err_or, n_or = oracle_error(args.workload, res["rho"])
    err_or64, _ = oracle_error(args.workload, ref["rho"])
    head = {"workload": args.workload, "precision": args.precision,
            args.precision: {"value": value, "ms_per_step": t_ms / args.steps, "roofline": res["roof"],
                             "rho_max_abs_err_vs_oracle": err_or, "oracle_steps": n_or}}
    if args.precision != "fp64":
        head["fp64"] = {"value": fp64_value, "ms_per_step": ref["t_ms"] / args.steps, "roofline": ref["roof"],
                        "rho_max_abs_err_vs_oracle": err_or64, "oracle_steps": n_or}
        head["c64"]["rho_max_abs_err_vs_fp64"] = rho_err
    line = {}
    # detail blocks first: the end of the line carries the figures the
    # metric is defined by (each configuration in a few numbers, the
    # comparison with the plain FP64 path, the oracle on the host cores)
    configs = []
    if not args.no_more_configs and world == 1:
        configs = [run_config("spin_boson_ohmic_dk8", 8, min(args.steps, 80), 1 << 20, precisions=("fp64", "c64")),
                   run_config("chain3_structured_dk12", 40, 50, 1 << 26),
                   run_config("tls_ohmic_full_dk13", 13, 10, 1 << 27),
                   run_config("tls_ohmic_full_dk14", 14, 10, 1 << 28, engine="stream")]
        if args.paper_scale:
            configs += [run_config("tls_ohmic_full_dk15", 15, 5, 1 << 30, engine="stream", precisions=("c64",)),
                        run_config("tls_ohmic_full_dk16", 16, 5, 1 << 32, engine="stream", precisions=("c64",))]
        line["more_configs"] = configs
    if not args.no_batched and world == 1:
        line["batched_sweep"] = run_batched_sweep()
        line["surrogate"] = run_surrogate()
        line["pre_vs_post"] = run_pre_vs_post()
        line["wide_keys"] = run_wide()
    line.update({"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": args.gpus, "steps": args.steps,
                 "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                 "scaling": "weak", "vs_baseline": None, "dtype": "c64" if args.precision == "c64" else "f64",
                 "data": "synthetic", "config": cfg, "clocks": res["clocks"], "roofline": res["roof"],
                 "e2e": {"value": res["e2e"], "unit": "paths/s", "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": res["d2h"],
                         "how": "the timed steps again through the public API, rho(t) to pinned host memory every "
                                "step; the stored set (the step's input) stays on the device",
                         "trajectory_value": res["e2e_traj"], "setup_h2d_bytes": res["setup_h2d"]},
                 "gpu_launches": args.steps * res["kernels_per_step"],
                 "s_per_step": t_ms / args.steps / 1e3,
                 "paths_per_step": {"extended_mean": ext / args.steps / max(1, world),
                                    "kept_last": int(res["stats"][-1][3])}})
    line["config"]["tuning"] = res["tuning"]
    g = lambda x: None if x is None else float(f"{x:.3g}")   # noqa: E731
    line["summary"] = {args.workload: compact(head)}
    line["summary"].update({c["workload"]: compact(c) for c in configs})
    line["vs_fp64_gpu"] = {"fp64_value": g(fp64_value), "fp64_ms_per_step": g(ref["t_ms"] / args.steps),
                           "speedup": g(value / fp64_value), "rho_max_abs_err_vs_fp64": g(rho_err),
                           "rho_err_steps": n, "rho_max_abs_err_vs_oracle": g(err_or),
                           "fp64_rho_max_abs_err_vs_oracle": g(err_or64), "oracle_steps": n_or}
    if not args.no_cpu_baseline and world == 1:
        name = args.workload
        line["cpu_baseline"] = oracle_on_host_cores(name, WORKLOADS[name].dkmax + 1, WORKLOADS[name].dkmax + 40)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
