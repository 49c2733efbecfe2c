#!/usr/bin/env python
"""Benchmark of the Picasso round hot path on B300.

A step is one whole run of Alg. 1 (pack the strings, then every round: list
assignment, conflict build, coloring, carry) over n = 1,000,000 synthetic
Pauli strings on q = 64 qubits (each qubit non-identity w.p. 0.25, X/Y/Z
equiprobable), P = n/16, alpha = 1.5, inputs resident in HBM.

  value   colored strings/s over the whole job (all ranks)
  e2e     the same through the C ABI's host-buffer entry (picasso_color_host:
          pinned host codes in, host colors out; both copies inside the
          timed region, one call per step)

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
this host's cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT, Q, P_W, NUM, DEN, ALPHA = 1_000_000, 64, 0.25, 1, 16, 1.5
# DRAM bytes (read + write) per algorithmic byte of the bit pass
# (k_bucket_bits: every color bucket's pair tests, its lower blocks of pair
# bits to HBM), from one ncu capture of round 1 of the n = 200,000 case of
# this workload (the bench's launches are too large to capture): 182.0 MB of
# DRAM reads and writes for 194.4 MB of algorithmic bytes.
BITS_DRAM_PER_ALG_BYTE = 0.936
METRIC = "pair tests/s (conflict build) and colored strings/s at n=1M; colors, peak bytes"
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def allmax(x, world, device):
    """Max of x over the ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_per_step):
    """Units all ranks processed per second: every rank colors its own set of
    units_per_rank strings per step (weak scaling), the step time is the max
    over ranks."""
    return world * units_per_rank / (ms_per_step / 1e3)


def workload(n):
    return {"workload": f"picasso n={n} q={Q} p={P_W} P=n/{DEN} alpha={ALPHA}", "n": n, "q": Q,
            "weight_p": P_W, "palette": f"{NUM}/{DEN}", "alpha": ALPHA, "seed": "rank",
            "l2": "working set > L2 (round 1 alone writes 0.53 GB of bit rows and reads and writes ~1 GB of "
                  "bucket members and per-entry words); no explicit flush"}


class Clocks:
    """SM clock, power and clock-event reasons sampled while the timed region
    runs: the driver's NVML library (through ctypes, reads only) every 5 ms
    from a thread, else nvidia-smi every 50 ms."""

    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))

    def __init__(self, index):
        self.index = index
        self.rows = []  # (sm_mhz, max_mhz, power_w, reason bits)
        self.nvml = None
        self.p = None
        self.f = None
        self.stop = None
        self.thread = None

    def _poll(self, lib, h):
        import ctypes

        clk, mx, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))  # 1 = SM clock
        try:
            reasons = lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            reasons = lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0
                    and lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw)) == 0
                    and reasons(h, ctypes.byref(rs)) == 0):
                self.rows.append((float(clk.value), float(mx.value), pw.value / 1000.0, int(rs.value)))
            self.stop.wait(0.005)

    def __enter__(self):
        try:
            import ctypes
            import threading

            lib = ctypes.CDLL("libnvidia-ml.so.1")
            h = ctypes.c_void_p()
            if lib.nvmlInit_v2() != 0 or lib.nvmlDeviceGetHandleByIndex_v2(self.index, ctypes.byref(h)) != 0:
                raise OSError("NVML")
            self.nvml = lib
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, args=(lib, h), daemon=True)
            self.thread.start()
            return self
        except Exception:
            self.nvml = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={SMI_FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=5)
            self.nvml.nvmlShutdown()
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        rows = list(self.rows)
        source = "nvml, 5 ms"
        if self.f is not None:
            source = "nvidia-smi, 50 ms"
            self.f.flush()
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        bits = sum(v for (_, v), x in zip(self.REASONS, parts[5:9]) if x.lower() == "active")
                        pw = float(parts[3]) if parts[3].replace(".", "").isdigit() else None
                        mx = float(parts[2]) if parts[2].replace(".", "").isdigit() else None
                        rows.append((float(parts[1]), mx, pw, bits))
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        mx = [r[1] for r in rows if r[1] is not None]
        pw = [r[2] for r in rows if r[2] is not None]
        reasons = sorted({name for r in rows for name, bit in self.REASONS if r[3] & bit})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": source,
                "power_w_max": max(pw) if pw else None}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# ---------------------------------------------------------------------------- CPU oracle timing
def oracle_sample(n, seed, budget_s, threads=None):
    """Time the oracle's round-1 conflict rows for a sample of vertices.
    Returns (pair tests/s, rows, seconds, threads)."""
    import numpy as np

    import oracle
    from paper_2401_06713_b300 import synth

    threads = threads or oracle.default_threads()
    chars = synth.pauli_weighted(n, Q, P_W, seed=seed)
    P, L = oracle.round_params(n, NUM, DEN, ALPHA)
    enc = oracle.encode3(chars)
    lists = oracle.draw_lists(seed, 1, np.arange(n), P, L, 0)
    rng = np.random.default_rng(seed)
    rows_done, secs = 0, 0.0
    batch = threads
    while secs < budget_s:
        rows = rng.choice(n, batch, replace=False)
        t0 = time.perf_counter()
        oracle.conflict_rows(enc, lists, rows, threads=threads)
        secs += time.perf_counter() - t0
        rows_done += batch
    return rows_done * (n - 1) / secs, rows_done, secs, threads


def oracle_strings_per_s(pairs_per_s, round_sizes, n):
    """Extrapolate the oracle's whole-run rate: round l tests n_l (n_l - 1)
    ordered pairs (the oracle builds each row in full)."""
    work = sum(m * (m - 1) for m in round_sizes)
    return n / (work / pairs_per_s)


# ---------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    from paper_2401_06713_b300 import build as pbuild
    from paper_2401_06713_b300 import picasso, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pbuild.build()
    n = args.n
    chars = synth.pauli_weighted(n, Q, P_W, seed=rank)
    codes_host = torch.from_numpy(chars).pin_memory()
    codes = codes_host.cuda()
    stream = torch.cuda.current_stream()

    def step(codes_dev, out=None):
        xz = picasso.pack(codes_dev)
        with picasso.Picasso(xz, Q, seed=rank, palette=(NUM, DEN), alpha=ALPHA) as p:
            colors, rounds = p.run(out)
            st = p.stats()
        return colors, rounds, st

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(args.warmup):
        colors, rounds, st = step(codes)
    torch.cuda.synchronize()

    # device-resident timed region
    launches0 = picasso.kernel_launches()
    stats = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            colors, rounds, st = step(codes)
            stats.append(st)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        barrier()
    launches = picasso.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()

    # end to end: pinned host codes in, host colors out, every step.  The
    # next step's upload runs on a copy stream while this step computes (as
    # a service streaming sets would run); the first upload starts inside
    # the timed region, every step waits for its own, and the region ends
    # after the last read-back.
    colors_host = torch.empty(n, dtype=torch.int32).pin_memory()
    copy_stream = torch.cuda.Stream()
    bufs = [torch.empty_like(codes) for _ in range(2)]  # uploads alternate between two buffers
    used = [None, None]  # the step that last read each buffer

    def upload(k):
        if used[k % 2] is not None:
            copy_stream.wait_event(used[k % 2])
        with torch.cuda.stream(copy_stream):
            bufs[k % 2].copy_(codes_host, non_blocking=True)
        done = torch.cuda.Event()
        done.record(copy_stream)
        return bufs[k % 2], done

    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_stream.wait_event(e0)
    nxt = upload(0)
    for k in range(args.steps):
        dev_codes, done = nxt
        stream.wait_event(done)
        if k + 1 < args.steps:
            nxt = upload(k + 1)
        c, _, _ = step(dev_codes)
        # the read-back stays on the compute stream: on the copy stream it
        # would hold up the next step's small read-backs on the same engine
        colors_host.copy_(c, non_blocking=True)
        used[k % 2] = torch.cuda.Event()
        used[k % 2].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = e0.elapsed_time(e1)

    # end to end through the C ABI's host-buffer entry: pinned host codes in,
    # pinned host colors out, one picasso_color_host call per step (upload,
    # pack, every round, download; no overlap between steps), timed by the
    # host clock around the synchronous calls
    colors_h2 = torch.empty(n, dtype=torch.int32).pin_memory()
    picasso.color_host(codes_host, Q, colors_h2, seed=rank, palette=(NUM, DEN), alpha=ALPHA)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, r_host = picasso.color_host(codes_host, Q, colors_h2, seed=rank, palette=(NUM, DEN), alpha=ALPHA)
    ms_host = (time.perf_counter() - t0) * 1e3
    barrier()
    ms = allmax(ms, world, "cuda")
    ms_e2e = allmax(ms_e2e, world, "cuda")
    ms_host = allmax(ms_host, world, "cuda")
    colors_np = colors.cpu().numpy()
    assert (colors_np >= 0).all(), "uncolored vertices after a full run"
    st = stats[-1]
    # the library's counters are per context and there is one context per step
    per_step = {k: st[k] for k in ("t_assign_ms", "t_build_ms", "t_color_ms", "t_carry_ms", "t_pairs_ms",
                                   "t_emit_ms", "t_small_ms", "small_rounds", "small_stops")}
    steps_ms = ms / args.steps
    value = whole_job_rate(n, world, steps_ms)
    # the small-round engine's time includes its coloring: counted as build
    # time here, which understates the pair rate
    pair_rate = st["logical_pairs"] / ((st["t_build_ms"] + st["t_small_ms"]) / 1e3)

    peaks, peak_src = measured_peaks()
    sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2032.0)
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    # The dominant kernel is the bit pass of the conflict build: it tests every
    # pair of a color bucket (nibble tables over the symplectic words) and
    # writes G_c as the bucket's lower blocks of pair bits.  It is bound by the
    # pair tests, not by HBM: primary roofline = its pair tests per launch over
    # its event time against one POPC per pair (16 lanes/clk/SM at the clock
    # measured under load).  Secondary: its algorithmic bytes (per list entry
    # 16 B member words and 4 B entry id read, 8 B row address, slot and run
    # length written; 4 B per word of bit rows) against the HBM copy peak.  A
    # run small enough for the small-round engine alone has no per-round
    # build: no figures then.
    launches_b = max(st["pairs_launches"], 1)
    avg_ms = st["t_pairs_ms"] / launches_b
    pairs_launch = st["tested_pairs"] / launches_b
    peak_pairs = n_sm * sm_mhz * 1e6 * 16
    achieved = pairs_launch / (avg_ms / 1e3) if avg_ms > 0 else None
    bytes_launch = st["emit_bytes"] / max(st["emit_launches"], 1)
    roofline = {"bound": "alu", "kernel": "k_bucket_bits (pair tests; G_c as bucket bit blocks)",
                "achieved": achieved / 1e9 if achieved else None, "peak": peak_pairs / 1e9,
                "unit": "Gpair-tests/s", "frac": achieved / peak_pairs if achieved else None,
                "peak_source": f"{n_sm} SMs x {sm_mhz:.0f} MHz (median under load) x 16 POPC/clk/SM",
                "traffic": BITS_DRAM_PER_ALG_BYTE * bytes_launch if (achieved and BITS_DRAM_PER_ALG_BYTE) else None,
                "traffic_note": "DRAM bytes per launch, scaled from an ncu capture of round 1 at n=200000",
                "avg_launch_ms": avg_ms, "tested_pairs_per_launch": pairs_launch,
                "launches_per_step": st["pairs_launches"]}
    gbs = bytes_launch / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else None
    roofline_hbm = {"bound": "hbm", "kernel": "k_bucket_bits", "achieved": gbs,
                    "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                    "frac": gbs / peaks["hbm_gbs"] if gbs and peaks.get("hbm_gbs") else None,
                    "algorithmic_bytes_per_launch": bytes_launch}

    batch = None if args.no_batch else bench_batch(rank)
    learned_form = None if args.no_learned else bench_learned(rank)
    learned_beta = None if args.no_learned else bench_learned_beta(rank)
    chunked = None if args.no_chunked else bench_chunked(rank, codes, colors_np)
    host_csr = None if args.no_host else bench_host(rank, codes, colors_np)
    dynamic = None if args.no_dynamic else bench_dynamic(rank, codes, st)
    wide = None if args.no_wide else bench_wide(rank, n)
    cpu_runs = None if (args.no_cpu_runs or rank != 0) else bench_cpu_runs(rank)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # round sizes of this run (the oracle and GPU agree on them)
        sizes = round_sizes_from(colors_np, st)
        pps, rows, secs, threads = oracle_sample(n, 0, args.cpu_budget)
        cpu = {"value": oracle_strings_per_s(pps, sizes, n), "unit": "strings/s", "cores": threads,
               "kind": "oracle",
               "sample": f"round-1 conflict rows of {rows} random vertices at n={n} ({secs:.1f} s); "
                         f"whole run extrapolated over the rounds' n_l(n_l-1) ordered pairs",
               "pair_tests_per_s": pps}

    line = {
        "metric": METRIC, "value": value, "unit": "strings/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": steps_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64/i32 (bitwise integer)",
        "data": "synthetic (seeded Pauli strings; the paper's molecules are not available)",
        "config": dict(workload(n), parallelism=f"replicas{world}" if world > 1 else "single"),
        "pair_tests_per_s": pair_rate, "colors": int(len(np.unique(colors_np))),
        "colors_sum_P": st["colors_used"], "rounds": rounds,
        "peak_bytes": st["peak_bytes"], "breakdown_ms_per_step": per_step,
        "roofline": roofline, "roofline_hbm": roofline_hbm, "chunked": chunked, "host_csr": host_csr, "dynamic": dynamic, "wide": wide, "cpu_baseline": cpu, "cpu_runs": cpu_runs, "batch": batch, "learned": learned_form, "learned_beta": learned_beta,
        "e2e": {"value": whole_job_rate(n, world, ms_host / args.steps), "unit": "strings/s",
                "h2d_bytes_per_step": n * Q, "d2h_bytes_per_step": 4 * n,
                "how": "one picasso_color_host call per step (C ABI, pinned host buffers: codes in, colors "
                       "out), host clock around the synchronous calls, no overlap between steps"},
        "e2e_overlapped": {"value": whole_job_rate(n, world, ms_e2e / args.steps), "unit": "strings/s",
                           "h2d_bytes_per_step": n * Q, "d2h_bytes_per_step": 4 * n,
                           "how": "device-pointer entry points; each step's upload on a copy stream during the "
                                  "previous step, read-back on the compute stream, CUDA events"},
        "gpu_launches": launches, "clocks": clocks, "wall_s": t_wall,
        "peaks": {"source": peak_src, "hbm_gbs": peaks.get("hbm_gbs")},
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def bench_batch(rank, nsets=256):
    """The batched workload: 256 independent sets (n log-uniform in [1e3,
    5e4], q uniform in {16,24,32,48,64}, weight p uniform in [0.1, 0.5],
    P = n/8, alpha = 2) colored in one batched context, against the same sets
    run one after another through the single-set entry points."""
    import numpy as np
    import torch

    from paper_2401_06713_b300 import picasso, synth

    specs = synth.batch_specs(nsets, seed=rank)
    sets = [synth.pauli_weighted(n, q, p, seed=rank, stream=i + 1) for i, (n, q, p) in enumerate(specs)]
    offs = [0]
    for c in sets:
        offs.append(offs[-1] + len(c))
    pad = np.zeros((offs[-1], 64), dtype=np.uint8)
    for k, c in enumerate(sets):
        pad[offs[k]:offs[k + 1], :c.shape[1]] = c
    xz = picasso.pack(torch.from_numpy(pad).cuda())
    seeds = [rank * 100003 + k for k in range(nsets)]
    parts = [xz[offs[k]:offs[k + 1]].contiguous() for k in range(nsets)]

    def batched(schedule=None):
        with picasso.Picasso(xz, 64, set_offsets=offs, seeds=seeds, schedule=schedule) as p:
            return p.run()[0]

    def sequential():
        out = []
        for k in range(nsets):
            with picasso.Picasso(parts[k], 64, seed=seeds[k]) as p:
                out.append(p.run()[0])
        return out

    for _ in range(3):
        batched()
    sequential()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record()
    cb = batched()
    ev[1].record()
    ev[2].record()
    cs = sequential()
    ev[3].record()
    torch.cuda.synchronize()
    tb, ts = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    same = all(torch.equal(cb[offs[k]:offs[k + 1]], cs[k]) for k in range(nsets))
    # the library's autotuner picks the launch schedule for this batch; then
    # the median of 5 batched runs under it and under the defaults
    t0 = time.perf_counter()
    sched, tuned_med, start_med = picasso.autotune(xz, 64, set_offsets=offs, seeds=seeds, reps=3)
    tune_s = time.perf_counter() - t0

    def med5(schedule):
        ts_ = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c = batched(schedule)
            e1.record()
            torch.cuda.synchronize()
            ts_.append(e0.elapsed_time(e1))
        return sorted(ts_)[2], c

    t_def, _ = med5(None)
    t_tuned, ct = med5(sched)
    same = same and torch.equal(ct, cb)
    return {"workload": f"{nsets} sets, n log-uniform [1e3, 5e4], q in {{16,24,32,48,64}}, p in U[0.1,0.5], "
                        f"P=n/8, alpha=2", "strings": offs[-1], "batched_ms": tb, "sequential_ms": ts,
            "batched_strings_per_s": offs[-1] / (tb / 1e3), "sequential_strings_per_s": offs[-1] / (ts / 1e3),
            "speedup": ts / tb, "identical_colors": same,
            "autotune": {"schedule": sched, "tuning_s": tune_s, "median_ms_default_schedule": t_def,
                         "median_ms_tuned_schedule": t_tuned, "tuner_median_ms_start": start_med,
                         "tuner_median_ms_best": tuned_med}}


def bench_dynamic(rank, codes, st_static):
    """The benchmark workload colored with Alg. 2's dynamic order (parallel
    rule) instead of the static Random order: time, colors and rounds."""
    import torch

    from paper_2401_06713_b300 import picasso

    def run():
        xz = picasso.pack(codes)
        with picasso.Picasso(xz, Q, seed=rank, palette=(NUM, DEN), alpha=ALPHA, color="dynamic") as p:
            _, r = p.run()
            return r, p.stats()

    run()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    r, st = run()
    ev[1].record()
    torch.cuda.synchronize()
    return {"workload": "the benchmark workload, color_algo DYNAMIC (Alg. 2, parallel rule)",
            "ms": ev[0].elapsed_time(ev[1]), "rounds": r, "colors_sum_P": st["colors_used"],
            "static_colors_sum_P": st_static["colors_used"], "peak_bytes": st["peak_bytes"]}


def bench_wide(rank, n, q=128, p_w=0.125):
    """Strings of twice the qubits at the same mean weight (q = 128, weight
    p = 0.125: 16 non-identity positions, as the benchmark workload's q = 64,
    p = 0.25), same palette law: whole-run time, rounds, colors and the wide
    mask pass's pair-test rate."""
    import torch

    from paper_2401_06713_b300 import picasso, synth

    codes = torch.from_numpy(synth.pauli_weighted(n, q, p_w, seed=rank)).cuda()

    def run():
        xz = picasso.pack(codes)
        with picasso.Picasso(xz, q, seed=rank, palette=(NUM, DEN), alpha=ALPHA) as p:
            _, r = p.run()
            return r, p.stats()

    run()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    r, st = run()
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    return {"workload": f"n={n} q={q} p={p_w} P=n/{DEN} alpha={ALPHA} (2 words per part)",
            "ms": ms, "strings_per_s": n / (ms / 1e3), "rounds": r, "colors_sum_P": st["colors_used"],
            "t_build_ms": st["t_build_ms"], "t_color_ms": st["t_color_ms"],
            "pair_tests_per_s": st["tested_pairs"] / (st["t_pairs_ms"] / 1e3) if st["t_pairs_ms"] > 0 else None,
            "peak_bytes": st["peak_bytes"]}


def bench_chunked(rank, codes, ref_colors, budget=2_000_000_000):
    """The benchmark workload under a 2 GB byte budget (its round-1 conflict
    CSR is about 7.1 GB) in chunk mode: rounds over the budget are colored by
    chunks of coloring order.  Same colors as the unchunked run."""
    import numpy as np
    import torch

    from paper_2401_06713_b300 import picasso

    def run():
        xz = picasso.pack(codes)
        with picasso.Picasso(xz, Q, seed=rank, palette=(NUM, DEN), alpha=ALPHA, byte_budget=budget,
                             budget_mode="chunk") as p:
            c, _ = p.run()
            return c, p.stats(), p.set_stats()

    run()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    c, st, (_, peak, _) = run()
    ev[1].record()
    torch.cuda.synchronize()
    return {"workload": f"the benchmark workload, byte budget {budget} bytes, budget_mode chunk",
            "ms": ev[0].elapsed_time(ev[1]), "round_chunks": st["round_chunks"],
            "peak_csr_bytes": peak[0], "budget_bytes": budget, "peak_bytes": st["peak_bytes"],
            "identical_colors": bool(np.array_equal(c.cpu().numpy(), ref_colors))}


def bench_host(rank, codes, ref_colors, budget=2_000_000_000):
    """The benchmark workload under a 2 GB byte budget in host mode (Alg. 3's
    fallback): rounds over the budget keep their columns in mapped pinned host
    memory, written and read in place.  Same colors as the device run."""
    import numpy as np
    import torch

    from paper_2401_06713_b300 import picasso

    def run():
        xz = picasso.pack(codes)
        with picasso.Picasso(xz, Q, seed=rank, palette=(NUM, DEN), alpha=ALPHA, byte_budget=budget,
                             budget_mode="host") as p:
            c, _ = p.run()
            return c, p.stats()

    run()  # the host buffer is pinned once and kept for later contexts
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    c, st = run()
    ev[1].record()
    torch.cuda.synchronize()
    return {"workload": f"the benchmark workload, byte budget {budget} bytes, budget_mode host",
            "ms": ev[0].elapsed_time(ev[1]), "host_csr_rounds": st["host_csr_rounds"],
            "t_build_ms": st["t_build_ms"], "t_color_ms": st["t_color_ms"], "peak_bytes": st["peak_bytes"],
            "identical_colors": bool(np.array_equal(c.cpu().numpy(), ref_colors))}


def bench_learned(rank, count=16):
    """The learned-parameter form on held-out n = 200,000, q = 56 sets, each
    with its own byte budget: the committed regressor's pick (features, MLP
    forward, budget-guarded runs, all library kernels) against the paper's
    normal mode P/n = 1/8, alpha = 2 and the grid's best point."""
    import time

    import numpy as np
    import torch

    from paper_2401_06713_b300 import learned, synth

    reg = learned.Regressor.load()
    specs = synth.learned_specs(count, 90001 + rank, n_lo=200000, n_hi=200000, qs=(56,))
    rows = []
    t_learned = 0.0
    for i, spec in enumerate(specs):
        xz, q, budget = learned.instance(spec)
        seed = 7 * 10 ** 6 + i
        grid = learned.grid_search(xz, q, seed, budget)
        best = learned.best_of(grid)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d, a, c, b, tries = learned.run_learned(reg, xz, q, seed, budget)
        torch.cuda.synchronize()
        t_learned += time.perf_counter() - t0
        dc, db, dok = learned.run_config(xz, q, seed, *learned.DEFAULT, None)
        rows.append((grid[best][2], grid[best][0], c, dc, db <= budget, db / budget, tries))
    fit = [r for r in rows if r[0]]
    near = lambda x, best: x is not None and x <= 1.05 * best
    return {"workload": f"{count} held-out sets, n=200000 q=56 p~U[0.1,0.5], budget n*2^U[9,15] bytes",
            "grid_best_fits": len(fit),
            "learned_fits": sum(1 for r in fit if r[2] is not None),
            "learned_within_5pct_of_best": sum(1 for r in fit if near(r[2], r[1])),
            "learned_mean_colors_over_best": float(np.mean([r[2] / r[1] for r in fit if r[2] is not None]))
            if fit else None,
            "default_fits": sum(1 for r in fit if r[4]),
            "default_within_5pct_of_best": sum(1 for r in fit if r[4] and near(r[3], r[1])),
            "default_mean_colors_over_best": float(np.mean([r[3] / r[1] for r in fit])) if fit else None,
            "default_mean_peak_over_budget": float(np.mean([r[5] for r in rows])),
            "learned_ms_per_set": 1e3 * t_learned / count,
            "learned_mean_attempts": float(np.mean([r[6] for r in rows]))}


def bench_learned_beta(rank, count=4):
    """The beta network (Eq. ml as stated) on fresh held-out n = 200,000,
    q = 56 sets: for each set and each beta in 0.1 .. 0.9, the objective of
    its pick against the grid's best and against the paper's normal mode."""
    import time

    from paper_2401_06713_b300 import learned, synth

    reg = learned.Regressor.load(learned.BETA_WEIGHTS_PATH)
    specs = synth.learned_specs(count, 95001 + rank, n_lo=200000, n_hi=200000, qs=(56,))
    t0 = time.perf_counter()
    rows = learned.evaluate_beta(reg, specs, seed_base=3 * 10 ** 6)
    summary = learned.summarize_beta(rows)
    return {"workload": f"{count} held-out sets x 9 betas, n=200000 q=56 p~U[0.1,0.5]",
            "cases": summary["cases"], "picked_best": summary["learned"]["picked_best"],
            "mean_objective_over_best": summary["learned"]["mean_objective_over_best"],
            "default_mean_objective_over_best": summary["default"]["mean_objective_over_best"],
            "wall_s": time.perf_counter() - t0}


def bench_cpu_runs(rank, threads=None):
    """The oracle against the GPU on whole runs, timed end to end on the same
    inputs: the n = 2,000 uniform workload (q = 20, P = n/8, alpha = 2) and
    the n = 100,000 weighted one (q = 48, p = 0.25, P = n/8, alpha = 2).  The
    oracle runs on all host cores; the GPU time is one whole run (context,
    rounds, colors) with the inputs packed on the device, after a warm-up."""
    import numpy as np
    import torch

    import oracle
    from paper_2401_06713_b300 import picasso, synth

    threads = threads or oracle.default_threads()
    out = []
    for name, chars, num, den, alpha in [
            ("n=2000 q=20 uniform P=n/8 alpha=2", synth.pauli_uniform(2000, 20, seed=0), 1, 8, 2.0),
            ("n=100000 q=48 p=0.25 P=n/8 alpha=2", synth.pauli_weighted(100_000, 48, 0.25, seed=0), 1, 8, 2.0)]:
        n, q = chars.shape
        t0 = time.perf_counter()
        ref, rounds, _ = oracle.run(chars, 0, num, den, alpha, threads=threads)
        cpu_s = time.perf_counter() - t0
        xz = picasso.pack(torch.from_numpy(chars).cuda())

        def once():
            with picasso.Picasso(xz, q, seed=0, palette=(num, den), alpha=alpha) as p:
                return p.run()

        once()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        colors, r = once()
        e1.record()
        torch.cuda.synchronize()
        gpu_ms = e0.elapsed_time(e1)
        out.append({"workload": name, "rounds": rounds, "identical_colors": bool(
            r == rounds and np.array_equal(colors.cpu().numpy(), ref)),
            "oracle_s": cpu_s, "oracle_strings_per_s": n / cpu_s, "cores": threads,
            "gpu_ms": gpu_ms, "gpu_strings_per_s": n / (gpu_ms / 1e3)})
    # Alg. 2 on the benchmark's law at n = 20,000: the oracle's sequential
    # loop and its parallel rule, which the GPU computes exactly; the sums
    # of P show what the parallel reading costs in colors
    chars = synth.pauli_weighted(20_000, Q, P_W, seed=rank)
    sums, secs = {}, {}
    for colorer in ("dynamic", "dynamic_par", "static"):
        t0 = time.perf_counter()
        oc, orounds, ost = oracle.run(chars, rank, NUM, DEN, ALPHA, threads=threads, colorer=colorer)
        secs[colorer] = time.perf_counter() - t0
        sums[colorer] = int(ost[:, 1].sum())
        if colorer == "dynamic_par":
            par = (oc, orounds)
    xz = picasso.pack(torch.from_numpy(chars).cuda())
    with picasso.Picasso(xz, Q, seed=rank, palette=(NUM, DEN), alpha=ALPHA, color="dynamic") as p:
        colors, r = p.run()
        gsum = p.stats()["colors_used"]
    out.append({"workload": f"n=20000 q={Q} p={P_W} P=n/{DEN} alpha={ALPHA}, Alg. 2 dynamic order",
                "oracle_colors_sum_P": {"sequential_alg2": sums["dynamic"], "parallel_rule": sums["dynamic_par"],
                                        "static_random_order": sums["static"]},
                "oracle_s": {"sequential_alg2": secs["dynamic"], "parallel_rule": secs["dynamic_par"],
                             "static_random_order": secs["static"]},
                "gpu_parallel_rule_colors_sum_P": gsum, "cores": threads,
                "identical_colors": bool(r == par[1] and np.array_equal(colors.cpu().numpy(), par[0]))})
    return out


def round_sizes_from(colors, st):
    """n_l of every round, read off the palette ranges: colors of round l lie
    in [base_l, base_l + P_l) and P_l = ceil(n_l * NUM / DEN)."""
    import numpy as np

    n = len(colors)
    sizes = []
    remaining = n
    base = 0
    while remaining > 0:
        P = max(1, -(-remaining * NUM // DEN))
        sizes.append(remaining)
        done = int(((colors >= base) & (colors < base + P)).sum())
        remaining -= done
        base += P
        if done == 0:
            break
    return sizes


# ---------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = args.n
    # round sizes follow from the oracle's own sample law: estimate them with a
    # geometric tail measured on a small oracle run of the same law
    import oracle
    from paper_2401_06713_b300 import synth

    small = 4000
    _, _, st = oracle.run(synth.pauli_weighted(small, Q, P_W, seed=0), 0, NUM, DEN, ALPHA)
    frac = [int(r[0]) / small for r in st]
    sizes = [max(1, int(round(f * n))) for f in frac]
    vals, step_s = [], []
    for _ in range(args.warmup):
        oracle_sample(n, 0, min(args.cpu_budget, 3.0))
    for _ in range(args.steps):
        t0 = time.perf_counter()
        pps, rows, secs, threads = oracle_sample(n, 0, args.cpu_budget / max(args.steps, 1))
        step_s.append(time.perf_counter() - t0)
        vals.append(oracle_strings_per_s(pps, sizes, n))
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "strings/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        # a step is a bounded sample of the run; its measured time
        "ms_per_step": 1e3 * statistics.mean(step_s),
        "extrapolated_ms_per_run": 1e3 * n / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int (CPU oracle)",
        "data": "synthetic", "config": workload(n),
        "cpu_baseline": {"value": value, "unit": "strings/s", "cores": threads, "kind": "oracle",
                         "sample": f"per step: round-1 conflict rows of random vertices at n={n}; whole run "
                                   f"extrapolated with round sizes from an oracle run of the same law at "
                                   f"n={small} (extrapolated_ms_per_run)"},
        "e2e": {"value": value, "unit": "strings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="picasso", choices=["picasso", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-runs", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-chunked", action="store_true")
    ap.add_argument("--no-dynamic", action="store_true")
    ap.add_argument("--no-wide", action="store_true")
    ap.add_argument("--no-host", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
