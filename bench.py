"""Benchmark: solved systems/s for very many small nonlinear systems on one GB300.

Workload (default): 2^20 independent instances of the dense cubic family
F(u) = A u + u.*u.*u - b with n = 8, A = 3 I + G (G ~ N(0, 0.3^2)),
b ~ U[-5, 5]^8, u0 = 0, abstol 1e-10, maxiters 50, seed 0.  One step solves
the whole batch four times: Newton with backtracking and trust-region
dogleg, each in FP64 and in mixed precision (FP32 Jacobian and LU, FP64
residual / norm / merit / update).  A system counts as solved when its
status is SUCCESS, i.e. its FP64 residual satisfies ||F||_inf <= 1e-10.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on the
host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# Load every kernel when the context is created: lazy loading on a kernel's
# first launch can stall the other streams of a serving run.
os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2403_16341_gb300 import inputs as I  # noqa: E402

N_SYS = 8
B_FULL = 1 << 20
ABSTOL = 1e-10
MAXITERS = 50
NEWTON, LS, TR = 0, 1, 2
MIXED = 1 << 8
REFINE = 1 << 14  # FP32 LU with classical iterative refinement of each Newton step
VARIANTS = [("newton_backtrack_fp64", LS), ("newton_backtrack_mixed", LS | MIXED),
            ("trust_dogleg_fp64", TR), ("trust_dogleg_mixed", TR | MIXED)]
WORKLOAD = "cubic n=8, 2^20 instances, NR+backtracking and TR-dogleg x {FP64, mixed}"
METRIC = "solved systems/s at ||F||inf<=1e-10 (FP64 vs mixed, 1 GB300)"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # SMs x DFMA/clk x flop/FMA x max clock
FP64_PROBED_TFLOPS = 1.19  # this repository's FP64 FMA-loop probe on a GB300 at 2.07 GHz


def algorithmic_fp64_flops(n: int, alg: int, iters: np.ndarray, nfev: np.ndarray,
                           ngrad: np.ndarray | None = None) -> float:
    """Useful FP64 flops of one solve batch (dual-number and padding overheads
    are implementation cost and not counted).  Per residual evaluation of the
    cubic: 2n^2 + 3n, plus 2n for the squared norm and 2n for forming the
    trial point.  In FP64 mode every pass also factors and solves:
    LU 2n^3/3 - n^2/2 - n/6, triangular solves 2n^2, analytic-equivalent
    Jacobian 2n, and 10n for the dogleg's scalar work (trust region).  The
    trust region forms g = J^T F and J g (2n^2 each) on the passes the kernel
    counts in ngrad (those whose Newton step leaves the region).  Products
    that linearity makes unnecessary are not counted: the line search's slope
    F^T J dN = -||F||^2 and the model's J d (J dN = -F, F.(J g) = g.g).  Mixed
    mode runs the Jacobian, the LU and the model products in FP32, so only
    the residual-side terms are FP64."""
    res = (2 * n * n + 3 * n) + 2 * n + 2 * n
    f = float(nfev.sum()) * res
    if not alg & MIXED:
        per_pass = (2 * n ** 3 / 3 - n * n / 2 - n / 6) + 2 * n * n + 2 * n
        per_pass += 0 if (alg & 0xFF) == LS else 10 * n
        f += float(iters.sum()) * per_pass
        if (alg & 0xFF) == TR and ngrad is not None:
            f += float(ngrad.sum()) * 4 * n * n
    return f


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    def __init__(self, index: int):
        self.index = index
        self.rows: list[list[str]] = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self) -> dict:
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 7 for i in range(4)
                          if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm)}


THREAD_KERNEL_SOURCES = ("nls_dual.cuh", "nls_common.cuh", "nls_thread.cuh",
                         "nls_thread_kernels.cuh", "nls_thread_cubic.cu")


def thread_kernel_hash() -> str:
    h = hashlib.sha256()
    for f in THREAD_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2403_16341_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dram_traffic(variant: str):
    """DRAM bytes per launch of `variant` from the committed ncu summary, or
    None when the kernel sources changed after the counters were taken."""
    path = os.path.join(ROOT, "profiles", "counters_thread_cubic_n8.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) == 3 and parts[0] == variant:
            return int(parts[1]) if parts[2] == thread_kernel_hash() else None
    return None


def reduce_over_ranks(dist, ms: float, solved: int, device):
    """Replicas: the job's time is the slowest rank's, its work the sum of all
    ranks' solved instances (weak scaling, no data exchange)."""
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([solved], device=device, dtype=torch.float64)
    dist.all_reduce(s)
    return float(t.item()), int(s.item())


def shard_seed(rank: int) -> int:
    """Each replica solves its own seeded batch."""
    return rank


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_rate(batch, threads: int, sample: int):
    """FP64 oracle over the first `sample` instances, both algorithms."""
    import oracle as O
    sub = I.Batch(batch.family, batch.n, np.ascontiguousarray(batch.params[:, :sample]),
                  np.ascontiguousarray(batch.u0[:, :sample]))
    solved, t0 = 0, time.perf_counter()
    for oalg in (O.ALG_NEWTON_BACKTRACK, O.ALG_TRUST_DOGLEG):
        _, st, *_ = O.solve_batch(sub.family, sub.params, sub.u0, oalg, ABSTOL, MAXITERS,
                                  threads=threads)
        solved += int((st == 0).sum())
    dt = time.perf_counter() - t0
    return solved / dt, dt, solved


def run_reference(args, world, rank):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    B = min(B_FULL, args.sample)
    batch = I.workload_cubic_n8(B)
    for _ in range(args.warmup):
        oracle_rate(batch, threads, min(B, 4096))
    rates, times = [], []
    for _ in range(args.steps):
        r, dt, _ = oracle_rate(batch, threads, B)
        rates.append(r)
        times.append(dt)
    value = float(np.median(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solved systems/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.median(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_instances": B, "algorithms": ["LS", "TR"]},
            "cpu_baseline": {"value": value, "unit": "solved systems/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"first {B} of the 2^20 instances, NR+backtracking and "
                                       "TR-dogleg in FP64 (the oracle has no mixed mode)"},
            "e2e": {"value": value, "unit": "solved systems/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def extras(args, nls, solver, batch, params, u0, stream, dev):
    """The FP64-Newton comparison bar and the end-to-end (host buffer) leg."""
    import torch
    B = batch.batch
    # the comparison bar: plain FP64 Newton, one static thread per instance
    solver.set_option(nls.NLS_OPT_PERSISTENT, 0)
    ub = torch.empty_like(u0)
    bo = tuple(torch.empty(B, dtype=dt, device=dev) for dt in
               (torch.int32, torch.int32, torch.float64, torch.int32))
    bt = []
    for r in range(4):
        ub.copy_(u0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        req = solver.submit(batch.family, params, ub, NEWTON, ABSTOL, MAXITERS, bo)
        solver.flush()
        e1.record(stream)
        sb = solver.wait(req)
        torch.cuda.synchronize()
        if r:
            bt.append(e0.elapsed_time(e1))
    solver.set_option(nls.NLS_OPT_PERSISTENT, 1)
    baseline = {"kernel": "plain FP64 Newton, one thread per instance, static grid",
                "ms": float(np.median(bt)), "solved_per_s": sb / (float(np.median(bt)) / 1e3)}

    # end to end through the C ABI on pinned host buffers: the step's four
    # solves are made as asynchronous host requests (uploads, solve and
    # downloads of one overlap the neighbours'), then waited for
    hp = torch.from_numpy(batch.params).pin_memory()
    hu0 = torch.from_numpy(batch.u0).pin_memory()
    hus = [torch.empty_like(hu0).pin_memory() for _ in VARIANTS]
    hsts = [torch.empty(B, dtype=torch.int32).pin_memory() for _ in VARIANTS]
    e2e_times, e2e_solved = [], 0
    for r in range(2 + args.steps):
        # the calls overwrite u with the roots: restore the starting points
        # (host bookkeeping of this loop, outside the timed region)
        for hu in hus:
            hu.copy_(hu0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        reqs = [nls.nls_solve_host_async(solver.h, batch.family, hp.data_ptr(), hu.data_ptr(), N_SYS,
                                         B, alg, ABSTOL, MAXITERS, hst.data_ptr())
                for (_, alg), hu, hst in zip(VARIANTS, hus, hsts)]
        ssum = sum(nls.nls_status(solver.h, q) for q in reqs)
        dt = time.perf_counter() - t
        if r >= 2:
            e2e_times.append(dt)
            e2e_solved += ssum
    e2e = {"value": e2e_solved / sum(e2e_times), "unit": "solved systems/s",
           "h2d_bytes_per_step": len(VARIANTS) * (hp.numel() + hu0.numel()) * 8,
           "d2h_bytes_per_step": len(VARIANTS) * (hu0.numel() * 8 + B * 4),
           "api": "nls_solve_host_async x4 per step (one per variant), then nls_status"}

    return baseline, e2e


def run_serving(args, nls, local, alg=LS | MIXED, rate=2000.0, warm_s=1.0, meas_s=10.0,
                pool=512, streams=4) -> dict:
    """Open-loop serving run: Poisson arrivals at `rate` requests/s, each a
    request of the config-3 mix (1-4096 instances, n in {3, 8, 16, 32},
    cubic or Bratu), solved by the continuous-batching server.  Latency runs
    from the scheduled arrival to the results being in host memory.  A whole
    warm-up pass (its own server, other arrival times) runs first and is
    discarded: the first pass of a process pays one-time costs.  streams = 1
    is the serial FIFO mode: one request wave at a time, in arrival order."""
    import torch
    payloads = I.serving_payloads(pool)
    pinned = []
    for b in payloads:
        p = torch.from_numpy(np.ascontiguousarray(b.params)).pin_memory()
        u = torch.zeros(b.u0.shape, dtype=torch.float64).pin_memory()
        st = torch.zeros(b.batch, dtype=torch.int32).pin_memory()
        pinned.append((p, u, st))
    _serve_pass(nls, local, payloads, pinned, alg, rate, 0.0, 2.0, pool, 1, streams)
    return _serve_pass(nls, local, payloads, pinned, alg, rate, warm_s, meas_s, pool, 0, streams)


def _serve_pass(nls, local, payloads, pinned, alg, rate, warm_s, meas_s, pool, seed,
                streams) -> dict:
    """One open-loop pass on a fresh server; requests arriving in the first
    warm_s seconds are not measured."""
    import gc
    count = int(rate * (warm_s + meas_s))
    arrivals = I.poisson_arrivals(count, rate, seed=seed)
    srv = nls.nls_server_create(local, 0, streams)
    tickets = [None] * count
    last_use = {}
    gc.collect()
    gc.disable()  # a collection in the client's submit loop delays arrivals by milliseconds
    try:
        t0 = nls.nls_server_now(srv) + 0.05
        for i in range(count):
            j = i % pool
            if j in last_use:  # the payload's buffers are free again once its last use is done
                prev = last_use.pop(j)
                tickets[prev] = (tickets[prev][0], nls.nls_server_wait_timed(srv, tickets[prev][0]))
            b = payloads[j]
            p, u, st = pinned[j]
            u.zero_()
            target = t0 + arrivals[i]
            while nls.nls_server_now(srv) < target:
                pass
            tk = nls.nls_server_submit(srv, b.family, p.data_ptr() if p.numel() else 0,
                                       u.data_ptr(), b.n, b.batch, alg, ABSTOL, MAXITERS,
                                       st.data_ptr())
            tickets[i] = (tk, None)
            last_use[j] = i
        for i in range(count):
            if tickets[i][1] is None:
                tickets[i] = (tickets[i][0], nls.nls_server_wait_timed(srv, tickets[i][0]))
        stats = nls.nls_server_stats(srv)
    finally:
        gc.enable()
        nls.nls_server_destroy(srv)
    meas = [i for i in range(count) if arrivals[i] >= warm_s]
    tm = [tickets[i][1][1] for i in meas]
    lat = np.array([t["t_done"] - (t0 + arrivals[i]) for t, i in zip(tm, meas)]) * 1e3
    lag = np.array([t["t_submit"] - (t0 + arrivals[i]) for t, i in zip(tm, meas)]) * 1e3
    solved = sum(tickets[i][1][0] for i in meas)
    asked = sum(payloads[i % pool].batch for i in meas)
    span = max(t["t_done"] for t in tm) - (t0 + arrivals[meas[0]])
    # where the time went: arrival -> submit (client), submit -> admit (queue),
    # admit -> launch (copies and solve enqueued), then on the device the
    # wave's input copies, its solve and the copy back; what is left of
    # launch -> done is waiting behind earlier work on the stream plus the
    # dispatcher noticing completion
    stages = {
        "submit_lag": lag,
        "queue": np.array([t["t_admit"] - t["t_submit"] for t in tm]) * 1e3,
        "enqueue": np.array([t["t_launch"] - t["t_admit"] for t in tm]) * 1e3,
        "h2d": np.array([t["h2d_ms"] for t in tm]),
        "solve": np.array([t["solve_ms"] for t in tm]),
        "d2h": np.array([t["d2h_ms"] for t in tm]),
    }
    dev = stages["h2d"] + stages["solve"] + stages["d2h"]
    server = np.array([t["t_done"] - t["t_submit"] for t in tm]) * 1e3  # the server's own part
    stages["stream_wait_and_notice"] = np.array([t["t_done"] - t["t_launch"] for t in tm]) * 1e3 - dev
    worst = int(lat.argmax())
    wreq = payloads[meas[worst] % pool]
    # who the tail is: requests above the p99 latency against all requests,
    # by the bytes their inputs move to the device and the share of their
    # latency spent in the wave's input copies
    in_mb = np.array([(payloads[i % pool].params.size + payloads[i % pool].u0.size) * 8 / 1e6
                      for i in meas])
    p99 = float(np.percentile(lat, 99))
    over = lat > p99
    tail = {"p99_ms": p99, "requests_over_p99": int(over.sum()),
            "input_mb_median_all": float(np.median(in_mb)),
            "input_mb_median_over_p99": float(np.median(in_mb[over])) if over.any() else None,
            "h2d_share_over_p99": float(np.median(stages["h2d"][over] / lat[over])) if over.any() else None,
            "p99_ms_inputs_below_1mb": float(np.percentile(lat[in_mb < 1.0], 99)) if (in_mb < 1.0).any() else None,
            "frac_requests_inputs_below_1mb": float((in_mb < 1.0).mean())}
    breakdown = {k: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)),
                     "max": float(v.max())} for k, v in stages.items()}
    return {"workload": "Poisson arrivals at 2000 req/s, 1-4096 instances per request "
                        "(log-uniform), n in {3,8,16,32}, cubic or Bratu, NR+backtracking mixed",
            "requests": len(meas), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "server_p50_ms": float(np.percentile(server, 50)),
            "server_p99_ms": float(np.percentile(server, 99)), "server_max_ms": float(server.max()),
            "sustained_solved_per_s": solved / span, "offered_instances_per_s": asked / meas_s,
            "solved_fraction": solved / asked, "max_queue": stats["max_queue"],
            "max_inflight": stats["max_inflight"], "streams": streams,
            "max_ms": float(lat.max()), "frac_over_1ms": float((lat > 1.0).mean()),
            "p99_submit_lag_ms": float(np.percentile(lag, 99)),
            "worst_at_s": float(arrivals[meas[worst]]),
            "stages_ms": breakdown, "tail": tail,
            "worst_request": {"latency_ms": float(lat[worst]), "n": wreq.n, "batch": wreq.batch,
                              "family": wreq.family, "wave_requests": tm[worst]["wave_requests"],
                              **{k: float(v[worst]) for k, v in stages.items()}}}


def run_ours(args, world, rank, local):
    import torch
    import paper_2403_16341_gb300 as nls

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    solver = nls.Solver(local, stream)
    if args.no_persistent:
        solver.set_option(nls.NLS_OPT_PERSISTENT, 0)

    # every rank solves its own 2^20 instances (weak scaling, no exchange)
    batch = I.cubic_batch(N_SYS, args.instances, seed=shard_seed(rank), config_id=1, b_half_width=5.0)
    params = torch.from_numpy(batch.params).to(dev)
    u0 = torch.from_numpy(batch.u0).to(dev)
    us = [torch.empty_like(u0) for _ in VARIANTS]
    B = batch.batch
    outs = [tuple(torch.empty(B, dtype=dt, device=dev) for dt in
                  (torch.int32, torch.int32, torch.float64, torch.int32, torch.int32))
            for _ in VARIANTS]
    def new_events():
        return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in VARIANTS]

    def step(events=None):
        reqs = []
        for i, (_, alg) in enumerate(VARIANTS):
            us[i].copy_(u0)
            if events:
                events[i][0].record(stream)
            reqs.append(solver.submit(batch.family, params, us[i], alg, ABSTOL, MAXITERS, outs[i]))
            solver.flush()
            if events:
                events[i][1].record(stream)
        return reqs

    def finish(reqs):
        return [solver.wait(r) for r in reqs]

    # the autotuner picks each variant's tiling and launch mode (untimed)
    chosen = {}
    if not args.no_autotune:
        for i, (name, alg) in enumerate(VARIANTS):
            us[i].copy_(u0)
            solver.autotune(batch.family, params, us[i], alg, ABSTOL, MAXITERS)
            e = nls.nls_tune_lookup(solver.h, batch.family, N_SYS, alg)
            mode = ("one block per 32 instances" if e["refill"] == -2 else
                    f"persistent, refill at {e['refill'] if e['refill'] >= 0 else 24} lanes")
            chosen[name] = {1 << 10: "thread", 1 << 11: "warp", 1 << 12: "cta"}[e["tiles"]] + \
                (f" ({e['lanes']} lanes)" if e["lanes"] else "") + ", " + mode
    for _ in range(max(args.warmup, 3)):
        finish(step())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    l0 = solver.launches()
    per_variant = [[] for _ in VARIANTS]
    solved_total = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        all_reqs, all_events = [], []
        for _ in range(args.steps):
            ev = new_events()
            all_reqs.append(step(ev))
            all_events.append(ev)
        t1.record(stream)
        torch.cuda.synchronize()
        for reqs, ev in zip(all_reqs, all_events):
            solved_total += sum(finish(reqs))
            for i in range(len(VARIANTS)):
                per_variant[i].append(ev[i][0].elapsed_time(ev[i][1]))
    launches = solver.launches() - l0
    ms_total = t0.elapsed_time(t1)
    if dist:
        ms_total, solved_total = reduce_over_ranks(dist, ms_total, solved_total, dev)
    ms_step = ms_total / args.steps
    value = solved_total / (ms_total / 1e3)

    # per-variant numbers and the roofline of the dominant kernel
    variants = {}
    dom, dom_ms = None, -1.0
    for i, (name, alg) in enumerate(VARIANTS):
        st, it, rs, nf, ng = (t.cpu().numpy() for t in outs[i])
        ms = float(np.median(per_variant[i]))
        fl = algorithmic_fp64_flops(N_SYS, alg, it, nf, ng)
        solved = int((st == 0).sum())
        variants[name] = {"ms": ms, "solved_per_s": solved / (ms / 1e3), "solved": solved,
                          "tiling": chosen.get(name, "default"),
                          "mean_iters": float(it.mean()), "max_iters": int(it.max()),
                          "mean_nfev": float(nf.mean()), "mean_gradient_passes": float(ng.mean()),
                          "fp64_gflop": fl / 1e9, "fp64_tflops": fl / (ms / 1e3) / 1e12,
                          "max_resid": float(rs.max())}
        if ms > dom_ms:
            dom, dom_ms = name, ms
    dv = variants[dom]

    baseline, e2e = None, None
    if not args.no_extras:
        baseline, e2e = extras(args, nls, solver, batch, params, u0, stream, dev)

    serving = None
    if not args.no_extras and not args.no_serving:
        serving = run_serving(args, nls, local)

    # the other configurations of the benchmark, each with its own clock record
    configs = None
    if not args.no_extras and not args.no_configs and world == 1:
        configs = {
            "config0_cubic_n3": config0_cubic3(torch, solver, dev, stream, 4000, 3),
            "config2_uneven": config2_uneven(torch, nls, local, dev, stream, 10, 3, modes=True),
            "config4_bratu_large": config4_bratu_large(torch, solver, dev, stream, 5, 3),
        }

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        sample = min(B, args.sample)
        rate, dt, _ = oracle_rate(batch, threads, sample)
        # and on one core, over a smaller sample
        rate1, dt1, _ = oracle_rate(batch, 1, min(sample, 1 << 14))
        cpu = {"value": rate, "unit": "solved systems/s", "cores": threads, "kind": "oracle",
               "sample": f"first {sample} of the 2^20 instances, NR+backtracking and TR-dogleg "
                         f"in FP64 ({dt:.1f} s on {threads} threads)",
               "single_thread_value": rate1,
               "single_thread_sample": f"first {min(sample, 1 << 14)} instances, both "
                                       f"algorithms, 1 thread ({dt1:.1f} s)"}

    traffic = dram_traffic(dom)
    achieved = dv["fp64_tflops"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solved systems/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances_per_gpu": B, "n": N_SYS,
                       "abstol": ABSTOL, "maxiters": MAXITERS,
                       "l2": "inputs larger than L2 (604 MB of parameters per batch)",
                       "parallelism": f"replicas x{world}"},
            "variants": variants, "baseline_fp64_newton": baseline,
            "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s (FP64)",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                         "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                         "peak_probed": FP64_PROBED_TFLOPS,
                         "frac_of_probed": achieved / FP64_PROBED_TFLOPS},
            "serving": serving, "configs": configs,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- other workloads

def _device_batches(torch, batches, dev):
    out = []
    for b in batches:
        p = torch.from_numpy(np.ascontiguousarray(b.params)).to(dev) if b.params.size else None
        u0 = torch.from_numpy(np.ascontiguousarray(b.u0)).to(dev)
        outs = (torch.empty(b.batch, dtype=torch.int32, device=dev),
                torch.empty(b.batch, dtype=torch.int32, device=dev),
                torch.empty(b.batch, dtype=torch.float64, device=dev),
                torch.empty(b.batch, dtype=torch.int32, device=dev))
        out.append((b, p, u0, torch.empty_like(u0), outs))
    return out


def time_flush(torch, solver, dbs, alg, steps, warmup, stream):
    """Solve every batch of `dbs` in one flush, `steps` times after `warmup`;
    `alg` is one algorithm word or one per batch.  Returns (median ms per
    flush, solved per flush, launches per flush)."""
    algs = list(alg) if isinstance(alg, (list, tuple)) else [alg] * len(dbs)
    times, solved, l0 = [], 0, None
    for r in range(warmup + steps):
        for _, _, u0, u, _ in dbs:
            u.copy_(u0)
        if r == warmup:
            l0 = solver.launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reqs = [solver.submit(b.family, p, u, a, ABSTOL, MAXITERS, outs)
                for (b, p, _, u, outs), a in zip(dbs, algs)]
        solver.flush()
        e1.record(stream)
        sv = sum(solver.wait(q) for q in reqs)
        torch.cuda.synchronize()
        if r >= warmup:
            times.append(e0.elapsed_time(e1))
            solved = sv
    return float(np.median(times)), solved, (solver.launches() - l0) // steps


def sampled_error(dbs, alg, per_batch=4, seed=0):
    """Max relative error of the GPU roots against the polished FP64 oracle
    on a sample of instances of every batch."""
    import oracle as O
    rng = np.random.default_rng(seed)
    worst = 0.0
    oalg = {0: O.ALG_NEWTON, 1: O.ALG_NEWTON_BACKTRACK, 2: O.ALG_TRUST_DOGLEG}[alg & 0xFF]
    for b, _, _, u, _ in dbs:
        idx = np.sort(rng.choice(b.batch, min(per_batch, b.batch), replace=False))
        ug = u.cpu().numpy()[:, idx]
        P = b.params[:, idx]
        ou, st, *_ = O.solve_batch(b.family, P, b.u0[:, idx], oalg, ABSTOL, MAXITERS)
        ref = O.polish_batch(b.family, P, ou)
        err = np.abs(ug - ref).max(axis=0) / np.maximum(1.0, np.abs(ref).max(axis=0))
        worst = max(worst, float(err.max()))
    return worst


TILE_NAMES = {1 << 10: "thread", 1 << 11: "warp", 1 << 12: "cta"}


def config0_cubic3(torch, solver, dev, stream, steps, warmup):
    """1,024 cubic n = 3 instances, plain FP64 Newton: one graph launch per
    batch (launch-latency bound), analytic and dual-number Jacobians."""
    dbs = _device_batches(torch, [I.workload_cubic_n3()], dev)
    res = {"config": "cubic n=3, 1024 instances, plain FP64 Newton, abstol 1e-10, maxiters 50"}
    with ClockSampler(dev.index or 0) as clk:
        for name, alg in (("analytic_jacobian", NEWTON | (1 << 9)), ("dual_jacobian", NEWTON)):
            ms, sv, nl = time_flush(torch, solver, dbs, alg, steps, max(warmup, 3), stream)
            res[name] = {"ms_per_batch": ms, "us_per_solve": 1e3 * ms / 1024,
                         "solved_per_s": sv / (ms / 1e3), "solved": sv, "launches": nl}
    res["clocks"] = clk.summary()
    for name, alg in (("analytic_jacobian", NEWTON | (1 << 9)), ("dual_jacobian", NEWTON)):
        time_flush(torch, solver, dbs, alg, 1, 0, stream)
        res[name]["max_rel_err"] = sampled_error(dbs, alg, 64)
    return res


def config2_uneven(torch, nls, local, dev, stream, steps, warmup, modes=True):
    """2^18 instances, n log-uniform in 2..32, half cubic and half Bratu,
    NR + backtracking: every (family, n) bucket in one graph flush, in FP64,
    in mixed precision, and both precisions in the same flush (each bucket
    twice); tilings autotuned per bucket and precision.  With `modes`, also
    the serial launch modes for comparison."""
    batches = I.workload_uneven()
    dbs = _device_batches(torch, batches, dev)
    dbs_m = _device_batches(torch, batches, dev)  # second set of buffers for the joint flush
    res = {"config": ("2^18 instances, n log-uniform in 2..32, half cubic half Bratu, "
                      f"NR+backtracking, {len(batches)} (family, n) buckets per precision")}
    solver = nls.Solver(local, stream)
    chosen = {}
    with ClockSampler(local) as clk:
        for prec, m in (("fp64", 0), ("mixed", MIXED)):
            alg = LS | m
            if modes:
                for mode, persistent, graph in (("direct_serial", 1, 0), ("static_serial", 0, 0)):
                    solver.set_option(nls.NLS_OPT_PERSISTENT, persistent)
                    solver.set_option(nls.NLS_OPT_GRAPH, graph)
                    ms, sv, nl = time_flush(torch, solver, dbs, alg, steps, max(warmup, 3), stream)
                    res[f"{prec}_{mode}"] = {"ms": ms, "solved_per_s": sv / (ms / 1e3),
                                             "solved": sv, "launches": nl}
                solver.set_option(nls.NLS_OPT_PERSISTENT, 1)
                solver.set_option(nls.NLS_OPT_GRAPH, 1)
                ms, sv, nl = time_flush(torch, solver, dbs, alg, steps, max(warmup, 3), stream)
                res[f"{prec}_graph_default_tiling"] = {"ms": ms, "solved_per_s": sv / (ms / 1e3),
                                                       "solved": sv, "launches": nl}
            for b, p, u0, u, _ in dbs:
                u.copy_(u0)
                chosen[f"{prec}:{b.family}:{b.n}"] = TILE_NAMES[solver.autotune(b.family, p, u, alg)]
            ms, sv, nl = time_flush(torch, solver, dbs, alg, steps, max(warmup, 3), stream)
            res[f"{prec}_graph_autotuned"] = {"ms": ms, "solved_per_s": sv / (ms / 1e3),
                                              "solved": sv, "launches": nl}
        # both precisions in one flush (the tuning table holds both)
        algs = [LS] * len(dbs) + [LS | MIXED] * len(dbs_m)
        ms, sv, nl = time_flush(torch, solver, dbs + dbs_m, algs, steps, max(warmup, 3), stream)
        res["fp64_and_mixed_one_flush"] = {"ms": ms, "solved_per_s": sv / (ms / 1e3), "solved": sv,
                                           "launches": nl, "instances": 2 * (1 << 18)}
    res["clocks"] = clk.summary()
    res["max_rel_err_fp64"] = sampled_error(dbs, LS, 2)
    res["max_rel_err_mixed"] = sampled_error(dbs_m, LS | MIXED, 2)
    res["tiles"] = chosen
    solver.close()
    return res


def lu_pass_flops(n: int, solves: int = 1) -> float:
    """Flops of one dense LU with partial pivoting (2n^3/3 - n^2/2 - n/6)
    plus `solves` pairs of triangular solves (2n^2 each)."""
    return 2 * n ** 3 / 3 - n ** 2 / 2 - n / 6 + solves * 2 * n ** 2


def config4_bratu_large(torch, solver, dev, stream, steps, warmup):
    """16,384 Bratu instances, n uniform in 64..128, trust-region dogleg, one
    CTA per instance: the FP32 LU with FP64 residual (Newton's own correction
    of the FP32 steps), the same with classical iterative refinement of every
    Newton step (two passes of r = -F - J dN in FP64), and the FP64 LU."""
    dbs = _device_batches(torch, I.workload_bratu_large(), dev)
    res = {"config": ("16,384 Bratu instances, n uniform in 64..128, lambda ~ U[0.5, 3], "
                      "trust-region dogleg, one CTA per instance")}
    with ClockSampler(dev.index or 0) as clk:
        for name, alg in (("fp32_lu_fp64_residual", TR | MIXED), ("fp32_lu_refined", TR | MIXED | REFINE),
                          ("fp64_lu", TR)):
            ms, sv, nl = time_flush(torch, solver, dbs, alg, steps, max(warmup, 3), stream)
            passes = sum(int(outs[1].sum().item()) for *_, outs in dbs) / sum(b.batch for b, *_ in dbs)
            # algorithmic flops of the factorisations and triangular solves of the
            # passes, in the LU's precision (a refined pass adds two more solves)
            nsolve = 3 if alg & REFINE else 1
            gf = sum(float(outs[1].sum().item()) * lu_pass_flops(b.n, nsolve) for b, *_, outs in dbs) / 1e9
            res[name] = {"ms": ms, "solved_per_s": sv / (ms / 1e3), "solved": sv, "launches": nl,
                         "mean_passes": passes, "lu_gflop": gf, "lu_tflops": gf / ms,
                         "lu_precision": "fp32" if alg & MIXED else "fp64"}
            res[name]["max_rel_err"] = sampled_error(dbs, alg, 1)
    res["clocks"] = clk.summary()
    return res


def run_workload(args, local):
    import torch
    import paper_2403_16341_gb300 as nls
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    solver = nls.Solver(local, stream)
    line = {"workload": args.workload, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "data": "synthetic", "unit": "solved systems/s", "results": {}}
    res = line["results"]
    if args.workload == "cubic3":
        line["results"] = config0_cubic3(torch, solver, dev, stream, args.steps, args.warmup)
    elif args.workload == "uneven":
        line["results"] = config2_uneven(torch, nls, local, dev, stream, args.steps, args.warmup)
    elif args.workload == "serving":
        line["config"] = "open-loop Poisson arrivals, config-3 request mix"
        # continuous batching on four worker streams, and the serial FIFO mode
        # (one stream: one request wave at a time) for comparison
        for name, alg, streams in (("mixed", LS | MIXED, 4), ("fp64", LS, 4),
                                   ("mixed_serial_fifo", LS | MIXED, 1),
                                   ("fp64_serial_fifo", LS, 1)):
            res[name] = run_serving(args, nls, local, alg=alg, streams=streams)
    elif args.workload == "adjoint":
        # sensitivities dL/dtheta of solved roots for random cotangents w, one
        # case per tiling: 2^20 cubic n = 8 (thread), 2^16 cubic n = 32 (warp
        # segment), 8192 Bratu n = 128 (CTA)
        cases = (("cubic8_thread", I.workload_cubic_n8()),
                 ("cubic32_warp", I.cubic_batch(32, 1 << 16, config_id=2)),
                 ("bratu128_cta", I.bratu_batch(128, 8192, config_id=2)))
        line["config"] = ("adjoint sensitivities (FP64): 2^20 cubic n=8 roots (thread), 2^16 cubic "
                          "n=32 (warp), 8192 Bratu n=128 (CTA)")
        for name, b in cases:
            dbs = _device_batches(torch, [b], dev)
            _, p, u0, u, outs = dbs[0]
            u.copy_(u0)
            solver.wait(solver.submit(b.family, p, u, LS | MIXED, ABSTOL, MAXITERS, outs))
            w = torch.randn_like(u0)
            grad = torch.empty_like(p)
            st = torch.empty(b.batch, dtype=torch.int32, device=dev)
            times = []
            for r in range(max(args.warmup, 3) + args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                nls.nls_adjoint(solver.h, b.family, p.data_ptr(), u.data_ptr(), b.n, b.batch,
                                w.data_ptr(), grad.data_ptr(), st.data_ptr())
                e1.record(stream)
                torch.cuda.synchronize()
                if r >= max(args.warmup, 3):
                    times.append(e0.elapsed_time(e1))
            ms = float(np.median(times))
            # params read, gradient written, root and cotangent read, status written
            bytes_moved = b.batch * 8 * (b.params.shape[0] * 2 + 2 * b.n) + b.batch * 4
            res[name] = {"ms": ms, "instances_per_s": b.batch / (ms / 1e3),
                         "hbm_gbs": bytes_moved / (ms / 1e3) / 1e9,
                         "singular": int((st != 0).sum().item())}
    elif args.workload == "poly":
        # (1) Rosenbrock n = 8 from the Sec. 3.3 starts, every third moved to
        # the Fig. 1 start where plain Newton fails; (2) 2^14 cubic n = 40,
        # where the poly-algorithm opens with its quasi-Newton phase
        b = I.rosenbrock_batch(8, 1 << 18, seed=0)
        b.u0[0, ::3] = -1.2
        b.u0[1:, ::3] = 1.0
        b40 = I.cubic_batch(40, 1 << 14, config_id=2)
        line["config"] = ("2^18 generalized Rosenbrock n=8, u0 ~ U[0,1)^8 with every third "
                          "at (-1.2, 1, ..., 1), maxiters 300; 2^14 cubic n=40 (b ~ U[-2,2]^40), "
                          "maxiters 50")
        for prefix, bb, mi in (("", b, 300), ("n40_", b40, MAXITERS)):
            dbs = _device_batches(torch, [bb], dev)
            for name, alg in (("newton", NEWTON), ("poly", 3), ("poly_mixed", 3 | MIXED)):
                times, solved, iters = [], 0, 0.0
                for r in range(max(args.warmup, 3) + args.steps):
                    _, p, u0, u, outs = dbs[0]
                    u.copy_(u0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    q = solver.submit(bb.family, p, u, alg, ABSTOL, mi, outs)
                    solver.flush()
                    e1.record(stream)
                    sv = solver.wait(q)
                    torch.cuda.synchronize()
                    if r >= max(args.warmup, 3):
                        times.append(e0.elapsed_time(e1))
                        solved = sv
                        iters = float(outs[3][:bb.batch].float().mean().item())
                ms = float(np.median(times))
                res[prefix + name] = {"ms": ms, "solved": solved, "solved_fraction": solved / bb.batch,
                                      "solved_per_s": solved / (ms / 1e3), "mean_nfev": iters}
    elif args.workload == "next4":
        # the higher-order, multi-step and quasi-Newton solvers next to Newton
        # with backtracking: the 2^20 cubic n = 8 workload (one thread per
        # instance), 2^16 cubic n = 32 (one warp per instance) and 2^14 cubic
        # n = 64 (one CTA per instance)
        keep = set(args.variants.split(",")) if args.variants else None
        cases = (("", I.workload_cubic_n8(args.instances)),
                 ("n32_", I.cubic_batch(32, 1 << 16, config_id=2)),
                 ("n64_", I.cubic_batch(64, 1 << 14, config_id=2)))
        line["config"] = (f"{cases[0][1].batch} cubic n=8 (b ~ U[-5,5]^8), 2^16 cubic n=32 and 2^14 "
                          "cubic n=64 (b ~ U[-2,2]^n), u0 = 0; Halley (Eq. 3), Potra-Ptak (Eq. 4), "
                          "Broyden / modified Broyden (Tab. 1); thread, warp and CTA tiling, "
                          "autotuned launch")
        for prefix, b in cases:
            dbs = _device_batches(torch, [b], dev)
            _, p, u0, u, outs = dbs[0]
            for name, alg in (("newton_backtrack", LS), ("halley", 5), ("potra_ptak", 4),
                              ("mod_broyden", 7), ("broyden", 6)):
                for prec, m in (("fp64", 0), ("mixed", MIXED)):
                    key = f"{prefix}{name}_{prec}"
                    if keep is not None and key not in keep:
                        continue
                    u.copy_(u0)
                    if not args.no_autotune:
                        solver.autotune(b.family, p, u, alg | m, ABSTOL, MAXITERS)
                    ms, sv, nl = time_flush(torch, solver, dbs, alg | m, args.steps,
                                            max(args.warmup, 3), stream)
                    it = outs[1][:b.batch].float()
                    res[key] = {"ms": ms, "solved": sv, "solved_per_s": sv / (ms / 1e3),
                                "mean_iters": float(it.mean().item()), "launches": nl}
    elif args.workload == "tr-schemes":
        # trust-region radius updates: the Simple reading and NocedalWright
        # (Tab. 3), on the cubic n = 8 workload and on Rosenbrock n = 8 from
        # the Sec. 3.3 starts
        nw = 1 << 13
        cases = (("cubic8", I.workload_cubic_n8(args.instances), MAXITERS),
                 ("rosenbrock8", I.rosenbrock_batch(8, 1 << 18, seed=0), 300))
        line["config"] = (f"trust-region dogleg, Simple vs NocedalWright radius update: "
                          f"{cases[0][1].batch} cubic n=8 (b ~ U[-5,5]^8, u0 = 0) and 2^18 "
                          "generalized Rosenbrock n=8 (u0 ~ U[0,1)^8, maxiters 300)")
        for cname, b, mi in cases:
            dbs = _device_batches(torch, [b], dev)
            _, p, u0, u, outs = dbs[0]
            for sname, flag in (("simple", 0), ("nocedal_wright", nw)):
                for prec, m in (("fp64", 0), ("mixed", MIXED)):
                    alg = TR | flag | m
                    times, solved = [], 0
                    for r in range(max(args.warmup, 3) + args.steps):
                        u.copy_(u0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        q = solver.submit(b.family, p, u, alg, ABSTOL, mi, outs)
                        solver.flush()
                        e1.record(stream)
                        sv = solver.wait(q)
                        torch.cuda.synchronize()
                        if r >= max(args.warmup, 3):
                            times.append(e0.elapsed_time(e1))
                            solved = sv
                    ms = float(np.median(times))
                    res[f"{cname}_{sname}_{prec}"] = {
                        "ms": ms, "solved": solved, "solved_per_s": solved / (ms / 1e3),
                        "mean_iters": float(outs[1][:b.batch].float().mean().item())}
    elif args.workload == "bratu-large":
        line["results"] = config4_bratu_large(torch, solver, dev, stream, args.steps, args.warmup)
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    if "config" not in line:
        line["config"] = line["results"].pop("config")
    solver.close()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sample", type=int, default=1 << 20,
                    help="instances the CPU oracle solves per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", default="",
                    help="comma-separated subset of the step's variants, or of the next4 "
                         "workload's lines (profiling runs)")
    ap.add_argument("--instances", type=int, default=B_FULL,
                    help="batch size (profiling runs; the benchmark uses 2^20)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default tiling instead of the autotuner's choice")
    ap.add_argument("--no-persistent", action="store_true",
                    help="one-block-per-chunk grids instead of persistent ones (comparison runs)")
    ap.add_argument("--workload", default="cubic8",
                    choices=["cubic8", "cubic3", "uneven", "bratu-large", "serving", "adjoint",
                             "poly", "next4", "tr-schemes"],
                    help="cubic8: the benchmark step; the others print their own JSON line")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the cubic n=3, uneven and Bratu n=64..128 configurations")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-Newton bar, the end-to-end leg and the CPU baseline")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.variants and args.workload == "cubic8":
        keep = set(args.variants.split(","))
        unknown = keep - {v for v, _ in VARIANTS}
        if unknown:
            ap.error(f"unknown variants {sorted(unknown)}")
        VARIANTS[:] = [v for v in VARIANTS if v[0] in keep]
    if args.no_extras:
        args.no_cpu_baseline = True
    if args.workload != "cubic8":
        run_workload(args, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
