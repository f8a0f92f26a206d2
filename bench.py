"""Benchmark: particles/s through the detector response on one B300.

A step is one pass of the whole response (propagation, efficiencies,
smearing, towers, energy flow, isolation, counts) over one batch of synthetic
events already resident in HBM: a single fused persistent launch.  The default
workload is the batched CMS-like configuration (100k events, Poisson(400) + 4
hard objects, ~40.4M particles).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload batched|ee|pileup|tiny]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

Under torchrun (N > 1) every rank runs an independent replica of the workload
on its own GPU (events are independent; no data-path collective) and the
slowest rank's time counts; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s through detector response at 1 B300 (% HBM roofline) vs per-event; p99 latency"
WORKLOAD_DESC = {
    "batched": "batched CMS-like: 100k events x (Poisson(400) + 4 hard objects), one ragged CSR launch",
    "ee": "e+e- ALEPH-like: 1M events x Poisson(35), sum E = 91.2 GeV",
    "pileup": "pileup CMS-like: 10k events x (Poisson(400) + 170 x Poisson(30)), vertex z spread",
    "tiny": "tiny CMS-like: 100 events x Poisson(50)",
}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            backend = os.environ.get("PDR_DIST_BACKEND", "nccl")
            dist.init_process_group(backend)
        return dist, dist.get_rank(), ws
    return None, 0, 1


def max_over_ranks(dist, x: float) -> float:
    """The slowest rank's value (all-reduce MAX); x itself on one process.
    The tensor lives where the process group's backend wants it."""
    if not dist:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_event_base(rank: int, n_events: int) -> int:
    """First event index of a rank's replica: ranks draw disjoint event indices
    (every random draw is keyed by the event index), so no two ranks repeat
    the same events."""
    return rank * n_events


def job_rate(units_per_rank: int, ws: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: units all ranks processed / the slowest rank's time."""
    return ws * units_per_rank * steps / (max_ms / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

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
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
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
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = {"fused_kernel": ("pdr_kernel.cu", "pdr_math.cuh", "pdr_ip.cuh", "pdr_ff.cuh", "pdr_internal.h"),
                  "pu_fill_kernel": ("pdr_pileup.cu", "pdr_math.cuh"),
                  "postprocess_kernel": ("pdr_postprocess.cu", "pdr_math.cuh"),
                  "track_ip_kernel": ("pdr_ip.cu", "pdr_math.cuh", "pdr_ip.cuh")}


def kernel_fingerprint(kernel: str = "fused_kernel") -> str:
    """sha1 of a kernel's source files without comments and whitespace (comment edits keep it)."""
    src = "".join(open(os.path.join(ROOT, "paper_2606_26089_b300", "csrc", f)).read()
                  for f in KERNEL_SOURCES[kernel])
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", "", src)
    return hashlib.sha1(src.encode()).hexdigest()[:12]


def _traffic_from_profile(workload: str, kernel: str = "fused_kernel"):
    """Per-launch DRAM bytes from the committed ncu summary, if it matches the kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    sha = kernel_fingerprint(kernel)
    m_sha = re.search(r"kernel_source_sha1:\s*([0-9a-f]+)", text)
    m_t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_t or m_sha.group(1) != sha:
        return None
    return float(m_t.group(1))


def bench_ours(args, dist, rank, ws):
    import torch

    from paper_2606_26089_b300 import binding as B
    from paper_2606_26089_b300 import build as pdr_build
    from paper_2606_26089_b300 import synth

    pdr_build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    batch = synth.make(args.workload, args.events)
    card_name = synth.card_for(args.workload)
    n_ev, n_p = batch.n_events, batch.n_particles
    ctx = B.Context(local, pool_bytes=int(args.pool_gb * (1 << 30)))
    cid = ctx.card_load(card_name)
    dev = B.batch_to_device(batch)
    out = B.alloc_outputs(n_ev, n_p)
    ob = B.make_outputs(out)
    base = replica_event_base(rank, n_ev)
    bt = B.make_batch(dev, cid, args.seed, event_base=base)
    if args.launch:
        best = B.pdr_launch()
        f = [int(x) for x in args.launch.split(",")]
        best.team, best.block = f[0], f[1]
        best.table_slots, best.grid = (f[2] if len(f) > 2 else 0), 0
    else:
        best = ctx.autotune(bt, ob)
    stream = torch.cuda.current_stream()

    # ---- device-resident throughput: K fused launches, per-launch CUDA events
    for _ in range(args.warmup):
        ctx.run(bt, ob, launch=best)
    torch.cuda.synchronize()
    ctx.check()
    counts = out["counts"].cpu().numpy().view(np.uint32)[:n_ev].astype(np.int64)
    tot = counts.sum(axis=0)
    in_bytes = batch.nbytes_input()
    out_bytes = 16 * tot[0] + 12 * tot[1] + 12 * tot[2] + (16 + 8) * tot[3] + 16 * n_ev
    alg_bytes = int(in_bytes + out_bytes)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    for k in range(args.steps):
        starts[k].record(stream)
        ctx.run(bt, ob, launch=best)
        stops[k].record(stream)
    t_all1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ctx.check()
    total_ms = t_all0.elapsed_time(t_all1)
    launch_ms = [a.elapsed_time(b) for a, b in zip(starts, stops)]
    total_ms = max_over_ranks(dist, total_ms)
    ms_per_step = total_ms / args.steps
    value = job_rate(n_p, ws, args.steps, total_ms)
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    achieved = alg_bytes / avg_launch_s / 1e9
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    traffic = _traffic_from_profile(args.workload)

    # ---- end to end through the host-buffer call: H2D inputs, run, D2H results
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        h_in = {k: (None if getattr(batch, k) is None else pin(getattr(batch, k)))
                for k in ("offsets", "pt", "eta", "phi", "mass", "pdg", "charge", "vz")}
        hb = B.pdr_batch()
        hb.n_events = n_ev
        for k, v in h_in.items():
            setattr(hb, k, None if v is None else v.ctypes.data)
        hb.seed, hb.event_index_base, hb.card_id, hb.max_event_size, hb.flags = args.seed, base, cid, 0, 0
        hb.max_event_size = int(batch.multiplicities().max())
        h_out = {k: torch.empty(shape, dtype=dt).pin_memory().numpy() for k, shape, dt in (
            ("tracks", (n_p, 4), torch.float32), ("towers", (n_p, 3), torch.float32),
            ("eflow", (n_p, 3), torch.float32), ("cands", (n_p, 4), torch.float32),
            ("iso", (n_p, 2), torch.float32), ("counts", (n_ev, 4), torch.int32))}
        ho = B.pdr_outputs()
        for k, v in h_out.items():
            setattr(ho, k, v.ctypes.data)
        for _ in range(max(1, min(args.warmup, 2))):
            ctx.run_host(hb, ho, launch=best)
        if dist:
            dist.barrier()
        times = []
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.run_host(hb, ho, launch=best)
            times.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(dist, statistics.mean(times))
        c2 = h_out["counts"].view(np.uint32).astype(np.int64).sum(axis=0)
        d2h = int(16 * c2[0] + 12 * c2[1] + 12 * c2[2] + (16 + 8) * c2[3] + 16 * n_ev)
        e2e = {"value": ws * n_p / e2e_s, "unit": "particles/s", "h2d_bytes_per_step": int(in_bytes),
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3}

    # ---- the plain per-event form (one launch per event) on a prefix
    per_event = None
    if not args.no_per_event and n_ev > 0:
        npre = min(args.per_event_events, n_ev)
        pre = batch.slice_events(0, npre)
        pdev = B.batch_to_device(pre)
        pout = B.alloc_outputs(npre, pre.n_particles)
        pb = B.make_batch(pdev, cid, args.seed, event_base=base)
        ctx.run_per_event(pb, B.make_outputs(pout))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run_per_event(pb, B.make_outputs(pout))
        e1.record(stream)
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        per_event = {"value": pre.n_particles / s, "unit": "particles/s", "events": npre,
                     "events_per_s": npre / s, "speedup_batched_over_per_event": (n_p / avg_launch_s) / (pre.n_particles / s)}

    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "events_per_s": job_rate(n_ev, ws, args.steps, total_ms),
        "config": {"workload": WORKLOAD_DESC[args.workload], "card": card_name, "n_events": n_ev,
                   "n_particles": n_p, "seed": args.seed, "launch": best.as_dict(),
                   "l2": f"inputs {in_bytes / 1e6:.0f} MB per step > 126 MB L2; no flush",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.4 TB/s",
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_launch_s * 1e3,
                     "kernel": "pdr::fused_kernel"},
        "e2e": e2e,
        "per_event_form": per_event,
        "clocks": clk,
        "gpu_launches": args.steps,
    }
    # the steps around the response, each timed in its own region (one GPU)
    if not args.no_track_ip and ws == 1:
        line["track_ip"] = bench_track_ip(args, B, ctx, bt, ob, n_ev, n_p, counts, launch=best,
                                          response_ms=avg_launch_s * 1e3)
    if not args.no_jets and ws == 1:
        line["jets"] = bench_jets(args, B, ctx, bt, ob, n_ev, n_p, counts)
    if not args.no_postprocess and ws == 1:
        line["postprocess"] = bench_postprocess(args, B, ctx, bt, ob, out, n_ev, counts)
    if not args.no_serving and ws == 1:
        line["serving"] = bench_serving(args, B, ctx)
    if not args.no_pileup_merge and ws == 1:
        line["pileup_merge"] = bench_pileup_merge(args, B, ctx)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch, card_name, args.seed, args.cpu_seconds)
        line["cpu_baseline"]["parity_sample"] = parity_sample(ctx, cid, batch, card_name, args.seed, base)
    ctx.close()
    return line


def bench_serving(args, B, ctx):
    """Continuous-batching serving loop vs one plain launch per request, on the
    same Poisson arrival schedules (at most --serving-max-requests a rate, so
    the highest rates saturate both forms).  Latency to device: submit ->
    results in device memory (the library's clock); to host: submit -> the
    request's counts and records (slot layout) copied back to pinned host
    memory, on a stream of the caller's."""
    import ctypes
    import threading as th

    import torch

    from paper_2606_26089_b300 import synth

    pools = synth.serving_pools(args.serving_pool)
    cards = {n: ctx.card_load(n) for n in synth.SERVING_CARDS}
    pinned = {}
    for g, pb in pools.items():
        pinned[g] = {k: (None if getattr(pb, k) is None else
                         torch.from_numpy(np.ascontiguousarray(getattr(pb, k))).pin_memory())
                     for k in ("pt", "eta", "phi", "mass", "pdg", "charge", "vz")}
    cudart = ctypes.CDLL("libcudart.so.13")
    cudart.cudaMemcpyAsync.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                       ctypes.c_void_p]
    d2h_stream = torch.cuda.Stream()
    REC = (("counts", 16, True), ("tracks", 16, False), ("towers", 12, False), ("eflow", 12, False),
           ("cands", 16, False), ("iso", 8, False))

    def host_batch(r):
        pb = pools[r.generator]
        off = (pb.offsets[r.start:r.start + r.n_events + 1] - pb.offsets[r.start]).astype(np.int64)
        o = torch.from_numpy(off).pin_memory()
        a0 = int(pb.offsets[r.start])
        hb = B.pdr_batch()
        hb.n_events = r.n_events
        hb.offsets = o.data_ptr()
        for k, t in pinned[r.generator].items():
            setattr(hb, k, None if t is None else t.data_ptr() + a0 * t.element_size())
        hb.seed, hb.event_index_base, hb.card_id, hb.flags = r.seed, 0, cards[r.card], 0
        hb.max_event_size = int(np.diff(off).max()) if r.n_events else 0
        return hb, o, a0, int(off[-1])

    def d2h(ptrs, n_ev, n_p, host):
        """Counts and every record array of one request (device pointers) into `host`."""
        off = 0
        for (name, size, per_event), p in zip(REC, ptrs):
            nb = size * (n_ev if per_event else n_p)
            if nb:
                rc = cudart.cudaMemcpyAsync(host.data_ptr() + off, p, nb, 2, d2h_stream.cuda_stream)
                if rc:
                    raise RuntimeError(f"cudaMemcpyAsync failed ({rc})")
            off += nb
        d2h_stream.synchronize()

    out = {"workload": "Poisson arrivals; requests of log-uniform(1, 5000) events from the batched, "
                       "e+e- and pile-up generators, card uniform among CMS-like, ATLAS-like, e+e-",
           "duration_s": args.serving_seconds, "max_requests_per_rate": args.serving_max_requests, "rates": {}}
    for rate in args.serving_rates:
        sched = synth.serving_schedule(rate, args.serving_seconds, args.serving_pool)[:args.serving_max_requests]
        if not sched:
            continue
        reqs = [host_batch(r) for r in sched]
        parts = sum(x[3] for x in reqs)
        max_b = max(16 * r.n_events + 64 * x[3] for r, x in zip(sched, reqs))
        host = torch.empty(max_b, dtype=torch.uint8).pin_memory()
        # ---- served: submit at arrival times; a helper thread waits for each
        # ticket, copies its results to the host and releases it
        ctx.serve_start()
        tickets, t_sub = [], []
        lat_host = []
        done = th.Event()
        failed = []
        t_last = [0.0]

        def releaser():
            # a failed request is released too (its pool memory would otherwise
            # block admission and the server would never drain)
            i = 0
            while not (done.is_set() and i >= len(tickets)):
                if i < len(tickets):
                    rc = ctx.wait(tickets[i], 120_000)
                    if rc != 0:
                        failed.append((i, rc))
                    else:
                        r = ctx.fetch(tickets[i])
                        d2h([r.counts, r.tracks, r.towers, r.eflow, r.cands, r.iso], r.n_events, r.n_particles,
                            host)
                        now = time.perf_counter()
                        lat_host.append((now - t_sub[i]) * 1e3)
                        t_last[0] = now
                    try:
                        ctx.release(tickets[i])
                    except B.PdrError:
                        failed.append((i, "release"))
                    i += 1
                else:
                    time.sleep(0.0002)

        rt = th.Thread(target=releaser)
        rt.start()
        t0 = time.perf_counter()
        for r, (hb, o, a0, np_) in zip(sched, reqs):
            while time.perf_counter() - t0 < r.t_arrival:
                time.sleep(0.0001)
            t_sub.append(time.perf_counter())
            tickets.append(ctx.serve_submit(hb))
        done.set()
        rt.join()
        st = ctx.serve_stats()
        ctx.serve_stop()
        if failed:
            raise RuntimeError(f"{len(failed)} serving requests failed (first: {failed[0]})")
        served_span = t_last[0] - (t0 + sched[0].t_arrival)
        # ---- baseline: one request at a time, one plain launch each (H2D, run,
        # sync), then the same copies back
        lat_dev, lat_h = [], []
        t0 = time.perf_counter()
        s = torch.cuda.current_stream()
        for r, (hb, o, a0, np_) in zip(sched, reqs):
            while time.perf_counter() - t0 < r.t_arrival:
                time.sleep(0.0001)
            dev = {"offsets": o.to("cuda", non_blocking=True)}
            for k, t in pinned[r.generator].items():
                dev[k] = None if t is None else t[a0:a0 + np_].to("cuda", non_blocking=True)
            dev["n_events"], dev["max_event_size"] = r.n_events, hb.max_event_size
            outb = B.alloc_outputs(r.n_events, np_)
            ctx.run(B.make_batch(dev, cards[r.card], r.seed), B.make_outputs(outb))
            s.synchronize()
            lat_dev.append((time.perf_counter() - t0 - r.t_arrival) * 1e3)
            d2h([outb[k].data_ptr() for k, _, _ in REC], r.n_events, np_, host)
            lat_h.append((time.perf_counter() - t0 - r.t_arrival) * 1e3)
        span = time.perf_counter() - t0 - sched[0].t_arrival
        lat_dev = np.array(lat_dev)
        lat_h = np.array(lat_h)
        lh = np.array(lat_host) if lat_host else np.zeros(1)
        served_ps = parts / served_span if served_span > 0 else None
        per_req_ps = parts / span if span > 0 else None
        out["rates"][str(rate)] = {
            "requests": len(sched), "particles": parts, "offered_s": sched[-1].t_arrival,
            "waves": st["waves"], "requests_per_wave": len(sched) / max(st["waves"], 1),
            "admission_waits": st["admission_waits"],
            "served": {"p50_ms_device": st["p50_ms"], "p99_ms_device": st["p99_ms"],
                       "p50_ms_host": float(np.percentile(lh, 50)), "p99_ms_host": float(np.percentile(lh, 99)),
                       "particles_per_s_device": st["particles_done"] / st["span_s"] if st["span_s"] > 0 else None,
                       "particles_per_s_host": served_ps},
            "per_request": {"p50_ms_device": float(np.percentile(lat_dev, 50)),
                            "p99_ms_device": float(np.percentile(lat_dev, 99)),
                            "p50_ms_host": float(np.percentile(lat_h, 50)), "p99_ms_host": float(np.percentile(lat_h, 99)),
                            "particles_per_s_host": per_req_ps},
            "served_over_per_request_throughput": (served_ps / per_req_ps) if served_ps and per_req_ps else None}
    return out


def bench_jets(args, B, ctx, bt, ob, n_ev, n_p, counts):
    """Anti-kT jets (R = 0.5, pT > 10 GeV, >= 2 constituents: the paper's
    PFlowJetsAntiKt05 pipeline) of the response's PFlow objects."""
    import torch

    stream = torch.cuda.current_stream()
    jets = torch.empty((n_p, 8), dtype=torch.float32, device="cuda")
    jc = torch.empty((n_ev,), dtype=torch.int32, device="cuda")
    prm = B.make_jet_params("pflow", "antikt", 0.5, 10.0, 2)
    reps = max(2, args.steps // 5)
    ctx.cluster_jets(bt, ob, prm, jets, jc)
    torch.cuda.synchronize()
    ctx.check()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.cluster_jets(bt, ob, prm, jets, jc)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    ctx.check()
    sec = statistics.mean(times)
    n_obj = int(counts[:, 0].sum() + counts[:, 2].sum())
    n_jets = int(jc.sum().item())
    return {"algorithm": "anti-kT R = 0.5, pT >= 10 GeV, >= 2 constituents", "events": n_ev, "objects": n_obj,
            "jets": n_jets, "ms": sec * 1e3, "events_per_s": n_ev / sec, "objects_per_s": n_obj / sec,
            "bound": "latency (a serial chain of clustering steps per event and warp; no DRAM or arithmetic roofline)",
            "reps": reps}


def bench_track_ip(args, B, ctx, bt, ob, n_ev, n_p, counts, launch=None, response_ms=None):
    """Track impact parameters (d0, z0 and their errors) of every track of the
    response's outputs, vertices on the axis (the workload has none off it)."""
    import torch

    stream = torch.cuda.current_stream()
    ip = torch.empty((n_p, 4), dtype=torch.float32, device="cuda")
    prm = B.make_ip_params()
    reps = max(3, args.steps)
    for _ in range(3):
        ctx.track_ip(bt, ob, prm, ip)
    torch.cuda.synchronize()
    ctx.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.track_ip(bt, ob, prm, ip)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    sec = e0.elapsed_time(e1) / 1e3 / reps
    nt = int(counts[:, 0].sum())
    # algorithmic bytes: offsets and track count (12 B an event); per track its
    # particle index (4 B), the particle's pT, eta, phi and charge (13 B) and
    # the record written (16 B)
    alg = 12 * n_ev + 33 * nt
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    achieved = alg / sec / 1e9
    # the fused form: the response writes each track's record beside the track
    # (pdr_run_ip); its cost is its launch time minus the plain response's
    for _ in range(3):
        ctx.run_ip(bt, ob, prm, ip, launch=launch)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        ctx.run_ip(bt, ob, prm, ip, launch=launch)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    fused = e0.elapsed_time(e1) / reps
    fused_out = {"ms_response_with_ip": fused, "ms_response": response_ms,
                 "ms_added": (fused - response_ms) if response_ms is not None else None,
                 "algorithmic_bytes_added": int(16 * nt),
                 "note": "the generated particles are read once, by the response"}
    return {"tracks": nt, "ms": sec * 1e3, "tracks_per_s": nt / sec,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": _traffic_from_profile("batched", "track_ip_kernel"),
                         "algorithmic_bytes_per_launch": int(alg), "kernel": "pdr::track_ip_kernel"},
            "fused": fused_out, "reps": reps}


def bench_postprocess(args, B, ctx, bt, ob, out, n_ev, counts):
    """Filter pipeline + event features (Sec. 2.4) on the response's outputs:
    PFlow objects with pT > 1 GeV and |eta| < 2.5, H_T and missing E_T of the
    survivors; timed without compaction (the outputs stay as they are), then
    once with the survivors moved down in place."""
    import torch

    stream = torch.cuda.current_stream()
    feats = torch.empty((n_ev, 4), dtype=torch.float32, device="cuda")
    spec = {"collection": "pflow", "combine": "all", "conditions": [
        {"field": "pt", "op": ">", "value": 1.0}, {"field": "eta", "op": "<", "value": 2.5, "abs": True}]}
    f_view = B.make_filter(spec, compact=False)
    reps = max(3, args.steps)
    for _ in range(3):
        ctx.postprocess(bt, ob, f_view, feats)
    torch.cuda.synchronize()
    ctx.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.postprocess(bt, ob, f_view, feats)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    s_view = e0.elapsed_time(e1) / 1e3 / reps
    # algorithmic bytes: offsets and counts (24 B an event), every track
    # (16 B) and EFlow neutral (12 B) read once, the features (16 B) written
    tot = counts.sum(axis=0)
    alg = 24 * n_ev + 16 * int(tot[0]) + 12 * int(tot[2]) + 16 * n_ev
    f_cmp = B.make_filter(spec, compact=True)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    ctx.postprocess(bt, ob, f_cmp, feats)
    c1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    kept = out["counts"].cpu().numpy().view(np.uint32)[:n_ev].astype(np.int64).sum(axis=0)
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    achieved = alg / s_view / 1e9
    return {"filter": "pflow: pt > 1 GeV and |eta| < 2.5", "events": n_ev,
            "objects": int(tot[0] + tot[2]), "kept_objects": int(kept[0] + kept[2]),
            "ms": s_view * 1e3, "events_per_s": n_ev / s_view,
            "compacting_ms": c0.elapsed_time(c1),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": _traffic_from_profile("batched", "postprocess_kernel"),
                         "algorithmic_bytes_per_launch": int(alg), "kernel": "pdr::postprocess_kernel"},
            "reps": reps}


def bench_pileup_merge(args, B, ctx):
    """Pile-up merging on the device (Sec. 2.2) at the pile-up workload's scale:
    10k hard events of Poisson(400) particles, Poisson(170) interactions each
    from a 10k-event minimum-bias pool, vertex z ~ N(0, 50 mm) truncated at
    250 mm and t ~ N(0, 160 ps) truncated at 800 ps; then the detector response
    of the merged batch."""
    import torch

    from paper_2606_26089_b300 import synth

    hard = synth.make_hard(args.pileup_events)
    pool = synth.make_minbias_pool(10_000)
    hd, pd = B.batch_to_device(hard), B.batch_to_device(pool)
    mean, sz, mz, seed = 170.0, 0.05, 0.25, 3
    hb = B.make_batch(hd, 0, seed)
    pu = B.make_pileup(pd, mean, sz, mz, True)
    n = hard.n_events
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    total = ctx.pileup_offsets(hb, pu, off)
    f = dict(dtype=torch.float32, device="cuda")
    m = {k: torch.empty(total, **f) for k in ("pt", "eta", "phi", "mass", "vz", "vt")}
    m["pdg"] = torch.empty(total, dtype=torch.int32, device="cuda")
    m["charge"] = torch.empty(total, dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream()
    reps = max(3, args.steps // 3)
    for _ in range(3):
        ctx.pileup_merge(hb, pu, off, m)
    torch.cuda.synchronize()
    ctx.check()
    t_off = []
    for _ in range(reps):
        t0 = time.perf_counter()
        ctx.pileup_offsets(hb, pu, off)
        t_off.append(time.perf_counter() - t0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    for k in range(reps):
        ev[2 * k].record(stream)
        ctx.pileup_merge(hb, pu, off, m)
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    fill_s = statistics.mean(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps)) / 1e3
    # algorithmic bytes: every merged particle written once (4 floats, vz, vt,
    # pdg, charge = 29 B), the hard particles and the pool read once, the offsets
    n_int = int(total - hard.n_particles)
    alg = 29 * total + hard.nbytes_input() + pool.nbytes_input() + 8 * (n + 1)
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0

    # detector response of the merged batch
    mdev = dict(m, offsets=off, n_events=n, n_particles=total, max_event_size=0)
    del mdev["vt"]
    cid = ctx.card_load("cms_like")
    out = B.alloc_outputs(n, total)
    bt = B.make_batch(mdev, cid, seed)
    sizes = torch.diff(off)
    bt.max_event_size = int(sizes.max().item())
    launch = B.pdr_launch()
    launch.team, launch.block, launch.table_slots, launch.grid = 1024, 1024, 0, 0
    ob = B.make_outputs(out)
    for _ in range(2):
        ctx.run(bt, ob, launch=launch)
    torch.cuda.synchronize()
    ctx.check()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(reps):
        ctx.run(bt, ob, launch=launch)
    r1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    resp_s = r0.elapsed_time(r1) / 1e3 / reps
    achieved = alg / fill_s / 1e9
    return {"hard_events": n, "pool_events": pool.n_events, "mean_interactions": mean,
            "sigma_z_m": sz, "max_z_m": mz, "merged_particles": int(total), "pool_particles_copied": n_int,
            "fill_ms": fill_s * 1e3, "offsets_ms_incl_sync": statistics.mean(t_off) * 1e3,
            "fill_particles_per_s": total / fill_s,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": _traffic_from_profile("pileup", "pu_fill_kernel"),
                         "algorithmic_bytes_per_launch": int(alg), "kernel": "pdr::pu_fill_kernel"},
            "response_ms": resp_s * 1e3, "response_launch": launch.as_dict(),
            "merge_and_response_particles_per_s": total / (fill_s + resp_s),
            "reps": reps}


def merge_only(args):
    """The pile-up merge object alone on one GPU (for profiling the merge)."""
    import torch

    from paper_2606_26089_b300 import binding as B
    from paper_2606_26089_b300 import build as pdr_build

    pdr_build.build()
    torch.cuda.set_device(0)
    ctx = B.Context(0, pool_bytes=int(args.pool_gb * (1 << 30)))
    try:
        return {"pileup_merge": bench_pileup_merge(args, B, ctx)}
    finally:
        ctx.close()


def cpu_baseline(batch, card_name, seed, target_s):
    """The oracle as it stands, on the host cores, on a bounded prefix of the workload."""
    import oracle

    oracle.build()
    card = oracle.load_card(card_name)
    cores = os.cpu_count() or 1
    n = min(batch.n_events, 200)
    t0 = time.perf_counter()
    oracle.run_batch(card, batch.slice_events(0, n), seed, nthreads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    n_sample = int(min(batch.n_events, max(n, n * target_s / dt)))
    sample = batch.slice_events(0, n_sample)
    t0 = time.perf_counter()
    oracle.run_batch(card, sample, seed, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": sample.n_particles / dt, "unit": "particles/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n_sample} of {batch.n_events} events ({sample.n_particles} particles), "
                      f"{dt:.1f} s on {cores} threads"}


def parity_sample(ctx, cid, batch, card_name, seed, event_base, n_events=200):
    """Marginal decisions of the parity protocol on a sample of the workload:
    the first n_events run again with debug records and compared with the
    oracle event by event (decisions within the oracle's band of their
    threshold are marginal; a flip is one the GPU took the other way)."""
    import oracle
    from tests import parity as P

    sub = batch.slice_events(0, min(n_events, batch.n_events))
    card = oracle.load_card(card_name)
    host = P.run_gpu(ctx, cid, sub, seed, event_base=event_base, debug=True)
    st = P.Stats()
    for e in range(sub.n_events):
        P.compare_event(card, sub.event(e), P.gpu_event(host, sub, e), seed, event_base + e, st)
    return {"events": st.events, "particles": st.particles, "marginal": st.marginal, "flips": st.flips,
            "marginal_per_particle": st.marginal / max(st.particles, 1),
            "flips_per_particle": st.flips / max(st.particles, 1),
            "max_rel": st.max_rel, "band": P.G_BAND}


def bench_reference(args, rank):
    """The reference arm: the FP64 oracle on the host cores, bounded samples."""
    from paper_2606_26089_b300 import synth
    import oracle

    if rank != 0:
        return None
    oracle.build()
    batch = synth.make(args.workload, args.events)
    card = oracle.load_card(synth.card_for(args.workload))
    cores = os.cpu_count() or 1
    n = min(batch.n_events, 200)
    t0 = time.perf_counter()
    oracle.run_batch(card, batch.slice_events(0, n), args.seed, nthreads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    per_step = min(10.0, 150.0 / max(args.steps + args.warmup, 1))
    n_sample = int(min(batch.n_events, max(n, n * per_step / dt)))
    sample = batch.slice_events(0, n_sample)
    for _ in range(args.warmup):
        oracle.run_batch(card, sample, args.seed, nthreads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run_batch(card, sample, args.seed, nthreads=cores)
        times.append(time.perf_counter() - t0)
    s = statistics.mean(times)
    value = sample.n_particles / s
    desc = f"first {n_sample} of {batch.n_events} events ({sample.n_particles} particles) per step"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[args.workload], "card": synth.card_for(args.workload),
                       "n_events": batch.n_events, "n_particles": batch.n_particles, "seed": args.seed,
                       "sample": desc},
            "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOAD_DESC), default="batched")
    ap.add_argument("--events", type=int, default=None, help="override the workload's event count")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--pool-gb", type=float, default=8.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--per-event-events", type=int, default=1000)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--launch", default=None,
                    help="fixed launch shape 'team,block[,table_slots]' (skips autotuning)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-rates", type=float, nargs="+", default=[50, 100, 200, 500, 1000, 2000, 5000])
    ap.add_argument("--serving-max-requests", type=int, default=300)
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--serving-pool", type=int, default=5000)
    ap.add_argument("--no-per-event", action="store_true")
    ap.add_argument("--no-pileup-merge", action="store_true")
    ap.add_argument("--no-postprocess", action="store_true")
    ap.add_argument("--no-track-ip", action="store_true")
    ap.add_argument("--no-jets", action="store_true")
    ap.add_argument("--merge-only", action="store_true",
                    help="time only the pile-up merge (and the merged batch's response); prints that object")
    ap.add_argument("--pileup-events", type=int, default=10_000, help="hard events of the pile-up merge")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.seed is None:
        args.seed = {"tiny": 0, "batched": 1, "ee": 2, "pileup": 3}[args.workload]
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        # rank 0 alone times the oracle; other ranks exit without work
        rank = int(os.environ.get("RANK", "0"))
        line = bench_reference(args, rank)
        if rank == 0 and line is not None:
            print(json.dumps(line), flush=True)
        return
    if args.merge_only:
        print(json.dumps(merge_only(args)), flush=True)
        return
    dist, rank, ws = _dist()
    line = bench_ours(args, dist, rank, ws)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
