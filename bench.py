#!/usr/bin/env python3
"""Benchmark of the multi-component progressive compression and retrieval path.

Workload (the large plain-method configuration): a 512^3 random-phase Gaussian
field with a k^-5/3 power spectrum, in float32 and in float64, compressed into
8 components with tau_i = 10^-(i+1) * range (i = 1..8), then retrieved at every
k = 1..8 (Algorithm 1 once, Algorithm 2 for each k).  One step = for each dtype:
range reduction -> tolerance schedule -> compress -> 8 queries + retrievals.

`value` is raw field bytes processed per second over the whole step (each
compress and each retrieval counts the field's bytes once), with the fields
resident in HBM when timing starts; both fields exceed the 129 MB L2, so no
flush is needed between steps.  `e2e` is the same metric through the same
calls with host (pinned) buffers: the kernels read the field from host memory
and write every retrieval to host memory in place, across the host link.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pcz|reference]

The line also carries `batched`: the uneven batch of 64 float32 fields (half
2D, half 3D, 6 components) compressed by one graph-replayed persistent launch
and retrieved by one launch per dimensionality, against per-field calls; and
`serving`: the progressive-query workload (16 float32
256^3 k^-5/3 fields resident on the device, 8 components each; 10,000 seeded
queries arriving as a Poisson stream at 2,000/s, each a brick-aligned sub-box
with sides log-uniform in [8, 256] at a relative tolerance log-uniform in
[1e-7, 1e-1]; 20 GB device-memory budget) replayed through the batched,
cached server and through the unbatched plain pipeline (one query per
launch, no cache), with p50/p99 latency from arrival to completion.

With --impl reference the CPU oracle (the test-infrastructure implementation
of the same method) is timed on a bounded sample of the same workload.  For
N > 1 (torchrun) every rank runs its own replica: the method has no data-path
exchange (bricks are independent), so there is no collective beyond the
timing barrier.
"""
import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_COMP = 8
METRIC = "compress/retrieve GB/s vs HBM roofline; progressive-query p50/p99 latency"
# DRAM bytes (read + write) and warp instructions per launch of the dominant kernel on this
# workload, means over the 16 retrieval launches of a step (k = 1..8, float32 and float64), from
# ncu captures of the current kernels at 512^3 (gpu__time_duration, dram__bytes_read/write,
# smsp__inst_executed: one pass), one per type.
TRAFFIC = {"retrieve": 1298626048}
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, mean over the 16 retrieval launches "
                  "(k = 1..8, float32 and float64) of this workload at 512^3")
INSTRUCTIONS = {"retrieve": 2046510995}
# Pipe utilisation (ncu --set full on the 320^3 case of this workload): the retrieval (k = 8)
# and compression kernels are bound by instruction issue, not by HBM.  The float32 retrieval
# figures are of the current kernel; the float64 ones of the kernel before the 32-bit decoding
# of narrow brick pairs (11 % less time at k = 8 since, with the int -> double conversions off
# the FP64 pipe); compression has since dropped a warp vote and some FP64 operations (2-4 %
# less time; float64 9 %, its magnitude tests no longer compiling to FP64 adds), its figures
# are of the kernel before that.
PIPES = {"launch": "320^3, retrieval at k = 8, compression of 8 components",
         "retrieve": {"alu": {"f32": 0.569, "f64": 0.574}, "fp64": {"f32": 0.0, "f64": 0.662},
                      "issue_active": {"f32": 0.677, "f64": 0.604}},
         "compress": {"alu": {"f32": 0.708, "f64": 0.598}, "fp64": {"f32": 0.0, "f64": 0.464},
                      "issue_active": {"f32": 0.762, "f64": 0.584}},
         "source": "ncu sm__inst_executed_pipe_{alu,fp64}.avg.pct_of_peak_sustained_active, "
                   "smsp__issue_active.avg.pct_of_peak_sustained_active; compression figures from the "
                   "kernel before its last changes (2-4 % less time since for float32, 9 % for float64, whose "
                   "magnitude tests no longer compile to FP64 adds); float64 retrieval figures from the "
                   "kernel before its 32-bit decoding of narrow brick pairs (11 % less time at k = 8 since)"}
BATCH_WORKLOAD = ("64 float32 fields, half 2D with extents in [256, 4096], half 3D between 32^3 and "
                  "384x384x256 (not multiples of 4), half sums of Gaussians and half k^-5/3 spectra, 6 components "
                  "(tau_i = 1e-(i+1) * range)")
SERVE_WORKLOAD = ("16 device-resident float32 256^3 k^-5/3 fields, 8 components (tau_i = 1e-(i+1) * range); "
                  "Poisson arrivals at 2000/s; brick-aligned sub-boxes with sides log-uniform in [8, 256]; "
                  "relative tolerance log-uniform in [1e-7, 1e-1]; 20 GB budget")
WORKLOAD = ("512^3 random-phase Gaussian field (P(k) ~ k^-5/3, unit variance), float32 and float64, "
            "8 components, tau_i = 1e-(i+1) * range, compress then retrieval at every k = 1..8")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.lines = []
        self.proc = None
        self.bus_id = bus_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(mhz)}


def issue_roofline(kernel, ms_per_launch, clocks):
    """The bound the kernels actually sit on: warp instructions issued per second
    (the kernel's instructions per launch from the ncu capture, over its live
    CUDA-event duration) against the SMs' issue peak, 152 SMs x 4 schedulers x one
    warp instruction per clock, at the median SM clock sampled in the timed region."""
    inst = INSTRUCTIONS.get(kernel)
    if not inst or ms_per_launch <= 0:
        return None
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    achieved = inst / (ms_per_launch * 1e-3)
    peak = 152 * 4 * mhz * 1e6
    return {"achieved": round(achieved / 1e9, 1), "peak": round(peak / 1e9, 1), "unit": "G warp-instructions/s",
            "frac": round(achieved / peak, 4), "sm_mhz": mhz,
            "instructions_per_launch": inst, "source": "ncu smsp__inst_executed.sum, mean over the same 16 launches"}


def max_over_ranks(ms, world, device):
    """The slowest rank's time (every rank gets it): the whole job is done
    when the last replica is."""
    if world <= 1:
        return ms
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_gbs(world, bytes_per_rank_step, steps, ms_total):
    """Whole-job throughput: every rank's bytes over the slowest rank's time."""
    return world * bytes_per_rank_step * steps / (ms_total * 1e-3) / 1e9


def make_fields(size, device, dtypes=("f32", "f64")):
    import torch

    import synth_fields as S

    f64 = S.powerlaw((size, size, size), seed=2, dtype=np.float64, device=device)
    out = {}
    if "f32" in dtypes:
        out["f32"] = f64.to(torch.float32).contiguous()
    if "f64" in dtypes:
        out["f64"] = f64.contiguous()
    torch.cuda.synchronize()
    return out


def algorithmic_bytes(st, field_bytes):
    """Bytes the method must move: compress = read x + write every component's
    payload and index; retrieval at k = read components 1..k + write x~."""
    comp_payload = []
    idx = 0
    for i in range(st.n):
        _, bits, ib = st.info(i)
        comp_payload.append(bits // 8)
        idx = ib
    compress = field_bytes + sum(comp_payload) + st.n * idx
    retrieve = [sum(comp_payload[:k]) + k * idx + field_bytes for k in range(1, st.n + 1)]
    return compress, retrieve, comp_payload


def e2e_two_streams(args, world, device, fields, hbufs, held, raw_bytes_step):
    """The e2e step with each field's pipeline (range and schedule, compress,
    query and retrieval at every k into pinned host memory) on a stream of its
    own, driven by a host thread of its own: one field's transfers over the
    host link overlap the other's kernels.  Same calls, inputs, outputs and
    bytes as the e2e step."""
    from concurrent.futures import ThreadPoolExecutor

    import torch

    import paper_2308_11759_gb300 as pcz

    names = list(fields)
    # the first field's pipeline at the higher priority: its retrievals (and
    # the transfers they feed) are scheduled ahead of the second field's
    # compression as CTAs drain, so the host link is busy while the SMs compress
    streams = {n: torch.cuda.Stream(device=device, priority=(-1 if j == 0 else 0)) for j, n in enumerate(names)}
    pool = ThreadPoolExecutor(max_workers=len(names))  # the same host threads every step

    def pipeline(name):
        s = streams[name]
        with torch.cuda.stream(s):
            x = hbufs[name]
            tau = pcz.field_tau_schedule(x, "decade", N_COMP, stream=s)
            if name in held:
                held.pop(name).close()
            st = pcz.compress(x, tau, stream=s)
            held[name] = st
            for k in range(1, N_COMP + 1):
                st.retrieve(k=st.query_k(tau[k - 1]), out=hbufs[name + "_out"], stream=s)

    def step():
        cur = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(cur)
        for s in streams.values():
            s.wait_event(start)
        for f in [pool.submit(pipeline, n) for n in names]:
            f.result()  # re-raises a pipeline's exception
        for s in streams.values():
            cur.wait_stream(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    gc.collect()
    gc.disable()
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    marks[0].record()
    for i in range(args.steps):
        step()
        marks[i + 1].record()
    torch.cuda.synchronize()
    gc.enable()
    pool.shutdown()
    ems = max_over_ranks(marks[0].elapsed_time(marks[-1]), world, device)
    return {"value": round(job_gbs(world, raw_bytes_step, args.steps, ems), 3), "unit": "GB/s",
            "ms_per_step": round(ems / args.steps, 3),
            "ms_steps": [round(marks[i].elapsed_time(marks[i + 1]), 2) for i in range(args.steps)],
            "note": "each field's pipeline on its own stream and (persistent) host thread; same calls and bytes as e2e"}


def run_pcz(args, rank, world, device):
    import torch

    import paper_2308_11759_gb300 as pcz

    pcz.lib()
    fields = make_fields(args.size, device, tuple(args.dtypes.split(",")))
    outs = {k: torch.empty_like(v) for k, v in fields.items()}
    nvox = args.size ** 3
    held = {}

    def step(host=False, hbufs=None):
        for name, x in fields.items():
            if host:  # e2e: the field is in pinned host memory; the kernels read it in place
                x = hbufs[name]
            tau = pcz.field_tau_schedule(x, "decade", N_COMP)  # a1: tau_0 = range, tau_i
            if name in held:
                held.pop(name).close()
            st = pcz.compress(x, tau)  # a2..a9
            held[name] = st
            dst = hbufs[name + "_out"] if host else outs[name]
            for k in range(1, N_COMP + 1):  # a10, a11: query at tau_k, then Algorithm 2
                kk = st.query_k(tau[k - 1])
                st.retrieve(k=kk, out=dst)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # sizes and per-component rates of this workload
    info = {}
    for name, x in fields.items():
        st = held[name]
        fb = x.numel() * x.element_size()
        cb, rb, pay = algorithmic_bytes(st, fb)
        info[name] = dict(field_bytes=fb, compress_bytes=cb, retrieve_bytes=rb,
                          rates=[round(8 * p / nvox, 4) for p in pay],
                          counts=[st.counts(i) for i in range(st.n)],
                          measured_over_tau=[float("%.4g" % (st.measured_error(i) / st.tau(i))) for i in range(st.n)])

    bus = None
    try:
        props = torch.cuda.get_device_properties(device)
        bus = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    except Exception:
        pass
    sampler = ClockSampler(bus)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    pcz.timing_enable(True)
    sampler.start()
    gc.collect()
    gc.disable()  # no collector pauses inside the timed steps (the host is on the steps' critical path)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        step()
    t1.record()
    torch.cuda.synchronize()
    gc.enable()
    clocks = sampler.stop()
    ktimes = pcz.timing_read()
    pcz.timing_enable(False)
    if world > 1:
        torch.distributed.barrier()
    ms_total = max_over_ranks(t0.elapsed_time(t1), world, device)
    ms_step = ms_total / args.steps
    raw_bytes_step = sum(v["field_bytes"] * (1 + N_COMP) for v in info.values())
    value = job_gbs(world, raw_bytes_step, args.steps, ms_total)

    # roofline of the dominant kernel, from its live CUDA-event durations
    hbm, peak_kind = peaks()
    alg = {"compress": sum(v["compress_bytes"] for v in info.values()) * args.steps,
           "retrieve": sum(sum(v["retrieve_bytes"]) for v in info.values()) * args.steps,
           "range": sum(v["field_bytes"] for v in info.values()) * args.steps,
           "pack": 2 * sum(v["compress_bytes"] - v["field_bytes"] for v in info.values()) * args.steps}
    dom = max(("compress", "retrieve"), key=lambda k: ktimes[k][0])
    dom_ms, dom_n = ktimes[dom]
    achieved = alg[dom] / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else 0.0
    kernels = {}
    for k, (ms, n) in ktimes.items():
        if n:
            kernels[k] = {"launches": n, "ms_per_launch": round(ms / n, 4), "share": round(ms / ms_total, 4),
                          "gbs_algorithmic": round(alg[k] / (ms * 1e-3) / 1e9, 1) if k in alg and ms > 0 else None}
    launches = sum(n for _, n in ktimes.values())

    # per field type: kernel times from the library's events, the median of
    # args.kernel_reps launches each (outside the timed step)
    per_dtype = {}
    reps = max(1, args.kernel_reps)
    for name, x in fields.items():
        st = held[name]
        fb = info[name]["field_bytes"]
        tau = [st.tau(i) for i in range(st.n)]
        cl = []
        for _ in range(reps):
            pcz.timing_enable(True)
            st2 = pcz.compress(x, tau)
            cl.append(pcz.timing_read()["compress"][0])
            pcz.timing_enable(False)
            st2.close()
        rms = []
        for k in range(1, N_COMP + 1):
            rl = []
            for _ in range(reps):
                pcz.timing_enable(True)
                st.retrieve(k=k, out=outs[name])
                rl.append(pcz.timing_read()["retrieve"][0])
            rms.append(statistics.median(rl))
        pcz.timing_enable(False)
        cms = statistics.median(cl)
        per_dtype[name] = {"compress_ms": round(cms, 3), "compress_gbs": round(fb / (cms * 1e-3) / 1e9, 2),
                           "launches_per_median": reps,
                           "compress_roofline_frac": round(info[name]["compress_bytes"] / (cms * 1e-3) / 1e9 / hbm, 5),
                           "retrieve_ms_per_k": [round(v, 3) for v in rms],
                           "retrieve_gbs": round(N_COMP * fb / (sum(rms) * 1e-3) / 1e9, 2),
                           "retrieve_roofline_frac": round(sum(info[name]["retrieve_bytes"]) / (sum(rms) * 1e-3) / 1e9
                                                           / hbm, 5)}

    # accuracy gain (Sec. 5.1.1): alpha_k = log2(sigma / RMSE_k) - R_k, with R_k the
    # stream bits per value of components 1..k (index included)
    gain = {}
    for name, x in fields.items():
        st = held[name]
        x64 = x.double()
        sigma = float(x64.std())
        tmp = torch.empty_like(x)
        rate, al = 0.0, []
        for k in range(1, N_COMP + 1):
            _, bits, ib = st.info(k - 1)
            rate += (bits + 8 * ib) / nvox
            st.retrieve(k=k, out=tmp)
            rmse = float(torch.sqrt(torch.mean((x64 - tmp.double()) ** 2)))
            al.append(round(math.log2(sigma / rmse) - rate, 3) if rmse > 0 else None)
        gain[name] = al
        del x64, tmp

    # progressive sweep (Sec. 4.2): x~_1, then x~_k refined in place from x~_(k-1)
    # for k = 2..n.  It yields the same n reconstructions as the independent
    # retrievals of the step, decoding each component once instead of k times.
    sweep = {}
    for name, x in fields.items():
        st = held[name]
        buf = torch.empty_like(x)

        def sweep_once():
            st.retrieve(k=1, out=buf)
            for k in range(2, N_COMP + 1):
                st.refine(k - 1, k, buf)

        sweep_once()
        torch.cuda.synchronize()
        same = bool(torch.equal(buf.view(torch.int32 if x.element_size() == 4 else torch.int64),
                                outs[name].view(torch.int32 if x.element_size() == 4 else torch.int64)))
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(args.steps):
            sweep_once()
        s1.record()
        torch.cuda.synchronize()
        ms = s0.elapsed_time(s1) / args.steps
        fb = info[name]["field_bytes"]
        sweep[name] = {"ms": round(ms, 3), "gbs_out": round(N_COMP * fb / (ms * 1e-3) / 1e9, 1),
                       "equals_independent_k%d" % N_COMP: same}
        del buf

    # e2e: the same step through host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hbufs = {}
        for name, x in fields.items():
            hbufs[name] = x.cpu().pin_memory()
            hbufs[name + "_out"] = torch.empty(x.shape, dtype=x.dtype).pin_memory()
        for _ in range(args.warmup):
            step(host=True, hbufs=hbufs)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        gc.collect()
        gc.disable()
        a = time.perf_counter()
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        marks[0].record()
        for i in range(args.steps):
            step(host=True, hbufs=hbufs)
            marks[i + 1].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - a
        gc.enable()
        ems = max_over_ranks(marks[0].elapsed_time(marks[-1]), world, device)
        h2d = sum(v["field_bytes"] for v in info.values())
        d2h = sum(v["field_bytes"] * N_COMP for v in info.values())
        e2e = {"value": round(job_gbs(world, raw_bytes_step, args.steps, ems), 3), "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(ems / args.steps, 3),
               "ms_steps": [round(marks[i].elapsed_time(marks[i + 1]), 2) for i in range(args.steps)],
               "host_wall_s": round(wall, 3)}
        if len(fields) > 1:
            e2e["two_streams"] = e2e_two_streams(args, world, device, fields, hbufs, held, raw_bytes_step)
    for st in held.values():
        st.close()
    return dict(value=value, ms_step=ms_step, info=info, clocks=clocks, kernels=kernels, launches=launches, gain=gain,
                per_dtype=per_dtype,
                sweep=sweep,
                roofline={"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm,
                          "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                          "traffic": TRAFFIC.get(dom),
                          "traffic_source": TRAFFIC_SOURCE if TRAFFIC.get(dom) else None,
                          "algorithmic_bytes_per_launch": int(alg[dom] / max(dom_n, 1)),
                          "ms_per_launch": round(dom_ms / max(dom_n, 1), 4),
                          "issue": issue_roofline(dom, dom_ms / max(dom_n, 1), clocks)},
                e2e=e2e, fields=fields)


def serve_queries(nq, nfields, size, ranges, seed=41, rate=2000.0):
    """The seeded request stream: (field, box, tau, k=0) and arrival times."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, nq))
    arrivals -= arrivals[0]
    qs = []
    for _ in range(nq):
        f = int(rng.integers(0, nfields))
        lo, hi = [], []
        for _a in range(3):
            side = 4 * int(round(np.exp(rng.uniform(np.log(8.0), np.log(float(size)))) / 4.0))
            side = min(max(side, 8), size)
            o = 4 * int(rng.integers(0, (size - side) // 4 + 1))
            lo.append(o)
            hi.append(o + side)
        rel = 10.0 ** rng.uniform(-7.0, -1.0)
        qs.append((f, (lo, hi), rel * ranges[f], 0))
    return qs, arrivals.tolist()


def run_serving(args, device):
    """Replays the request stream through the batched, cached server and
    through the unbatched plain pipeline; p50/p99 latency and throughput."""
    import torch

    import paper_2308_11759_gb300 as pcz
    import synth_fields as S

    size, nf = args.serve_size, 16
    streams, ranges = [], []
    for f in range(nf):
        x = S.powerlaw((size, size, size), seed=100 + f, dtype=np.float32, device=device)
        lo, hi = pcz.field_range(x)
        ranges.append(hi - lo)
        streams.append(pcz.compress(x, pcz.field_tau_schedule(x, "decade", N_COMP)))
        del x
    torch.cuda.synchronize()
    qs, arr = serve_queries(args.serve_queries, nf, size, ranges)
    budget = 20 * 10 ** 9
    out = {"workload": SERVE_WORKLOAD, "queries": len(qs), "rate_per_s": 2000, "budget_bytes": budget,
           "latency": "arrival to the batch's completion on the device (a host function queued behind the batch); "
                      "results stay in device memory"}
    # the same queries at a 10x higher Poisson rate, and in bursts (groups of 100
    # arriving together, bursts Poisson at 200/s: 20,000 queries/s on average)
    _, arr_fast = serve_queries(args.serve_queries, nf, size, ranges, rate=20000.0)
    brng = np.random.default_rng(np.random.PCG64(43))
    burst_t = np.cumsum(brng.exponential(1.0 / 200.0, (len(qs) + 99) // 100))
    arr_burst = [float(burst_t[j // 100] - burst_t[0]) for j in range(len(qs))]
    streams_in = {"poisson_20000_per_s": arr_fast, "bursts_of_100_at_200_per_s": arr_burst}

    def summary(lat, stats):
        lat_ms = 1e3 * lat
        return {"p50_ms": round(float(np.percentile(lat_ms, 50)), 4),
                "p99_ms": round(float(np.percentile(lat_ms, 99)), 4),
                "mean_ms": round(float(lat_ms.mean()), 4), "max_ms": round(float(lat_ms.max()), 4),
                "throughput_qps": round(stats["queries"] / stats["wall_s"], 1),
                "gbs_out": round(stats["bytes_out"] / stats["wall_s"] / 1e9, 3),
                "batches": stats["batches"], "mean_batch": round(stats["queries"] / max(stats["batches"], 1), 2),
                "max_batch": stats["max_batch"], "max_inflight": stats["max_inflight"],
                "peak_device_gb": round(stats["peak_device_bytes"] / 1e9, 3), "wall_s": round(stats["wall_s"], 3)}

    for name, kw in (("batched", {"max_batch": 512}), ("plain", {"serial": True, "cache": False})):
        srv = pcz.Server(budget, **kw)
        for st in streams:
            srv.add_field(st)
        warm_q, warm_a = serve_queries(64, nf, size, ranges, seed=7)
        srv.replay(warm_q, [0.0] * len(warm_q))  # warm-up (kernels loaded, arena touched)
        srv.reset_cache()
        lat, stats = srv.replay(qs, arr)
        out[name] = summary(lat, stats)
        for sname, sarr in streams_in.items():
            srv.reset_cache()
            lat2, stats2 = srv.replay(qs, sarr)
            out[name][sname] = summary(lat2, stats2)
        srv.reset_cache()
        blat, bstats = srv.replay(qs, [0.0] * len(qs))  # saturation: the whole stream waiting at once
        out[name]["all_at_once"] = summary(blat, bstats)
        srv.close()
    for st in streams:
        st.close()
    return out


def run_batched(args, device):
    """The uneven batch: one graph-replayed persistent launch for all 64
    fields against a loop of per-field compress calls; batched retrieval of
    every field at k = 6 against per-field retrievals."""
    import torch

    import paper_2308_11759_gb300 as pcz
    import synth_fields as S

    shapes = S.batched_shapes(64, seed=3)
    fields = []
    for j, sh in enumerate(shapes):
        if (j // 2) % 2 == 0:
            fields.append(S.gaussians(sh, seed=200 + j, dtype=np.float32, device=device).contiguous())
        else:
            fields.append(S.powerlaw(sh, seed=200 + j, dtype=np.float32, device=device).contiguous())
    taus = []
    for x in fields:
        taus.append(pcz.field_tau_schedule(x, "decade", 6))
    torch.cuda.synchronize()
    raw = sum(x.numel() * 4 for x in fields)
    plan = pcz.Batch(shapes, np.float32, 6)
    t_tune = time.perf_counter()
    for st in plan.compress(fields, taus):  # first call: the autotuner times its schedules
        st.close()
    t_tune = time.perf_counter() - t_tune
    reps = max(2, args.steps)

    def timed(fn):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def batched():
        for st in plan.compress(fields, taus):
            st.close()

    def loop():
        for x, t in zip(fields, taus):
            pcz.compress(x, t).close()

    ms_b = timed(batched)
    ms_l = timed(loop)
    sts = plan.compress(fields, taus)
    outs = [torch.empty_like(x) for x in fields]
    ms_rb = timed(lambda: pcz.retrieve_batch(sts, [6] * len(sts), outs=outs))

    def rloop():
        for st, o in zip(sts, outs):
            st.retrieve(k=6, out=o)

    ms_rl = timed(rloop)
    bits = sum(st.info(i)[1] for st in sts for i in range(6)) / (raw / 4)
    for st in sts:
        st.close()
    info = plan.info()
    plan.close()
    # the oracle on a sample of the batch: a 512^2 corner of the first 2D field
    # and a 64^3 corner of the first 3D field, compress + retrieval at k = 6
    import oracle as O

    sample = [np.ascontiguousarray(fields[0][:512, :512].cpu().numpy()),
              np.ascontiguousarray(fields[1][:64, :64, :64].cpu().numpy())]
    oracle = {}
    for cores in (1, os.cpu_count() or 1):
        t = time.perf_counter()
        for xs in sample:
            tau = O.tau_decade(O.value_range(xs), 6)
            O.Streams(xs, tau, nthreads=cores).retrieve(6)
        secs = time.perf_counter() - t
        nbytes = sum(xs.nbytes for xs in sample)
        oracle["single_core" if cores == 1 else "all_cores"] = {
            "gbs": round(2 * nbytes / secs / 1e9, 5), "cores": cores,
            "sample": "512^2 corner of the first 2D field and 64^3 corner of the first 3D field, "
                      "compress + retrieval at k = 6 (bytes counted twice)"}
    return {"workload": BATCH_WORKLOAD, "fields": len(shapes), "raw_bytes": raw,
            "compress": {"batched_gbs": round(raw / (ms_b * 1e-3) / 1e9, 3), "batched_ms": round(ms_b, 3),
                         "per_field_loop_gbs": round(raw / (ms_l * 1e-3) / 1e9, 3),
                         "per_field_loop_ms": round(ms_l, 3)},
            "retrieve_k6": {"batched_gbs": round(raw / (ms_rb * 1e-3) / 1e9, 3), "batched_ms": round(ms_rb, 3),
                            "per_field_loop_gbs": round(raw / (ms_rl * 1e-3) / 1e9, 3),
                            "per_field_loop_ms": round(ms_rl, 3)},
            "bits_per_value": round(bits, 3),
            "autotuner": {"schedule": info["schedule"], "order": info["order"],
                          "chunks_per_item": info["chunks_per_item"], "items_per_claim": info["items_per_claim"],
                          "ctas_per_sm_3d": info["ctas_per_sm"], "warps_per_cta_1d2d": info["warps_small"],
                          "one_kernel_for_both": bool(info["mixed"]),
                          "candidates": "3D CTAs of 16 warps per SM {2, 1} x 1D/2D warps per CTA {4, 8, 16}, and "
                                        "for 2 CTAs: 1D/2D warps {2, 4, 8, 16} x chunks per warp per item {1, 2} "
                                        "(two kernels); one kernel for both with 1 or 2 chunks per warp; two items "
                                        "per claim or the fields in the given order for 3 shapes",
                          "candidate_ms": [round(v, 3) for v in info["candidate_ms"]],
                          "spread": round(max(v for v in info["candidate_ms"] if v > 0)
                                          / min(v for v in info["candidate_ms"] if v > 0) - 1.0, 4),
                          "first_call_s": round(t_tune, 3)},
            "graph": bool(info["graph"]), "timing": "CUDA events around whole calls (host work included)",
            "oracle": oracle}


def run_lossless(device):
    """Sec. 5.1.3 on synthetic fields: components (binary schedule, delta = 4,
    8 and 16) until the computed tolerance is 0, the bits per value that takes
    (index included), and the lossless compression ratio."""
    import torch

    import paper_2308_11759_gb300 as pcz
    import synth_fields as S

    out = {}
    cases = (("powerlaw_128^3_f32", lambda: S.powerlaw((128,) * 3, seed=2, dtype=np.float32, device=device)),
             ("powerlaw_128^3_f64", lambda: S.powerlaw((128,) * 3, seed=2, dtype=np.float64, device=device)),
             ("fronts_128^3_f64", lambda: S.fronts((128,) * 3, seed=5, dtype=np.float64, device=device)),
             ("gaussians_64^3_f64", lambda: torch.from_numpy(S.gaussians((64,) * 3, seed=1)).to(device)))
    for name, make in cases:
        x = make().contiguous()
        out[name] = {}
        for delta in (4, 8, 16):
            r = pcz.lossless_sweep(x, delta=delta)
            out[name][f"delta{delta}"] = {"components": r["k"],
                                          "bits_per_value": round(r["bits_per_value"], 3) if r["k"] else None,
                                          "ratio": round(r["ratio"], 3) if r["k"] else None}
            r["streams"].close()
    return out


class L2Flush:
    """Writes a buffer larger than the 129 MB L2 between timed launches of a
    small configuration, so that no launch starts with its inputs cached."""

    def __init__(self, device):
        import torch

        self.buf = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=device)  # 256 MB

    def __call__(self):
        self.buf.fill_(1.0)


def timed_events(fn, reps, flush=None):
    """Mean ms of fn over reps launches, each bracketed by CUDA events on the
    current stream (the flush, if any, runs outside the brackets)."""
    import torch

    total = 0.0
    for _ in range(reps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    return total / reps


def run_config1(args, device, nthreads):
    """The small plain-method configuration: a 64^3 float64 sum of 32 random
    anisotropic Gaussians plus N(0, 1e-3) noise, 4 components, tau_i =
    2^-4i * range (Delta = 4): compress, then retrieval at every k.  The field
    (2 MiB) fits in L2, so L2 is flushed before every timed launch.  The
    oracle is timed on the same field, whole, on one core and on all cores."""
    import torch

    import oracle as O
    import paper_2308_11759_gb300 as pcz
    import synth_fields as S

    xn = S.gaussians((64, 64, 64), seed=1)
    x = torch.from_numpy(xn).to(device)
    tau = pcz.field_tau_schedule(x, "binary", 4, param=4)
    flush = L2Flush(device)
    reps = max(5, args.steps)
    st = pcz.compress(x, tau)
    pcz.timing_enable(True)
    ms_c = timed_events(lambda: pcz.compress(x, tau).close(), reps, flush)
    kt = pcz.timing_read()
    out = torch.empty_like(x)
    ms_r = []
    for k in range(1, 5):
        ms_r.append(timed_events(lambda: st.retrieve(k=k, out=out), reps, flush))
    kt2 = pcz.timing_read()
    pcz.timing_enable(False)
    fb = x.numel() * 8
    cb, rb, pay = algorithmic_bytes(st, fb)
    hbm, _ = peaks()
    k_comp_ms = kt["compress"][0] / max(kt["compress"][1], 1)
    k_ret_ms = (kt2["retrieve"][0] - kt["retrieve"][0]) / max(kt2["retrieve"][1] - kt["retrieve"][1], 1)
    st.close()
    # the oracle on the whole field: one core (the paper's mode) and all cores
    oc = {}
    for cores in (1, nthreads):
        t = time.perf_counter()
        s = O.Streams(xn, tau, nthreads=cores)
        for k in range(1, 5):
            s.retrieve(k)
        secs = time.perf_counter() - t
        oc[cores] = {"value": round(fb * 5 / secs / 1e9, 5), "unit": "GB/s", "cores": cores, "seconds": round(secs, 3)}
    return {"workload": "64^3 float64 sum of 32 Gaussians + N(0, 1e-3) noise, 4 components, tau_i = 2^-4i range",
            "compress": {"ms": round(ms_c, 4), "gbs": round(fb / (ms_c * 1e-3) / 1e9, 2),
                         "kernel_ms": round(k_comp_ms, 4),
                         "roofline_frac_kernel": round(cb / (k_comp_ms * 1e-3) / 1e9 / hbm, 5)},
            "retrieve": {"ms_per_k": [round(v, 4) for v in ms_r],
                         "gbs": round(4 * fb / (sum(ms_r) * 1e-3) / 1e9, 2),
                         "kernel_ms_mean": round(k_ret_ms, 4),
                         "roofline_frac_kernel": round((sum(rb) / 4) / (k_ret_ms * 1e-3) / 1e9 / hbm, 5)},
            "rates_bits_per_value": [round(8 * p / (fb / 8), 4) for p in pay],
            "timing": "CUDA events around whole C-ABI calls (host work included), L2 flushed before each",
            "oracle_single_core": oc[1], "oracle_all_cores": oc[nthreads]}


def run_use_case(args, device):
    """Sec. 5.3's progressive use case on a synthetic stand-in for a velocity
    field (three k^-5/3 components, 384 x 384 x 256 float64, the shape of the
    paper's Miranda field, scaled to standard deviation 4), each compressed
    with the tolerances of the paper's figure, tau = 1, 2^-4, 2^-9: per k the
    errors of the velocity, of omega_z = v_x - u_y and of w_zz against the
    derivatives of the original field; then the derivative kernels timed
    against the HBM roofline on float64 and float32 fields."""
    import torch

    import paper_2308_11759_gb300 as pcz
    import synth_fields as S

    shape = (256, 384, 384)  # (nz, ny, nx)
    tau = [1.0, 2.0 ** -4, 2.0 ** -9]
    vel = [S.powerlaw(shape, seed=700 + c, dtype=np.float64, device=device) * 4.0 for c in range(3)]
    streams = [pcz.compress(c, tau) for c in vel]
    om_ref = pcz.fd_vorticity_z(vel[0], vel[1])
    wzz_ref = pcz.fd_second(vel[2], 2)
    om_max, wzz_max = float(om_ref.abs().max()), float(wzz_ref.abs().max())
    per_k = []
    for k in range(1, 4):
        rec = [st.retrieve(k=k) for st in streams]
        d_vel = max(float((r - c).abs().max()) for r, c in zip(rec, vel))
        d_om = float((pcz.fd_vorticity_z(rec[0], rec[1]) - om_ref).abs().max())
        d_wzz = float((pcz.fd_second(rec[2], 2) - wzz_ref).abs().max())
        bits = sum(sum(st.info(i)[1] + 8 * st.info(i)[2] for i in range(k)) for st in streams) / (3 * rec[0].numel())
        per_k.append({"k": k, "tau": tau[k - 1], "bits_per_value": round(bits, 3),
                      "velocity_max_err": float("%.4g" % d_vel),
                      "vorticity_max_err": float("%.4g" % d_om), "vorticity_rel": float("%.4g" % (d_om / om_max)),
                      "w_zz_max_err": float("%.4g" % d_wzz), "w_zz_rel": float("%.4g" % (d_wzz / wzz_max))})
        del rec
    for st in streams:
        st.close()
    # the kernels: fields larger than L2, so every timed launch reads DRAM
    hbm, _ = peaks()
    kern = {}
    reps = max(5, args.steps)
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        u, v, w = (c.to(dt) for c in vel)
        out = torch.empty_like(u)
        nb = u.numel() * u.element_size()
        res = {}
        for op, fn, nbytes in (("vorticity_z", lambda: pcz.fd_vorticity_z(u, v, out=out), 3 * nb),
                               ("w_zz", lambda: pcz.fd_second(w, 2, out=out), 2 * nb)):
            fn()
            pcz.timing_enable(True)
            for _ in range(reps):
                fn()
            kt = pcz.timing_read()
            pcz.timing_enable(False)
            ms = kt["fd"][0] / max(kt["fd"][1], 1)
            res[op] = {"ms": round(ms, 4), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                       "roofline_frac": round(nbytes / (ms * 1e-3) / 1e9 / hbm, 4),
                       "algorithmic_bytes": nbytes}
        kern[name] = res
        del u, v, w, out
    # the oracle (numpy, one host thread) on the same float64 fields, beside the kernels
    from oracle import derivatives as D

    hu, hv, hw = (c.cpu().numpy() for c in vel)
    t = time.perf_counter()
    D.vorticity_z(hu, hv)
    t_om = time.perf_counter() - t
    t = time.perf_counter()
    D.second(hw, 2)
    t_wzz = time.perf_counter() - t
    nb = hu.nbytes
    kern["oracle_f64"] = {"vorticity_z": {"ms": round(1e3 * t_om, 1), "gbs": round(3 * nb / t_om / 1e9, 3)},
                          "w_zz": {"ms": round(1e3 * t_wzz, 1), "gbs": round(2 * nb / t_wzz / 1e9, 3)},
                          "cores": 1, "kind": "oracle (numpy)"}
    return {"workload": "3 float64 components of 384 x 384 x 256 (k^-5/3, std 4), tau = 1, 2^-4, 2^-9, h = 1",
            "per_k": per_k, "vorticity_max": round(om_max, 4), "w_zz_max": round(wzz_max, 4),
            "kernels": kern, "bound": "hbm (algorithmic bytes: inputs read once, output written once)"}


def run_config5(args, device, nthreads):
    """The near-lossless large configuration: a 1024^3 float64 k^-5/3 field plus
    sharp tanh fronts (8 GiB), 12 components, tau_i = 10^-i * range: compress,
    the full progressive sweep (retrieve k = 1, then refine in place up to 12),
    and a mixed-tolerance query stream through the batched, cached server and
    through the plain pipeline.  The oracle is timed on a 128^3 corner and
    extrapolated per brick (bricks are coded independently)."""
    import torch

    import oracle as O
    import paper_2308_11759_gb300 as pcz
    import synth_fields as S

    n = 12
    size = args.c5_size
    x = S.fronts((size, size, size), seed=5, dtype=np.float64, device=device).contiguous()
    tau = pcz.field_tau_schedule(x, "decade", n, param=1)
    xs128 = np.ascontiguousarray(x[:min(128, size), :min(128, size), :min(128, size)].cpu().numpy())
    xs64 = np.ascontiguousarray(xs128[:64, :64, :64])
    torch.cuda.synchronize()
    fb = x.numel() * 8
    st = pcz.compress(x, tau)
    st.close()
    reps = 2
    pcz.timing_enable(True)
    holder = {}

    def comp():
        if "st" in holder:
            holder.pop("st").close()
        holder["st"] = pcz.compress(x, tau)

    ms_c = timed_events(comp, reps)
    kt = pcz.timing_read()
    st = holder["st"]
    buf = torch.empty_like(x)

    def sweep():
        st.retrieve(k=1, out=buf)
        for k in range(2, n + 1):
            st.refine(k - 1, k, buf)

    ms_s = timed_events(sweep, reps)
    kt2 = pcz.timing_read()
    pcz.timing_enable(False)
    eq1 = []
    for k in (1, 6, 12):
        st.retrieve(k=k, out=buf)
        eq1.append(float((x - buf).abs().max().item()) <= tau[k - 1])
    hbm, _ = peaks()
    cb, rb, pay = algorithmic_bytes(st, fb)
    k_comp_ms = kt["compress"][0] / max(kt["compress"][1], 1)
    # sweep bytes: every component read once, x~ read and written per refinement
    sweep_bytes = sum(pay) + n * (st.info(0)[2]) + fb + (n - 1) * 2 * fb
    k_sweep_ms = kt2["retrieve"][0] - kt["retrieve"][0]
    del buf
    # the mixed-tolerance query stream: brick-aligned boxes with sides log-uniform
    # in [8, 512], relative tolerance log-uniform in [1e-12, 1e-1], Poisson arrivals
    rng = np.random.default_rng(np.random.PCG64(55))
    nq = args.c5_queries
    arr = np.cumsum(rng.exponential(1.0 / 1000.0, nq))
    arr -= arr[0]
    lo_v, hi_v = pcz.field_range(x)
    qs = []
    for _ in range(nq):
        lo, hi = [], []
        for _a in range(3):
            side = min(max(4 * int(round(np.exp(rng.uniform(np.log(8.0), np.log(512.0))) / 4.0)), 8), size)
            o = 4 * int(rng.integers(0, (size - side) // 4 + 1))
            lo.append(o)
            hi.append(o + side)
        qs.append((0, (lo, hi), 10.0 ** rng.uniform(-12.0, -1.0) * (hi_v - lo_v), 0))
    del x
    torch.cuda.empty_cache()
    serve = {}
    for name, kw in (("batched", {"max_batch": 256}), ("plain", {"serial": True, "cache": False})):
        srv = pcz.Server(64 * 10 ** 9, **kw)
        srv.add_field(st)
        srv.replay(qs[:16], [0.0] * 16)
        srv.reset_cache()
        lat, stats = srv.replay(qs, arr.tolist())
        srv.close()
        lat_ms = 1e3 * lat
        serve[name] = {"p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
                       "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
                       "throughput_qps": round(stats["queries"] / stats["wall_s"], 1),
                       "gbs_out": round(stats["bytes_out"] / stats["wall_s"] / 1e9, 3),
                       "mean_batch": round(stats["queries"] / max(stats["batches"], 1), 2)}
    st.close()
    torch.cuda.empty_cache()
    # the oracle on corners of the same field, extrapolated per brick: one core
    # on 64^3, all cores on 128^3
    oc = {}
    for cores, corner in ((1, xs64), (nthreads, xs128)):
        sub = corner.shape[0]
        t = time.perf_counter()
        s = O.Streams(corner, tau, nthreads=cores)
        secs_c = time.perf_counter() - t
        t = time.perf_counter()
        xk = s.retrieve(1)
        for k in range(2, n + 1):
            xk = s.retrieve(k, k0=k - 1, inout=xk)
        secs_s = time.perf_counter() - t
        scale = (size / sub) ** 3
        oc[cores] = {"compress_gbs": round(corner.nbytes / secs_c / 1e9, 5),
                     "sweep_gbs": round(n * corner.nbytes / secs_s / 1e9, 5), "cores": cores,
                     "sample": f"{sub}^3 corner, extrapolated x{scale:.0f} by bricks",
                     "compress_s_extrapolated": round(secs_c * scale, 1),
                     "sweep_s_extrapolated": round(secs_s * scale, 1)}
    return {"workload": f"{size}^3 float64 k^-5/3 field + 24 tanh fronts, 12 components, tau_i = 10^-i range",
            "compress": {"ms": round(ms_c, 3), "gbs": round(fb / (ms_c * 1e-3) / 1e9, 2),
                         "kernel_ms": round(k_comp_ms, 3),
                         "roofline_frac_kernel": round(cb / (k_comp_ms * 1e-3) / 1e9 / hbm, 5)},
            "progressive_sweep": {"ms": round(ms_s, 3), "gbs_out": round(n * fb / (ms_s * 1e-3) / 1e9, 2),
                                  "kernel_ms": round(k_sweep_ms / reps, 3),
                                  "roofline_frac_kernels": round(sweep_bytes / (k_sweep_ms / reps * 1e-3) / 1e9 / hbm, 5)},
            "eq1_holds_k1_k6_k12": eq1,
            "rates_bits_per_value": [round(8 * p / (fb / 8), 4) for p in pay],
            "query_stream": dict(serve, queries=nq, rate_per_s=1000,
                                 boxes="brick-aligned, sides log-uniform in [8, 512]",
                                 tolerance="relative, log-uniform in [1e-12, 1e-1]"),
            "oracle_single_core": oc[1], "oracle_all_cores": oc[nthreads]}


def oracle_sample(fields_np, sub, nthreads, per_dtype=None):
    """Times the CPU oracle on a sub^3 corner of each field: Algorithm 1 then
    Algorithm 2 at every k.  Returns (GB/s of raw bytes, seconds, description);
    per_dtype, if a dict, receives each field's compress and retrieval GB/s."""
    import oracle as O

    total_bytes = 0
    t = time.perf_counter()
    for name, x in fields_np.items():
        xs = np.ascontiguousarray(x[:sub, :sub, :sub])
        tau = O.tau_decade(O.value_range(xs), N_COMP)
        a = time.perf_counter()
        s = O.Streams(xs, tau, nthreads=nthreads)
        b = time.perf_counter()
        for k in range(1, N_COMP + 1):
            s.retrieve(O.query_k(tau, tau[k - 1]))
        c = time.perf_counter()
        total_bytes += xs.nbytes * (1 + N_COMP)
        if per_dtype is not None:
            per_dtype[name] = {"compress_gbs": round(xs.nbytes / (b - a) / 1e9, 5),
                               "retrieve_gbs": round(N_COMP * xs.nbytes / (c - b) / 1e9, 5)}
    secs = time.perf_counter() - t
    desc = f"{sub}^3 corner of each field (f32 and f64), compress + retrieval at every k"
    return total_bytes / secs / 1e9, secs, desc


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pcz", choices=["pcz", "reference"])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--sample", type=int, default=128, help="edge of the oracle's sample sub-volume")
    ap.add_argument("--dtypes", default="f32,f64", help="field types in a step (profiling runs use one)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-lossless", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--serve-queries", type=int, default=10000)
    ap.add_argument("--serve-size", type=int, default=256)
    ap.add_argument("--no-configs", action="store_true", help="skip the 64^3 and 1024^3 configuration legs")
    ap.add_argument("--no-use-case", action="store_true", help="skip the derivatives-of-reconstructions leg")
    ap.add_argument("--kernel-reps", type=int, default=20, help="launches per median in the per-type kernel times")
    ap.add_argument("--c5-size", type=int, default=1024)
    ap.add_argument("--c5-queries", type=int, default=2000)
    args = ap.parse_args()
    rank, world, local = dist_setup()
    nthreads = os.cpu_count() or 1

    if args.impl == "reference":
        if rank != 0:
            return
        import synth_fields as S

        x64 = S.powerlaw((args.sample, args.sample, args.sample), seed=2, dtype=np.float64)
        fields_np = {"f32": x64.astype(np.float32), "f64": x64}
        for _ in range(args.warmup):
            oracle_sample(fields_np, args.sample, nthreads)
        vals, secs = [], 0.0
        for _ in range(args.steps):
            v, s, desc = oracle_sample(fields_np, args.sample, nthreads)
            vals.append(v)
            secs += s
        value = float(np.mean(vals))
        line = {"impl": "reference", "metric": METRIC, "value": round(value, 5),
                "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1e3 * secs / args.steps, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32,f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "parallelism": "replicas", "reference_sample": desc},
                "cpu_baseline": {"value": round(value, 5), "unit": "GB/s", "cores": nthreads, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": round(value, 5), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch

    if world > 1:
        torch.distributed.init_process_group("nccl")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    r = run_pcz(args, rank, world, device)
    serving = None
    if not args.no_serving:
        r["fields"] = {k: v[: args.sample, : args.sample, : args.sample].cpu() for k, v in r["fields"].items()}
        torch.cuda.empty_cache()
        serving = run_serving(args, device)
    lossless = None if args.no_lossless else run_lossless(device)
    configs = None
    if not args.no_configs:
        configs = {"c1_64cube_f64": run_config1(args, device, nthreads),
                   "c5_1024cube_f64_fronts": run_config5(args, device, nthreads)}
    batched = None if args.no_batched else run_batched(args, device)
    use_case = None if args.no_use_case else run_use_case(args, device)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fields_np = {k: v[: args.sample, : args.sample, : args.sample].cpu().numpy() for k, v in r["fields"].items()}
        pdN, pd1 = {}, {}
        v, s, desc = oracle_sample(fields_np, args.sample, nthreads, pdN)
        cpu = {"value": round(v, 5), "unit": "GB/s", "cores": nthreads, "kind": "oracle", "sample": desc,
               "seconds": round(s, 2), "per_dtype": pdN}
        # the paper's own mode: one core, on a smaller corner of the same fields
        sub1 = max(4, args.sample // 2)
        v1, s1, desc1 = oracle_sample(fields_np, sub1, 1, pd1)
        cpu["single_core"] = {"value": round(v1, 5), "unit": "GB/s", "cores": 1, "sample": desc1,
                              "seconds": round(s1, 2), "per_dtype": pd1}
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(r["value"], 3),
            "unit": "GB/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(r["ms_step"], 3),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32,f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "size": args.size, "components": N_COMP,
                       "inputs_exceed_l2": True, "l2_flush": False, "parallelism": "replicas"},
            "e2e": r["e2e"],
            "roofline": r["roofline"],
            "pipe_utilisation": PIPES,
            "cpu_baseline": cpu,
            "clocks": r["clocks"],
            "gpu_launches": r["launches"],
            "kernels": r["kernels"],
            "per_dtype": r["per_dtype"],
            "rates_bits_per_value": {k: v["rates"] for k, v in r["info"].items()},
            "computed_tolerances": {k: v["measured_over_tau"] for k, v in r["info"].items()},
            "accuracy_gain": r["gain"],
            "progressive_sweep": dict(r["sweep"], note="retrieve k=1 then refine k-1 -> k in place, k = 2..%d; "
                                      "outside the timed step, not part of value" % N_COMP),
            "lossless": lossless,
            "configurations": configs,
            "batched": batched,
            "serving": serving,
            "use_case_derivatives": use_case,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
