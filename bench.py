#!/usr/bin/env python3
"""Benchmark of the PLV / iPLV / ciPLV hot path on one or more GB300s.

One step = the whole hot path over one batch: analytic signal + unit phasors
(K1) and the Hermitian Gram with the fused read-outs (Gram kernel) for every
epoch of the workload, inputs already resident in HBM.  Prints ONE JSON line.

Workload (default): N = 8192 sources, T = 8192 samples, 20 epochs of
band-limited (8-12 Hz, 4th-order Butterworth, fs = 1000 Hz) noise with 5 % of
pairs coupled at 5-40 ms lags and 20 % of channels as zero-lag leakage
mixtures -- synthetic stand-in for whole-brain MEG source-space data -- on
the BF16x3 split-precision tensor-core Gram, with the plain FP32 path timed
on the same input beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P]
  python bench.py --impl reference      # FP64 CPU oracle on a sample

Multi-GPU: epochs are independent problems; every rank runs its own copy of
the workload on its own GPU (weak scaling, no collective on the data path).
``--gpus N`` without a process group spawns the N ranks itself (one process
per GPU, torch.distributed.run on 127.0.0.1).
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

METRIC = ("channel-pair·samples/s (N²T/s) for PLV+ciPLV, % tensor "
          "peak, vs FP32 at stated error")
UNIT = "channel-pair·samples/s"

WORKLOADS = {
    # name: (E, N, T, seed)
    "bandlimited-N4096-T4096-E30": (30, 4096, 4096, 1002),
    "bandlimited-N8192-T8192-E20": (20, 8192, 8192, 1003),
    # small cases of the two, for ncu captures (still larger than L2)
    "bandlimited-N4096-T4096-E4": (4, 4096, 4096, 1002),
    "bandlimited-N8192-T8192-E2": (2, 8192, 8192, 1003),
}
DEFAULT_WORKLOAD = "bandlimited-N8192-T8192-E20"
# uneven batch: 256 subjects, N ~ U{68..2000}, T ~ U{500..10000} per subject,
# 5 frequency bands each (1280 problems of one epoch), fs = 1000 Hz
GROUPED = "grouped-256subj-5bands-N68to2000-T500to10000"
# differentiable loss: 16 recordings, N = 1024, T = 4096, loss = sum of ciPLV
# over a seeded 10 % pair mask; forward + hand-written backward per step
BACKWARD = "backward-ciplv-loss-B16-N1024-T4096"
BANDS = [(4.0, 8.0), (8.0, 12.0), (13.0, 30.0), (30.0, 45.0), (55.0, 80.0)]


def max_over_ranks(value, dist=None, device=None):
    """The largest of every rank's value (for times: the slowest rank), or
    the value itself without a process group."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_per_step):
    """Whole-job throughput: the units all ranks processed per second of the
    slowest rank's step time."""
    return units_per_rank * world / (ms_per_step / 1e3)


def rank_seed(seed, rank):
    """Each replica generates its own input: the workload's seed plus its
    rank."""
    return seed + rank


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,"
         "clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        """Start sampling and wait (at most 3 s) until the sampler runs, so
        that even a short timed region gets a sample."""
        self.first = 0
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.01)
            self.first = len(self.lines)  # samples before the timed region
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        # at least one sample taken from the timed region on (at most 1 s)
        t0 = time.time()
        while len(self.lines) <= self.first and time.time() - t0 < 1.0:
            time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines[self.first:] or self.lines[-1:]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


# DRAM traffic per launch of the dominant kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of a smaller case of the same
# N and T, scaled to the timed launch by epochs (the Gram's traffic is per
# epoch: its tiles never span epochs).  Keyed by kernel, workload and
# precision; an entry is removed when the kernel changes after its capture.
TRAFFIC = {
    # k_gram_tc on bandlimited-N8192-T8192-E2 (super-block raster of width 8,
    # MMA width per tile, collector-buffer A reuse, 1024-sample summation
    # chunks), read + write of its 4th launch, scaled by 20 / 2 epochs
    ("k_gram_tc", "bandlimited-N8192-T8192-E20", "bf16x3"): (9.401593344e9 + 2.281091840e9) * 10,
}


def workload_config(workload, N, T, E, prec, world, in_bytes=4):
    """The ``config`` object of a bench line for the N x N x T x E workload:
    the same dict in both arms, so that they name the same job."""
    return {"workload": workload, "N": N, "T": T, "epochs_per_gpu": E,
            "precision": prec, "input_dtype": "f32",
            "l2": "inputs larger than L2 (x %.1f GB, phasors %.1f GB, "
                  "outputs %.1f GB per step)" % (
                      E * N * T * in_bytes / 1e9, E * N * T * 8 / 1e9,
                      3 * E * N * N * 4 / 1e9),
            "parallelism": f"weak: {world} independent replicas"}


def gram_flops(N, T, E, prec):
    """Algorithmic flops of the Gram per launch: 8 real flops per complex MAC
    over the N(N+1)/2 upper-triangle pairs, times 3 for the hi/lo split."""
    f = 8.0 * (N * (N + 1) / 2) * T * E
    return f * (3.0 if prec in ("bf16x3", "fp16x3") else 1.0)


def k1_bytes(N, T, E, in_bytes=4):
    """Algorithmic HBM bytes of K1: read x once, write 8 B of phasor per
    sample (padding excluded)."""
    return float(E) * N * T * (in_bytes + 8)


def run_ours(args):
    import torch
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    E, N, T, seed = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)
    h = plv.Handle(precision=args.precision, device=local)
    x = synth.bandlimited(E, N, T, seed=rank_seed(seed, rank), device=dev)
    P = h.empty_phasors(E, N, T)
    out = {k: torch.empty((E, N, N), dtype=torch.float32, device=dev)
           for k in ("plv", "iplv", "ciplv")}
    s = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(evs=None):
        if evs:
            evs[0].record(s)
        h.plv_analytic(x, P)
        if evs:
            evs[1].record(s)
        h.plv_gram(P, E, N, T, out=out)
        if evs:
            evs[2].record(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    t0, t1 = ev(), ev()
    per = [[ev(), ev(), ev()] for _ in range(args.steps)]
    t0.record(s)
    for k in range(args.steps):
        step(per[k])
    t1.record(s)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    k1_ms = statistics.mean(p[0].elapsed_time(p[1]) for p in per)
    gram_ms = statistics.mean(p[1].elapsed_time(p[2]) for p in per)
    ms = max_over_ranks(ms, dist, dev)
    ms_step = ms / args.steps
    units = float(N) * N * T * E  # channel-pair x samples per step per rank
    value = job_value(units, world, ms_step)
    device_status = h.plv_sync_status()

    # end to end through the C ABI: host x -> device, path, outputs -> host.
    # The epochs go in chunks on two streams, so one chunk's copies overlap
    # another chunk's kernels (every byte still crosses inside the timed
    # region, every step).  Chunk c of every step runs on the same stream,
    # so the stream's order keeps each reused buffer's uses apart, and steps
    # follow each other without a join: the next step's uploads overlap this
    # step's last downloads, as in a stream of recordings.
    e2e = None
    e2e_buffers = None
    if not args.no_e2e:
        xh = x.cpu().pin_memory()
        oh = {k: torch.empty((E, N, N), dtype=torch.float32).pin_memory()
              for k in out}
        xd = torch.empty_like(x)
        nch = max(1, min(E, args.e2e_chunks))
        bounds = [(E * c // nch, E * (c + 1) // nch) for c in range(nch)]
        streams = [torch.cuda.Stream(dev) for _ in range(max(1, args.e2e_streams))]
        Ps = [h.empty_phasors(max(b - a for a, b in bounds), N, T) for _ in streams]

        def e2e_step():
            for c, (a, b) in enumerate(bounds):
                k = c % len(streams)
                with torch.cuda.stream(streams[k]):
                    xd[a:b].copy_(xh[a:b], non_blocking=True)
                    h.plv_analytic(xd[a:b], Ps[k])
                    h.plv_gram(Ps[k], b - a, N, T,
                               out={kk: v[a:b] for kk, v in out.items()})
                    for kk in out:
                        oh[kk][a:b].copy_(out[kk][a:b], non_blocking=True)

        def join():
            for st_ in streams:
                s.wait_stream(st_)

        for st_ in streams:
            st_.wait_stream(s)
        for _ in range(max(1, min(args.warmup, 2))):
            e2e_step()
        join()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        a_, b_ = ev(), ev()
        a_.record(s)
        for st_ in streams:
            st_.wait_stream(s)
        marks = []
        for _ in range(args.steps):
            e2e_step()
            m_ = ev()
            m_.record(streams[(nch - 1) % len(streams)])  # after the step's last download
            marks.append(m_)
        join()
        b_.record(s)
        torch.cuda.synchronize(dev)
        gaps = [a_.elapsed_time(marks[0])] + [marks[i - 1].elapsed_time(marks[i])
                                              for i in range(1, len(marks))]
        ems = a_.elapsed_time(b_)
        ems = max_over_ranks(ems, dist, dev)
        e2e_buffers = (xh, oh, xd, Ps)
        del xh, oh, xd, Ps
        e2e = {"value": job_value(units, world, ems / args.steps), "unit": UNIT,
               "h2d_bytes_per_step": int(x.numel() * x.element_size()),
               "d2h_bytes_per_step": int(sum(v.numel() * 4 for v in out.values())),
               "ms_per_step": ems / args.steps,
               "pipeline": f"{nch} epoch chunks on {len(streams)} streams, steps not joined",
               "step_ms": {"min": min(gaps), "median": statistics.median(gaps),
                           "max": max(gaps)}}

    # sampled outputs of epoch 0 for the comparison with the FP64 oracle
    sub = sample_channels(N, seed, args.cpu_sample)
    sub_t = torch.as_tensor(sub, device=dev)

    def sampled(o):
        return {k: o[k][0].index_select(0, sub_t).index_select(1, sub_t)
                .double().cpu().numpy() for k in ("plv", "iplv", "ciplv")}

    samp = {args.precision: sampled(out)}

    # the plain FP32 path on the same input: time and agreement
    fp32 = None
    if args.precision != "fp32" and not args.no_fp32_compare:
        h32 = plv.Handle(precision="fp32", device=local)
        out32 = {k: torch.empty_like(v) for k, v in out.items()}
        P32 = h32.empty_phasors(E, N, T)

        def step32():
            h32.plv_analytic(x, P32)
            h32.plv_gram(P32, E, N, T, out=out32)

        step32()
        torch.cuda.synchronize(dev)
        n32 = max(1, min(args.steps, 3))
        a, b = ev(), ev()
        a.record(s)
        for _ in range(n32):
            step32()
        b.record(s)
        torch.cuda.synchronize(dev)
        ms32 = a.elapsed_time(b) / n32
        step()  # refresh the split-precision outputs for the comparison
        torch.cuda.synchronize(dev)
        agree = {k: float((out[k] - out32[k]).abs().max()) for k in out}
        samp["fp32"] = sampled(out32)
        fp32 = {"ms_per_step": ms32, "value": job_value(units, world, ms32),
                "speedup_of_split_path": ms32 / ms_step,
                "max_abs_diff_vs_split_path": agree, "steps": n32}
        del out32, P32
        h32.close()

    peaks, peak_kind = _peaks()
    prec = args.precision
    flops = gram_flops(N, T, E, prec)
    # the Gram runs inside a timed region of back-to-back steps; beyond about
    # a second of it the power cap sets the clock, which the sustained peak
    # (a seconds-long cuBLAS loop) is measured under
    timed_s = ms / 1e3
    sustained = args.peak == "sustained" or (args.peak == "auto" and timed_s >= 1.0)
    if prec == "fp32":
        # plain-ALU bound: FP32 FMA pipes, 152 SMs x 128 lanes x 2 flop x clock
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": "k_gram_fp32",
                "achieved": flops / (gram_ms / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s",
                "peak_source": f"derived: 152 SMs x 128 FP32 FMA/clk x 2 x "
                               f"{sm_mhz:.0f} MHz (max SM clock, {peak_kind})"}
    else:
        burst = float(peaks["bf16_tflops"])
        peak = float(peaks["bf16_tflops_sustained"]) if sustained else burst
        roof = {"bound": "tensor", "kernel": "k_gram_tc",
                "achieved": flops / (gram_ms / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s",
                "peak_source": f"{peak_kind} bf16 dense "
                               f"({'sustained: the Gram is timed inside %.1f s of back-to-back steps' % timed_s if sustained else 'burst'})",
                "frac_of_burst": flops / (gram_ms / 1e3) / 1e12 / burst}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TRAFFIC.get((roof["kernel"], args.workload, prec))
    roof["launch_ms"] = gram_ms
    roof["flops_per_launch"] = flops
    roof["algorithmic_bytes_per_launch"] = E * N * T * 8.0 + 3 * 4.0 * E * N * N
    k1b = k1_bytes(N, T, E, x.element_size())
    k1 = {"kernel": "k_hilbert_pairs", "bound": "hbm", "launch_ms": k1_ms,
          "achieved": k1b / (k1_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
          "unit": "GB/s", "bytes_per_launch": k1b}
    k1["frac"] = k1["achieved"] / k1["peak"]

    # device memory high-water mark of the run (the analogue of the paper's
    # RAM column): caller-owned tensors (torch) plus the handle's own
    hcur, hpeak = h.memory_usage()
    mem = {"torch_peak_bytes": int(torch.cuda.max_memory_allocated(dev)),
           "library_peak_bytes": hpeak,
           "note": "torch peak covers inputs, phasors, outputs and the end-to-end and FP32 "
                   "legs' buffers; library peak is the handle's tables and plans"}

    cpu = None
    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        ref = {}
        cpu = cpu_baseline(E, N, T, seed, args.cpu_sample, x=x, values=ref)
        accuracy = oracle_errors(samp, ref, len(sub), N)

    # the uneven-batch workload (256 subjects x 5 bands, one grouped plan
    # under CUDA graphs), measured after the main workload's buffers are freed
    in_bytes = x.element_size()
    grouped = None
    configs = None
    if not args.no_grouped or not args.no_configs:
        del x, P, out, e2e_buffers
        torch.cuda.empty_cache()
    if not args.no_grouped:
        grouped = grouped_measure(args, dev, dist, rank, world)
    if not args.no_configs:
        # the other configurations of the same job, each in its own launch
        # configuration, so one line carries every workload the metric names
        configs = {"fp32-N4096-T4096-E30": fp32_workload_measure(args, dev, dist, rank, world),
                   BACKWARD: backward_measure(args, dev, dist, rank, world)}
        if rank == 0:
            configs["tones-N64-T2048"] = parity_measure(args, dev)
            configs["grouped-small-N-long-T"] = split_k_measure(args, dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16x3": "bf16x3 (bf16 products, f32 "
                      "accumulate)", "fp16x3": "fp16x3 (fp16 products, f32 "
                      "accumulate)"}[prec],
            "data": "synthetic (seeded band-limited noise, coupled pairs, "
                    "leakage mixtures; MEG recording not available)",
            "config": workload_config(args.workload, N, T, E, prec, world, in_bytes),
            "roofline": roof,
            "k1_roofline": k1,
            "cpu_baseline": cpu,
            "accuracy_vs_oracle": accuracy,
            "fp32_path": fp32,
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,
            "clocks": clk,
            "device_status": device_status,
            "device_memory": mem,
            "grouped": grouped,
            "configs": configs,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


def grouped_problems(seed=1004, nsub=256):
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for sj in range(nsub):
        N = int(rng.integers(68, 2001))
        T = int(rng.integers(500, 10001))
        for b, band in enumerate(BANDS):
            out.append((N, T, band, seed * 10000 + sj * 5 + b))
    return out


def _conv_M(T):
    """Transform length of the any-length engine for T: the smallest 2^a,
    3 2^a or 5 2^a (>= 32) that is >= 2T - 1."""
    need, best, p = 2 * T - 1, None, 32
    while p <= 24576:
        for m in (p, 3 * p, 5 * p):
            if m >= need and m <= 24576 and (best is None or m < best):
                best = m
        p *= 2
    return best


def grouped_measure(args, dev, dist, rank, world):
    """The uneven batch on one plan: per step, the grouped phasor launches
    (one persistent launch per thread class of the any-length engine, one
    CUDA graph) and the grouped Gram (one persistent launch, a second graph),
    inputs resident in HBM.  Returns the measurement as a dict."""
    import torch
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    h = plv.Handle(precision=args.precision, device=dev.index)
    specs = grouped_problems(seed=rank_seed(1004, rank), nsub=args.subjects)
    t_gen = time.perf_counter()
    probs = []
    for (N, T, band, sd) in specs:
        x = synth.bandlimited(1, N, T, seed=sd, band=band, device=dev)
        h.prepare(T)
        probs.append({"x": x, "P": h.empty_phasors(1, N, T), "batch": 1,
                      "N": N, "T": T})
    t_gen = time.perf_counter() - t_gen
    grp = h.plv_group_create(probs)
    s = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)

    def k1_all():
        h.plv_analytic_grouped(grp)

    with torch.cuda.stream(s):
        k1_all()
        h.plv_gram_grouped(grp)
    torch.cuda.synchronize(dev)
    # launch shapes picked by the library's autotuner (timed on the plan's
    # own buffers, outside the timed region)
    tune = None
    if not args.no_tune:
        t_tune = time.perf_counter()
        with torch.cuda.stream(s):
            tune = h.plv_group_tune(grp, reps=3)
        torch.cuda.synchronize(dev)
        tune["seconds"] = time.perf_counter() - t_tune
    g1, g2 = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g1, stream=s):
            k1_all()
        with torch.cuda.graph(g2, stream=s):
            h.plv_gram_grouped(grp)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            g1.replay()
            g2.replay()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        clocks = ClockSampler(dev.index)
        clocks.start()
        per = [[ev(), ev(), ev()] for _ in range(args.steps)]
        for p in per:
            p[0].record(s)
            g1.replay()
            p[1].record(s)
            g2.replay()
            p[2].record(s)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
    ms = sum(p[0].elapsed_time(p[2]) for p in per)
    k1_ms = statistics.mean(p[0].elapsed_time(p[1]) for p in per)
    gram_ms = statistics.mean(p[1].elapsed_time(p[2]) for p in per)
    ms = max_over_ranks(ms, dist, dev)
    ms_step = ms / args.steps
    units = float(sum(N * N * T for (N, T, _, _) in specs))
    value = job_value(units, world, ms_step)
    flops = sum(gram_flops(N, T, 1, args.precision) for (N, T, _, _) in specs)
    # the executed tensor work: 128-row tiles, columns rounded to 16
    exe = 0.0
    for (N, T, _, _) in specs:
        nrb = (N + 127) // 128
        ld = (T + 31) // 32 * 32
        for J in range(nrb):
            w = min(128, ((min(128, N - 128 * J) + 15) // 16) * 16)
            exe += (J + 1) * 128 * w * ld * 8.0 * 3
    peaks, peak_kind = _peaks()
    peak = float(peaks["bf16_tflops"])
    roof = {"bound": "tensor", "kernel": "k_gram_tc (grouped, one launch)",
            "achieved": flops / (gram_ms / 1e3) / 1e12, "peak": peak,
            "unit": "TFLOP/s", "peak_source": f"{peak_kind} bf16 dense (burst)",
            "traffic": None, "launch_ms": gram_ms,
            "executed_tile_flops": exe,
            "executed_frac": exe / (gram_ms / 1e3) / 1e12 / peak}
    roof["frac"] = roof["achieved"] / roof["peak"]
    k1b = sum(N * T * 12 for (N, T, _, _) in specs)
    k1_launches = (tune["k1_launches"] if tune else
                   len({min(3, max(0, (_conv_M(T) > 3072) + (_conv_M(T) > 6144)
                                   + (_conv_M(T) > 12288))) for (_, T, _, _) in specs}))
    device_status = h.plv_sync_status()
    out = {"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms_step,
           "config": {"workload": GROUPED, "problems": len(specs),
                      "sum_N2T": units, "precision": args.precision,
                      "graphs": "grouped phasor launches in one CUDA graph, "
                                "grouped Gram in another",
                      "autotune": tune, "generation_s": t_gen},
           "roofline": roof,
           "k1": {"launches": k1_launches, "ms": k1_ms,
                  "algorithmic_GBps": k1b / (k1_ms / 1e3) / 1e9,
                  "frac_of_hbm": k1b / (k1_ms / 1e3) / 1e9 / float(peaks["hbm_gbs"])},
           "gpu_launches": (k1_launches + 1) * args.steps,
           "clocks": clk, "device_status": device_status}
    grp.close()
    h.close()
    del probs
    torch.cuda.empty_cache()
    return out


def split_k_measure(args, dev, nsub=8):
    """The corner of the uneven batch where few long tiles leave the grid
    idle: nsub subjects with N in 68..300 and T in 5000..10000, five bands
    each, on one grouped plan.  Times the grouped Gram (CUDA events, inputs
    resident) unsplit and with each split-K factor, and what the autotuner
    keeps; reports the largest output difference split vs unsplit."""
    import numpy as np
    import torch
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    if args.precision == "fp32":
        return None
    h = plv.Handle(precision=args.precision, device=dev.index)
    rng = np.random.default_rng(1014)
    specs = []
    for sj in range(nsub):
        N, T = int(rng.integers(68, 301)), int(rng.integers(5000, 10001))
        for b, band in enumerate(BANDS):
            specs.append((N, T, band, 1014 * 1000 + sj * 5 + b))
    probs = []
    for (N, T, band, sd) in specs:
        x = synth.bandlimited(1, N, T, seed=sd, band=band, device=dev)
        h.prepare(T)
        probs.append({"x": x, "P": h.empty_phasors(1, N, T), "batch": 1, "N": N, "T": T})
    grp = h.plv_group_create(probs)
    s = torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(reps=20):
        with torch.cuda.stream(s):
            for _ in range(3):
                h.plv_gram_grouped(grp)
            a, b = ev(), ev()
            a.record(s)
            for _ in range(reps):
                h.plv_gram_grouped(grp)
            b.record(s)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    with torch.cuda.stream(s):
        h.plv_analytic_grouped(grp)
    times = {}
    for f in (0, 1, 2, 4):
        with torch.cuda.stream(s):
            h.plv_group_configure(grp, gram_split=f)
        times[f] = timed()
        if f == 0:
            ref = [q["plv"].clone() for q in probs]
    diff = max(float((q["plv"] - r).abs().max()) for q, r in zip(probs, ref))
    with torch.cuda.stream(s):
        h.plv_group_configure(grp)
        tune = h.plv_group_tune(grp, reps=3)
    tuned = timed()
    units = float(sum(N * N * T for (N, T, _, _) in specs))
    out = {"metric": METRIC, "value": units / (tuned / 1e3), "unit": UNIT,
           "ms_per_step": tuned,
           "config": {"workload": "grouped-small-N-long-T", "problems": len(specs),
                      "N": "68..300", "T": "5000..10000", "precision": args.precision,
                      "what": "the grouped Gram alone (phasors resident)"},
           "gram_ms_by_split_factor": {str(f): v for f, v in times.items()},
           "speedup_of_tuned_over_unsplit": times[0] / tuned,
           "autotune": {k: tune[k] for k in ("gram_schedule", "gram_tile_cost", "gram_split",
                                             "gram_split_tiles", "gram_ms_default",
                                             "gram_ms_tuned")},
           "max_abs_plv_diff_split_vs_unsplit": diff,
           "gpu_launches": 1, "device_status": h.plv_sync_status()}
    grp.close()
    h.close()
    del probs
    torch.cuda.empty_cache()
    return out


def parity_measure(args, dev):
    """The parity workload (64 channels, T = 2048, fs = 512 Hz tones, FP64
    input, one epoch): the whole path on the GPU in FP32 and BF16x3 (CUDA
    events), and the full FP64 oracle (every row's direct-DFT analytic
    signal, the pairwise loop over all 64^2 pairs, no sampling) on the host
    cores, with each GPU path's largest error per metric against it."""
    import numpy as np
    import torch
    import oracle
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    x, _ = synth.tones(seed=1001)
    E, N, T = x.shape
    t0 = time.perf_counter()
    ref = oracle.connectivity(x[0])
    t_oracle = time.perf_counter() - t0
    units = float(N) * N * T
    rec = {"workload": f"tones-N{N}-T{T}-E{E} (FP64 input, 16 lagged pairs, 8 zero-lag "
                       f"mixtures, noise 0.5)",
           "oracle": {"seconds": t_oracle, "value": units / t_oracle, "unit": UNIT,
                      "cores": oracle.threads(),
                      "what": "full oracle: direct-DFT analytic signal of every row, pairwise "
                              "loop over all ordered pairs"}}
    xd = torch.tensor(x, device=dev)
    c = ref["c"]
    d = np.maximum((1 - c.real) * (1 + c.real), 1e-12)
    for prec, tol in (("fp32", 1e-5), ("bf16x3", 2e-5)):
        h = plv.Handle(precision=prec, device=dev.index)
        P = h.empty_phasors(E, N, T)
        out = {k: torch.empty((E, N, N), dtype=torch.float32, device=dev)
               for k in ("plv", "iplv", "ciplv")}
        s = torch.cuda.current_stream(dev)

        def step():
            h.plv_analytic(xd, P)
            h.plv_gram(P, E, N, T, out=out)

        for _ in range(max(3, args.warmup)):
            step()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(args.steps):
            step()
        b.record(s)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / args.steps
        got = {k: v[0].double().cpu().numpy() for k, v in out.items()}
        bound = tol / np.sqrt(d) + np.abs(c.imag * c.real) * tol / d ** 1.5 + 1e-6
        ce = np.abs(got["ciplv"] - ref["ciplv"])
        rec[prec] = {"ms_per_step": ms, "value": units / (ms / 1e3),
                     "speedup_vs_oracle": t_oracle / (ms / 1e3),
                     "max_abs_err": {k: float(np.abs(got[k] - ref[k]).max())
                                     for k in ("plv", "iplv", "ciplv")},
                     "ciplv_within_conditioned_bound": bool(np.all(ce <= bound)),
                     "bound_plv_iplv": tol}
        h.close()
    return rec


def fp32_workload_measure(args, dev, dist, rank, world):
    """The plain FP32 workload: N = T = 4096, 30 epochs, analytic signal and
    the CUDA-core Gram with fused read-outs (the same generator as the
    headline); per-metric error against the FP64 oracle on a 128-channel
    sample of epoch 0 (rank 0)."""
    import torch
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    wl = "bandlimited-N4096-T4096-E30"
    E, N, T, seed = WORKLOADS[wl]
    h = plv.Handle(precision="fp32", device=dev.index)
    x = synth.bandlimited(E, N, T, seed=rank_seed(seed, rank), device=dev)
    P = h.empty_phasors(E, N, T)
    out = {k: torch.empty((E, N, N), dtype=torch.float32, device=dev)
           for k in ("plv", "iplv", "ciplv")}
    s = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(e=None):
        if e:
            e[0].record(s)
        h.plv_analytic(x, P)
        if e:
            e[1].record(s)
        h.plv_gram(P, E, N, T, out=out)
        if e:
            e[2].record(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    per = [[ev(), ev(), ev()] for _ in range(args.steps)]
    for p_ in per:
        step(p_)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(sum(p_[0].elapsed_time(p_[2]) for p_ in per), dist, dev)
    k1_ms = statistics.mean(p_[0].elapsed_time(p_[1]) for p_ in per)
    k2_ms = statistics.mean(p_[1].elapsed_time(p_[2]) for p_ in per)
    ms_step = ms / args.steps
    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    flops = gram_flops(N, T, E, "fp32")
    rec = {"workload": wl, "value": job_value(float(N) * N * T * E, world, ms_step),
           "unit": UNIT, "ms_per_step": ms_step,
           "roofline": {"bound": "alu", "kernel": "k_gram_fp32", "launch_ms": k2_ms,
                        "achieved": flops / (k2_ms / 1e3) / 1e12, "peak": alu_peak,
                        "unit": "TFLOP/s", "frac": flops / (k2_ms / 1e3) / 1e12 / alu_peak,
                        "peak_source": f"derived: 152 SMs x 128 FP32 FMA/clk x 2 x {sm_mhz:.0f} MHz"},
           "k1_ms": k1_ms,
           "k1_frac_of_hbm": k1_bytes(N, T, E) / (k1_ms / 1e3) / 1e9 / float(peaks["hbm_gbs"])}
    if rank == 0 and not args.no_cpu_baseline:
        sub = sample_channels(N, seed, 128)
        ref, _, _, _ = oracle_step(x[0], sub)
        sub_t = torch.as_tensor(sub, device=dev)
        got = {k: out[k][0].index_select(0, sub_t).index_select(1, sub_t).double().cpu().numpy()
               for k in ("plv", "iplv", "ciplv")}
        rec["accuracy_vs_oracle"] = oracle_errors({"fp32": got}, ref, len(sub), N)
    h.close()
    del x, P, out
    torch.cuda.empty_cache()
    return rec


def run_grouped(args):
    """The uneven batch alone, as its own bench line."""
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    g = grouped_measure(args, dev, dist, rank, world)
    if rank == 0:
        line = {"metric": g["metric"], "value": g["value"], "unit": g["unit"],
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": g["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
                "data": "synthetic", "config": g["config"], "roofline": g["roofline"],
                "k1": g["k1"], "gpu_launches": g["gpu_launches"], "clocks": g["clocks"],
                "device_status": g["device_status"]}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def backward_measure(args, dev, dist, rank, world):
    """Forward (analytic signal, Gram with C) and backward (recompute,
    S = G + G^H, Gamma = S P / T, adjoint Hilbert) of the masked ciPLV loss;
    returns the measurement as a dict (a bench line without the run keys)."""
    import torch
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    local = dev.index
    B, N, T = 16, 1024, 4096
    hf = plv.Handle(precision=args.precision, device=local)
    hb = hf  # split handles take the backward contraction to the tensor cores
    x = synth.bandlimited(B, N, T, seed=rank_seed(1005, rank), device=dev)
    mask = synth.random_pair_mask(N, 0.10, seed=1005, device=dev)
    g3 = mask.to(torch.float32).expand(B, N, N).contiguous()
    P = hf.empty_phasors(B, N, T)
    out = {k: torch.empty((B, N, N), dtype=torch.float32, device=dev)
           for k in ("ciplv",)}
    out["C"] = torch.empty((B, N, N), dtype=torch.complex64, device=dev)
    grad = torch.empty((B, N, T), dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(e=None):
        if e:
            e[0].record(s)
        hf.plv_analytic(x, P)
        hf.plv_gram(P, B, N, T, plv=False, iplv=False, ciplv=True, C=True,
                    out=out)
        if e:
            e[1].record(s)
        hb.plv_backward(x, out["C"], None, None, g3, grad_x=grad)
        if e:
            e[2].record(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    per = [[ev(), ev(), ev()] for _ in range(args.steps)]
    for p in per:
        step(p)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = sum(p[0].elapsed_time(p[2]) for p in per)
    ms = max_over_ranks(ms, dist, dev)
    fwd_ms = statistics.mean(p[0].elapsed_time(p[1]) for p in per)
    bwd_ms = statistics.mean(p[1].elapsed_time(p[2]) for p in per)
    ms_step = ms / args.steps
    units = float(N) * N * T * B
    value = job_value(units, world, ms_step)
    ld = (T + 31) // 32 * 32
    gemm_flops = 8.0 * N * N * ld * B
    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    split = args.precision != "fp32"
    peak = float(peaks["bf16_tflops"]) if split else fp32_peak
    # the FP32 CUDA-core backward on the same input, for comparison
    fp32_bwd = None
    if split and not args.no_fp32_compare:
        h32 = plv.Handle(precision="fp32", device=local)
        g32 = torch.empty_like(grad)
        h32.plv_backward(x, out["C"], None, None, g3, grad_x=g32)
        torch.cuda.synchronize(dev)
        a, b = ev(), ev()
        a.record(s)
        for _ in range(2):
            h32.plv_backward(x, out["C"], None, None, g3, grad_x=g32)
        b.record(s)
        torch.cuda.synchronize(dev)
        rel = float(torch.linalg.norm(grad - g32) / torch.linalg.norm(g32))
        fp32_bwd = {"backward_ms": a.elapsed_time(b) / 2,
                    "rel_l2_diff_vs_split": rel}
        h32.close()
    # the same loss with the forward's phasors kept for the backward pass
    # (plv_analytic_save / plv_backward_saved: no recompute), where the
    # handle supports it
    saved_mode = None
    if args.precision in ("fp32", "bf16x3"):
        grad_s = torch.empty_like(grad)

        def step_saved(e=None):
            if e:
                e[0].record(s)
            sv = hf.plv_analytic_save(x)
            hf.plv_gram(sv["P"], B, N, T, plv=False, iplv=False, ciplv=True, C=True,
                        out=out)
            if e:
                e[1].record(s)
            hb.plv_backward_saved(sv, out["C"], None, None, g3, grad_x=grad_s)
            if e:
                e[2].record(s)

        for _ in range(args.warmup):
            step_saved()
        torch.cuda.synchronize(dev)
        per_s = [[ev(), ev(), ev()] for _ in range(args.steps)]
        for p in per_s:
            step_saved(p)
        torch.cuda.synchronize(dev)
        ms_s = max_over_ranks(sum(p[0].elapsed_time(p[2]) for p in per_s), dist, dev)
        saved_mode = {
            "ms_per_step": ms_s / args.steps,
            "value": job_value(units, world, ms_s / args.steps),
            "forward_ms": statistics.mean(p[0].elapsed_time(p[1]) for p in per_s),
            "backward_ms": statistics.mean(p[1].elapsed_time(p[2]) for p in per_s),
            "rel_l2_diff_vs_recompute": float(torch.linalg.norm(grad_s - grad)
                                              / torch.linalg.norm(grad)),
            "memory": "phasors and 1/|z| kept from the forward pass ("
                      f"{20 if split else 12} bytes per sample)",
            "gpu_launches": (2 + 3) * args.steps}
        del grad_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{args.precision} (backward contraction "
                 f"{'bf16x3' if args.precision != 'fp32' else 'f32'}, "
                 f"rest f32)",
        "data": "synthetic",
        "config": {"workload": BACKWARD, "B": B, "N": N, "T": T,
                   "loss": "sum of ciPLV over a seeded 10% mask of ordered "
                           "pairs", "recompute": "analytic signal "
                   "recomputed in the backward pass"},
        "forward_ms": fwd_ms, "backward_ms": bwd_ms,
        "backward_contraction": {
            "flops_per_step": gemm_flops * (3 if split else 1),
            "note": ("Gamma = S P / T on the tensor cores, BF16 hi+lo "
                     "splits (3 products per term); bound: tensor, "
                     "peak %s BF16 burst" % peak_kind) if split else
                    ("Gamma = S P / T, FP32 on the CUDA cores; bound: "
                     "alu, peak derived from 152 SMs x 128 FMA x 2 x "
                     "max SM clock"),
            "peak_tflops": peak,
            "lower_bound_tflops_over_whole_backward":
                gemm_flops * (3 if split else 1) / (bwd_ms / 1e3) / 1e12},
        "fp32_backward": fp32_bwd,
        "saved_analytic_signal": saved_mode,
        # forward: K1, Gram; backward: recompute, S, contraction, adjoint (and
        # the split P's padding rows when N % 128 != 0)
        "gpu_launches": (2 + 4 + (1 if split and N % 128 else 0)) * args.steps,
        "clocks": clk, "device_status": hb.plv_sync_status()}
    hf.close()
    return line


def run_backward(args):
    """The differentiable-loss workload alone, as its own bench line."""
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = backward_measure(args, torch.device("cuda", local), dist, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


TIMERES = "time-resolved-E64-N512-T1000"


def run_time_resolved(args):
    """The time-resolved PLV over trials (Eq. 1 / 8): analytic signal of
    every trial (FP32 phasors), the trial operands of every sample, and one
    Gram per sample with K = trials (outputs L x N x N per metric)."""
    import torch
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    E, N, T = 64, 512, 1000
    h = plv.Handle(precision=args.precision, device=local)
    h32 = h._fp32()
    x = synth.bandlimited(E, N, T, seed=rank_seed(1006, rank), device=dev)
    ld = plv.phasor_ld(T)
    V = h32.empty_phasors(E, N, T)
    P = h.empty_phasors(T, N, E)
    out = {k: torch.empty((T, N, N), dtype=torch.float32, device=dev)
           for k in ("plv", "iplv", "ciplv")}
    s = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(e=None):
        if e:
            e[0].record(s)
        h32.plv_analytic(x, V)
        if e:
            e[1].record(s)
        h.plv_trial_operands(V, E, N, ld, 0, T, "asis", P)
        if e:
            e[2].record(s)
        h.plv_gram(P, T, N, E, out=out)
        if e:
            e[3].record(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    per = [[ev(), ev(), ev(), ev()] for _ in range(args.steps)]
    for p in per:
        step(p)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = max_over_ranks(sum(p[0].elapsed_time(p[3]) for p in per), dist, dev)
    k1_ms = statistics.mean(p[0].elapsed_time(p[1]) for p in per)
    tr_ms = statistics.mean(p[1].elapsed_time(p[2]) for p in per)
    gram_ms = statistics.mean(p[2].elapsed_time(p[3]) for p in per)
    ms_step = ms / args.steps
    units = float(N) * N * E * T  # channel pairs x trials x samples
    peaks, peak_kind = _peaks()
    # the Gram over K = E = 64 trials is output-bound: its algorithmic bytes
    # are the operands read once and the three full N x N outputs per sample
    ldE = plv.phasor_ld(E)
    gram_bytes = T * ((N + 127) // 128 * 128) * ldE * 8 + 3 * 4 * T * N * N
    roof = {"bound": "hbm", "kernel": "k_gram_tc (batch = samples, K = trials)",
            "achieved": gram_bytes / (gram_ms / 1e3) / 1e9,
            "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
            "peak_source": f"{peak_kind} HBM copy", "traffic": None,
            "launch_ms": gram_ms}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if rank == 0:
        line = {
            "metric": "channel-pair·trial·samples/s (N²·E·T/s), time-resolved "
                      "PLV+iPLV+ciPLV over trials",
            "value": job_value(units, world, ms_step),
            "unit": "channel-pair·trial·samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": TIMERES, "E_trials": E, "N": N, "T": T,
                       "outputs": "3 x T x N x N FP32 (3.1 GB per step)"},
            "roofline": roof,
            "parts_ms": {"analytic_fp32": k1_ms, "trial_operands": tr_ms,
                         "gram": gram_ms},
            "gpu_launches": 3 * args.steps, "clocks": clk,
            "device_status": h.plv_sync_status()}
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


COHERENCY = "coherency-E64-N1024-T1000-F64"


def run_coherency(args):
    """Coherency across trials (Eq. 12) from raw trials: the DFT of every
    trial's rows at 64 consecutive bins (4-67 Hz at fs = 1000 Hz, T = 1000),
    the RMS-normalised trial operands of every bin, and one Gram per bin
    with K = trials (coherence, imaginary coherency, lagged coherence)."""
    import torch
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    E, N, T, f0, F = 64, 1024, 1000, 4, 64
    h = plv.Handle(precision=args.precision, device=local)
    x = synth.bandlimited(E, N, T, seed=rank_seed(1009, rank), band=(2.0, 120.0), device=dev)
    ldF = plv.phasor_ld(F)
    V = torch.empty((E, N, 2, ldF), dtype=torch.float32, device=dev)
    P = h.empty_phasors(F, N, E)
    out = {k: torch.empty((F, N, N), dtype=torch.float32, device=dev)
           for k in ("plv", "iplv", "ciplv")}
    s = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(e=None):
        if e:
            e[0].record(s)
        h.plv_dft_bins(x, f0, F, V)
        if e:
            e[1].record(s)
        h.plv_trial_operands(V, E, N, ldF, 0, F, "rms", P)
        if e:
            e[2].record(s)
        h.plv_gram(P, F, N, E, out=out)
        if e:
            e[3].record(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    per = [[ev(), ev(), ev(), ev()] for _ in range(args.steps)]
    for p in per:
        step(p)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = max_over_ranks(sum(p[0].elapsed_time(p[3]) for p in per), dist, dev)
    dft_ms = statistics.mean(p[0].elapsed_time(p[1]) for p in per)
    tr_ms = statistics.mean(p[1].elapsed_time(p[2]) for p in per)
    gram_ms = statistics.mean(p[2].elapsed_time(p[3]) for p in per)
    ms_step = ms / args.steps
    units = float(N) * N * E * F  # channel pairs x trials x bins
    peaks, peak_kind = _peaks()
    # the DFT at F bins is a thin real GEMM on the CUDA cores: 4 flops per
    # (row, sample, bin), against the FP32 FMA peak at the maximum SM clock
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    dft = {"kernel": "k_dft_bins", "bound": "alu", "ms": dft_ms,
           "achieved": 4.0 * E * N * T * F / (dft_ms / 1e3) / 1e12, "peak": alu_peak,
           "unit": "TFLOP/s"}
    dft["frac"] = dft["achieved"] / dft["peak"]
    # the Gram over K = 64 trials is output-bound: operands read once, three
    # full N x N outputs per bin
    ldE = plv.phasor_ld(E)
    gram_bytes = F * ((N + 127) // 128 * 128) * ldE * 8 + 3 * 4 * F * N * N
    roof = {"bound": "hbm", "kernel": "k_gram_tc (batch = bins, K = trials)",
            "achieved": gram_bytes / (gram_ms / 1e3) / 1e9,
            "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
            "peak_source": f"{peak_kind} HBM copy", "traffic": None,
            "launch_ms": gram_ms}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if rank == 0:
        line = {
            "metric": "channel-pair·trial·bins/s (N²·E·F/s), coherence, imaginary "
                      "coherency and lagged coherence across trials",
            "value": job_value(units, world, ms_step),
            "unit": "channel-pair·trial·bins/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": COHERENCY, "E_trials": E, "N": N, "T": T,
                       "bins": [f0, f0 + F - 1],
                       "outputs": "3 x F x N x N FP32 (0.8 GB per step)"},
            "roofline": roof, "dft": dft,
            "parts_ms": {"dft_bins": dft_ms, "trial_operands_rms": tr_ms,
                         "gram": gram_ms},
            "gpu_launches": 3 * args.steps, "clocks": clk,
            "device_status": h.plv_sync_status()}
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


WINDOWS = "sliding-N1024-T4096-W512-hop256-E8"


def run_windows(args):
    """Dynamic PLV: the analytic signal of every epoch, then the Gram of
    every window of 512 samples at a hop of 256 (15 windows per epoch), one
    persistent launch over all (epoch, window) matrices."""
    import torch
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    E, N, T, W, hop = 8, 1024, 4096, 512, 256
    nw = (T - W) // hop + 1
    h = plv.Handle(precision=args.precision, device=local)
    x = synth.bandlimited(E, N, T, seed=rank_seed(1007, rank), device=dev)
    P = h.empty_phasors(E, N, T)
    out = {k: torch.empty((E, nw, N, N), dtype=torch.float32, device=dev)
           for k in ("plv", "iplv", "ciplv")}
    s = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(e=None):
        if e:
            e[0].record(s)
        h.plv_analytic(x, P)
        if e:
            e[1].record(s)
        h.plv_gram_windows(P, E, N, T, 0, W, hop, nw, out=out)
        if e:
            e[2].record(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    per = [[ev(), ev(), ev()] for _ in range(args.steps)]
    for p in per:
        step(p)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = max_over_ranks(sum(p[0].elapsed_time(p[2]) for p in per), dist, dev)
    k1_ms = statistics.mean(p[0].elapsed_time(p[1]) for p in per)
    gram_ms = statistics.mean(p[1].elapsed_time(p[2]) for p in per)
    ms_step = ms / args.steps
    units = float(N) * N * W * nw * E  # channel pairs x window samples
    peaks, peak_kind = _peaks()
    flops = gram_flops(N, W, E * nw, args.precision)
    split = args.precision != "fp32"
    roof = {"bound": "tensor" if split else "alu", "kernel": "k_gram_tc (windows)",
            "achieved": flops / (gram_ms / 1e3) / 1e12,
            "peak": float(peaks["bf16_tflops"]) if split else
            152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12,
            "unit": "TFLOP/s", "peak_source": f"{peak_kind}", "traffic": None,
            "launch_ms": gram_ms}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": job_value(units, world, ms_step), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": WINDOWS, "E": E, "N": N, "T": T, "W": W, "hop": hop,
                       "windows": nw, "outputs": f"3 x {E * nw} x N x N FP32"},
            "roofline": roof, "parts_ms": {"analytic": k1_ms, "gram_windows": gram_ms},
            "gpu_launches": 2 * args.steps, "clocks": clk,
            "device_status": h.plv_sync_status()}
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


BANDS_WL = "bands-5-N2048-T4096-E8"
# the same with a length that is not a power of two (any-length band engine)
BANDS_WL_ANY = "bands-5-N2048-T4000-E8"


def run_bands(args):
    """The multi-band front end: broadband x, five band masks (4-8, 8-12,
    13-30, 30-45, 55-80 Hz, 4th-order Butterworth magnitude squared), the
    band-limited phasors of every band from one forward FFT per row pair,
    then one grouped Gram over the five bands."""
    import numpy as np
    import torch
    import paper_1710_08037_gb300 as plv
    from paper_1710_08037_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    E, N, T = 8, 2048, (4000 if args.workload == BANDS_WL_ANY else 4096)
    nb = len(BANDS)
    h = plv.Handle(precision=args.precision, device=local)
    x = synth.bandlimited(E, N, T, seed=rank_seed(1008, rank), band=(1.0, 120.0), device=dev)
    masks = torch.tensor(np.stack([synth.butter_power(T, 1000.0, b) for b in BANDS]),
                         dtype=torch.float32, device=dev)
    P = h.plv_analytic_bands(x, masks)
    probs = [{"P": P[b], "batch": E, "N": N, "T": T} for b in range(nb)]
    grp = h.plv_group_create(probs)
    s = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(e=None):
        if e:
            e[0].record(s)
        h.plv_analytic_bands(x, masks, P)
        if e:
            e[1].record(s)
        h.plv_gram_grouped(grp)
        if e:
            e[2].record(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    per = [[ev(), ev(), ev()] for _ in range(args.steps)]
    for p in per:
        step(p)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = max_over_ranks(sum(p[0].elapsed_time(p[2]) for p in per), dist, dev)
    fe_ms = statistics.mean(p[0].elapsed_time(p[1]) for p in per)
    gram_ms = statistics.mean(p[1].elapsed_time(p[2]) for p in per)
    # the per-band analytic signal alone (no band-pass), five times, for scale
    Pa = h.empty_phasors(E, N, T)
    a, b_ = ev(), ev()
    h.plv_analytic(x, Pa)
    a.record(s)
    for _ in range(nb):
        h.plv_analytic(x, Pa)
    b_.record(s)
    torch.cuda.synchronize(dev)
    five_hilbert_ms = a.elapsed_time(b_)
    ms_step = ms / args.steps
    units = float(N) * N * T * E * nb
    peaks, peak_kind = _peaks()
    flops = gram_flops(N, T, E * nb, args.precision)
    roof = {"bound": "tensor", "kernel": "k_gram_tc (grouped over bands)",
            "achieved": flops / (gram_ms / 1e3) / 1e12, "peak": float(peaks["bf16_tflops"]),
            "unit": "TFLOP/s", "peak_source": f"{peak_kind} bf16 dense (burst)",
            "traffic": None, "launch_ms": gram_ms}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # front end bytes: x read once, 8 B of phasor per sample and band written
    fe_bytes = E * N * T * (4 + 8 * nb)
    if rank == 0:
        line = {
            "metric": METRIC, "value": job_value(units, world, ms_step), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": args.workload, "E": E, "N": N, "T": T, "bands": BANDS},
            "roofline": roof,
            "front_end": {"kernel": ("k_hilbert_bands" if T & (T - 1) == 0
                                     else "k_hilbert_conv_bands"), "ms": fe_ms, "bound": "hbm",
                          "achieved_GBps": fe_bytes / (fe_ms / 1e3) / 1e9,
                          "peak": float(peaks["hbm_gbs"]),
                          "five_plain_analytic_ms": five_hilbert_ms},
            "gpu_launches": (1 + nb + 1) * args.steps, "clocks": clk,
            "device_status": h.plv_sync_status()}
        print(json.dumps(line), flush=True)
    grp.close()
    h.close()
    if dist:
        dist.destroy_process_group()


def oracle_errors(samp, ref, nsub, N):
    """Per-metric max / mean absolute error of each GPU path against the
    FP64 oracle on the sampled |S| x |S| pairs of epoch 0.  ciPLV is also
    given over the pairs whose Eq. 14 denominator sqrt(1 - Re^2) is at least
    0.05 (its error grows as 1 / sqrt(1 - Re^2))."""
    import numpy as np
    d = 1.0 - ref["plv"] ** 2 + ref["iplv"] ** 2  # 1 - Re^2 = 1 - |C|^2 + Im^2
    well = np.sqrt(np.maximum(d, 0.0)) >= 0.05
    out = {"sample": f"epoch 0, {nsub} of {N} channels, all {nsub}^2 ordered "
                     f"pairs (diagonal included)",
           "ciplv_well_conditioned_pairs": int(well.sum())}
    for path, got in samp.items():
        e = {}
        for k in ("plv", "iplv", "ciplv"):
            err = np.abs(got[k] - ref[k])
            e[k] = {"max": float(err.max()), "mean": float(err.mean())}
        err = np.abs(got["ciplv"] - ref["ciplv"])[well]
        e["ciplv_well_conditioned"] = {"max": float(err.max()) if err.size else 0.0,
                                       "mean": float(err.mean()) if err.size else 0.0}
        out[path] = e
    return out


def sample_channels(N, seed, nsub):
    """The channel subset S the oracle legs use: ``nsub`` of N, seeded."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=min(nsub, N), replace=False))


def _epoch0(N, T, seed, x=None):
    """Epoch 0 of the workload's input: from ``x`` if given, else generated
    (epoch 0 of an E-epoch draw equals a one-epoch draw of the same seed)."""
    import torch
    from paper_1710_08037_gb300 import synth
    if x is None:
        x = synth.bandlimited(1, N, T, seed=seed, device="cpu"
                              if not torch.cuda.is_available() else "cuda")
    return x[0]


def oracle_step(x0, sub):
    """One bounded step of the FP64 oracle: the direct-DFT analytic signal of
    the channel subset ``sub`` of epoch-0 rows ``x0``, then the pairwise
    loop over all |sub|^2 ordered pairs.  Returns (outputs, z, seconds of
    the analytic signal, seconds of the pairwise loop)."""
    import torch
    import oracle
    xs = x0[torch.as_tensor(sub, device=x0.device)].double().cpu().numpy()
    t0 = time.perf_counter()
    z = oracle.analytic(xs)
    t1 = time.perf_counter()
    ref = oracle.pairwise(z)
    t2 = time.perf_counter()
    return ref, z, t1 - t0, t2 - t1


def extrapolated_epoch_s(N, nsub, t_hilbert, t_pairs):
    """Seconds the oracle would take for one full epoch of N channels: its
    analytic signal is linear in rows, its pairwise loop in pairs."""
    r = N / nsub
    return t_hilbert * r + t_pairs * r * r


def cpu_baseline(E, N, T, seed, nsub, x=None, values=None):
    """The FP64 oracle as it stands, on a bounded sample of the same
    workload: one epoch, a random subset S of ``nsub`` channels; direct-DFT
    analytic signal of S, then the pairwise loop over all |S|^2 pairs.
    ``value`` is the measured rate on that sample, |S|^2 T per second of
    oracle time; the rate extrapolated to a full epoch (analytic signal
    linear in rows, pairs quadratic) is given beside it.  ``x``: the
    workload's input (epoch 0 is used), else it is generated; ``values``: a
    dict that receives the oracle's PLV / iPLV / ciPLV of the sample."""
    import numpy as np
    import oracle
    sub = sample_channels(N, seed, nsub)
    ref, z, th, tp = oracle_step(_epoch0(N, T, seed, x), sub)
    if values is not None:
        values.update({k: ref[k] for k in ("plv", "iplv", "ciplv")})
    # context: the paper's reformulation on the same sample and host,
    # unit phasors once, then one complex FP64 matrix product (numpy's BLAS)
    t3 = time.perf_counter()
    az = np.abs(z)
    Pz = np.where(az > 0, z / np.where(az > 0, az, 1.0), 0.0)
    _ = (Pz @ Pz.conj().T) / z.shape[1]
    t4 = time.perf_counter()
    t_epoch = extrapolated_epoch_s(N, len(sub), th, tp)
    return {"value": float(len(sub)) ** 2 * T / (th + tp), "unit": UNIT,
            "cores": oracle.threads(), "kind": "oracle",
            "sample": f"1 of {E} epochs, {len(sub)} of {N} channels: "
                      f"direct-DFT analytic signal {th:.2f} s, pairwise "
                      f"loop over {len(sub)}^2 pairs {tp:.2f} s; value = "
                      f"{len(sub)}^2 x {T} channel-pair samples / {th + tp:.2f} s",
            "sample_s": th + tp,
            "extrapolated_full_epoch": {
                "value": float(N) * N * T / t_epoch, "unit": UNIT,
                "epoch_s": t_epoch,
                "how": "analytic signal x N/|S|, pairwise loop x (N/|S|)^2"},
            "context_gram_vs_pairwise": {
                "pairwise_loop_s": tp, "gram_fp64_blas_s": t4 - t3,
                "speedup": tp / max(t4 - t3, 1e-9),
                "note": "the paper's reformulation (unit phasors once, one "
                        "complex matrix product; numpy BLAS) against the "
                        "pairwise loop on the same sample and host; the paper "
                        "reports ~100x for its Gram over its vectorised loop "
                        "(MATLAB, CPU not stated)"}}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores.
    Each step is one bounded sample of the workload (epoch 0, the seeded
    channel subset the GPU arm's cpu_baseline uses, all its ordered pairs);
    ms_per_step is that step's measured wall time and value the sample's
    channel-pair samples per second of it.  Under torchrun only rank 0
    runs."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    E, N, T, seed = WORKLOADS[args.workload]
    x0 = _epoch0(N, T, seed)
    sub = sample_channels(N, seed, args.cpu_sample)
    for _ in range(args.warmup):
        oracle_step(x0, sub)
    walls, parts = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, _, th, tp = oracle_step(x0, sub)
        walls.append(time.perf_counter() - t0)
        parts.append((th, tp))
    ms_step = 1e3 * sum(walls) / len(walls)
    units = float(len(sub)) ** 2 * T
    value = units / (ms_step / 1e3)
    th = statistics.mean(p[0] for p in parts)
    tp = statistics.mean(p[1] for p in parts)
    t_epoch = extrapolated_epoch_s(N, len(sub), th, tp)
    cpu = {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
           "sample": f"per step: epoch 0 of {E}, {len(sub)} of {N} channels "
                     f"(seeded), direct-DFT analytic signal {th:.2f} s + "
                     f"pairwise loop over {len(sub)}^2 pairs {tp:.2f} s",
           "extrapolated_full_epoch": {
               "value": float(N) * N * T / t_epoch, "unit": UNIT, "epoch_s": t_epoch,
               "how": "analytic signal x N/|S|, pairwise loop x (N/|S|)^2"}}
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, N, T, E, args.precision,
                                      int(os.environ.get("WORLD_SIZE", "1"))),
            "units_per_step": units,
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _free_port():
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def spawn_replicas(n, argv, script=None):
    """Run ``script`` (this file by default) as n ranks of one node, one
    process per GPU, through torch.distributed.run on 127.0.0.1; returns
    its exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={n}", "--master-addr=127.0.0.1",
           f"--master-port={_free_port()}", script or os.path.abspath(__file__),
           *argv]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16x3", "fp16x3"],
                    default="bf16x3")
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="skip timing the plain FP32 path beside the split one")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + [GROUPED, BACKWARD, TIMERES,
                                                               COHERENCY,
                                                               WINDOWS, BANDS_WL,
                                                               BANDS_WL_ANY],
                    default=DEFAULT_WORKLOAD)
    ap.add_argument("--subjects", type=int, default=256,
                    help="subjects of the grouped workload")
    ap.add_argument("--peak", choices=["auto", "burst", "sustained"], default="auto",
                    help="tensor peak of the Gram's roofline: burst, sustained, or "
                         "(auto) sustained when the timed region lasts a second or more")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-grouped", action="store_true",
                    help="main workload: skip the uneven-batch sub-record")
    ap.add_argument("--no-configs", action="store_true",
                    help="main workload: skip the FP32, backward and parity sub-records")
    ap.add_argument("--no-tune", action="store_true",
                    help="grouped workload: keep the plan's default launch shapes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=384)
    ap.add_argument("--e2e-chunks", type=int, default=6)
    ap.add_argument("--e2e-streams", type=int, default=2)
    args = ap.parse_args()
    world_env = os.environ.get("WORLD_SIZE")
    if world_env is None and args.gpus > 1:
        # no process group yet: launch the N ranks here
        sys.exit(spawn_replicas(args.gpus, sys.argv[1:]))
    if world_env is not None and int(world_env) != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world_env}", file=sys.stderr)
        sys.exit(2)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == GROUPED:
        run_grouped(args)
    elif args.workload == BACKWARD:
        run_backward(args)
    elif args.workload == TIMERES:
        run_time_resolved(args)
    elif args.workload == COHERENCY:
        run_coherency(args)
    elif args.workload == WINDOWS:
        run_windows(args)
    elif args.workload in (BANDS_WL, BANDS_WL_ANY):
        run_bands(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
