#!/usr/bin/env python
"""Throughput of the distilled-nucleon hot path on B300.

One step = the whole hot path for one gauge configuration of the workload:
elementals Phi[t][p] for every timeslice and momentum, the N_B x N_B
correlation matrix C_ab(t) for every (t, p) (source at t0 = 0) and the GEVP
of every (p, t).  The metric is C_ab(t) entries per second (N_p N_B^2 N_t
entries per step per configuration); algorithmic TFLOP/s is reported beside
it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 1..5]
                    [--mode auto|fp16x6|fp16x3|bf16x6|bf16x3|fp32|fp64]
                    [--impl ours|reference] [--ncfg K] [--nt NT]
                    [--no-cpu-baseline] [--no-parity] [--no-plain]

Default: workload 3 (L=32, N_t=64, N_v=128, 5 momenta, 6 profiles), mode
fp16x6, 3 warm-up and 3 timed steps, plus the end-to-end leg (host inputs
in, C out), a sampled parity check against the FP64 oracle, the oracle's own
throughput on the host cores, and the plain FP32/FP64 paths on one
timeslice.  Workload 4 runs an ensemble of --ncfg configurations with
uneven N_v as one graph-captured plan.  --impl reference times the FP64
oracle, one (t, p) slice per step.

With N > 1 (launched by torch.distributed.run) every rank processes its own
configurations (configuration c on rank c mod N): weak scaling, no
collective on the data path; entries are summed over ranks and the time is
the slowest rank's.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_37723_b300 import synth  # noqa: E402  (host-only, no CUDA)

METRIC = "C_ab(t) entries/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


# --------------------------------------------------------------------------- inputs

def log(msg: str):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def _eig_worker(args):
    cid, cfg, ts, shm_name, shape, dtype = args
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    out = np.ndarray(shape, dtype=dtype, buffer=shm.buf)
    p = synth.config(cid, cfg)
    for t in ts:
        out[t] = p.eigvecs(t)
    del out
    shm.close()
    return len(ts)


def make_inputs(cid: int, cfg: int, workers: int, nt: int = 0):
    """Host inputs of one configuration (numpy, identical bytes to the tests).
    Timeslices are drawn in parallel processes straight into shared memory.
    nt > 0 keeps only the first nt timeslices (a smaller case of the same
    shapes, for profilers)."""
    p = synth.config(cid, cfg)
    if nt > 0:
        p = dataclasses.replace(p, nt=min(p.nt, nt))
    shape = (p.nt, p.nv, p.V3, 3)
    dtype = np.dtype(p.dtype)
    if workers > 1 and p.nt > 1:
        import multiprocessing as mp
        from multiprocessing import shared_memory
        shm = shared_memory.SharedMemory(create=True, size=int(np.prod(shape)) * dtype.itemsize)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"   # one BLAS thread per worker process (inherited at spawn)
        try:
            chunks = [list(range(w, p.nt, workers)) for w in range(workers)]
            with mp.get_context("spawn").Pool(workers) as pool:
                pool.map(_eig_worker, [(cid, cfg, c, shm.name, shape, dtype.str) for c in chunks if c])
            v = np.array(np.ndarray(shape, dtype=dtype, buffer=shm.buf))
        finally:
            shm.close()
            shm.unlink()
    else:
        v = p.all_eigvecs()
    tau = p.all_perambulators()
    return p, v, tau


# --------------------------------------------------------------------------- flops

def algorithmic_flops(p: synth.Problem) -> dict:
    """Counting convention for TFLOP/s (8 real flops per complex MAC):
    elementals 8*3V3*T3 per (t, p) (i<j<k only) and correlator
    8*92*N_B*N_v^4 per (t, p)."""
    tp = p.nt * p.np_
    el = 8.0 * 3 * p.V3 * p.T3 * tp
    co = 8.0 * 92 * p.nb * p.nv ** 4 * tp
    return {"elementals": el, "correlator": co, "total": el + co}


def executed_cmacs(p: synth.Problem) -> dict:
    """Complex MACs the library's contraction kernels execute per step:
    elementals np*nv x P2 x 3V3 dense tiles (triangle-skipped at tile level,
    counted dense here), correlator 12 N_B n^4 (step i) + 24 N_B n^4 (step j)
    + 2.5 N_B n^4 (source, i'<j') per (t, p)."""
    n = p.nv
    P2 = n * (n - 1) // 2
    tp = p.nt * p.np_
    return {"step_i": 12.0 * p.nb * n ** 4 * tp, "step_j": 24.0 * p.nb * n ** 4 * tp,
            "source": 5.0 * p.nb * P2 * n * n * tp}


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- cpu baseline

class OracleSlices:
    """The FP64 oracle, as it stands, on (t, p = 0) slices of a workload: the
    source elementals at t = 0 once (momentum 0), then per slice the sink
    elementals of that t and momentum and that slice's C_ab(t).  Input
    generation is not timed.  The source elementals serve every (t, p) slice
    of the real workload, so a slice is charged 1/N_t of their time."""

    def __init__(self, cid: int, nt: int = 0):
        from oracle import nucleon as orc
        self.orc = orc
        p = synth.config(cid, 0)
        if nt > 0:
            p = dataclasses.replace(p, nt=min(p.nt, nt))
        self.p = p
        self.mom0 = p.mom[:1]
        v0 = p.eigvecs(0)
        t0 = time.perf_counter()
        self.phi_src = orc.elementals_t(v0, p.L, self.mom0)[0]
        self.src_s = time.perf_counter() - t0

    def slice(self, t: int) -> float:
        """Seconds of oracle work for slice t (source share included)."""
        p = self.p
        vt, tau = p.eigvecs(t), p.perambulator(t)
        t0 = time.perf_counter()
        phi = self.orc.elementals_t(vt, p.L, self.mom0)[0]
        self.orc.correlator_tp(phi, self.phi_src, tau, p.prof, p.prof)
        return time.perf_counter() - t0 + self.src_s / p.nt

    @staticmethod
    def cores() -> int:
        try:
            import threadpoolctl
            info = threadpoolctl.threadpool_info()
            return int(max(i.get("num_threads", 1) for i in info)) if info else 1
        except Exception:
            return os.cpu_count() or 1


def cpu_baseline(cid: int, budget_s: float = 15.0) -> dict:
    """The oracle on slices t = 1, 2, ... until about `budget_s` seconds of
    CPU work are spent (at least one slice)."""
    o = OracleSlices(cid)
    p = o.p
    elapsed, done = 0.0, 0
    for t in range(1, max(2, p.nt)):
        elapsed += o.slice(t if p.nt > 1 else 0)
        done += 1
        if elapsed > budget_s:
            break
    entries = done * p.nb * p.nb
    return {"value": entries / elapsed, "unit": METRIC, "cores": o.cores(), "kind": "oracle",
            "sample": f"{done} (t, p=0) slice(s) of {p.nt * p.np_}: sink elementals + C_ab(t) each, plus "
                      f"1/N_t of the t=0 source elementals ({o.src_s:.1f} s); {elapsed:.1f} s; "
                      f"numpy FP64 with BLAS threads",
            "seconds": elapsed}


# --------------------------------------------------------------------------- ranks

def shard_configs(ncfg: int, rank: int, world: int) -> list:
    """Configurations of an ensemble handled by `rank`: c with c mod world = rank
    (independent problems: no data-path collective)."""
    return [c for c in range(ncfg) if c % world == rank]


def job_throughput(entries_local: float, ms_local: float, steps: int, dist=None, device=None):
    """Whole-job throughput: entries summed over ranks / the slowest rank's
    time.  Returns (entries/s, all entries per step, max ms)."""
    import torch
    t = torch.tensor([float(entries_local), float(ms_local)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        e, m = t[:1].clone(), t[1:].clone()
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
        t = torch.cat([e, m])
    all_entries, ms_max = float(t[0]), float(t[1])
    return all_entries * steps / (ms_max / 1e3), all_entries, ms_max


def gather_C(C_local: dict, ncfg: int, dist=None):
    """Rank 0 collects every configuration's correlation matrices after the
    run (the one exchange of the sharded path; N_p N_B^2 N_t complex numbers
    per configuration).  C_local maps configuration -> host tensor; returns
    the list indexed by configuration on rank 0 (None elsewhere)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [C_local[c] for c in range(ncfg)]
    parts = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object({c: t.numpy() for c, t in C_local.items()}, parts, dst=0)
    if dist.get_rank() != 0:
        return None
    merged = {}
    for part in parts:
        merged.update(part)
    return [merged[c] for c in range(ncfg)]


# --------------------------------------------------------------------------- ours

def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cid = args.workload
    workers = min(32, os.cpu_count() or 1)
    log(f"generating inputs of workload {cid} (cfg {rank}) with {workers} processes")
    p, v_h, tau_h = make_inputs(cid, rank, workers, args.nt)   # before any CUDA call
    log(f"inputs ready: v {v_h.nbytes / 1e9:.2f} GB")

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_2609_37723_b300 import distil
    mode = args.mode
    if mode == "auto":
        mode = next((m for m in ("fp16x6", "bf16x6") if distil.mode_available(m)), "fp32")
    c128 = mode == "fp64"
    cdt = np.complex128 if c128 else np.complex64
    v_h = np.ascontiguousarray(v_h.astype(cdt))
    tau_h = np.ascontiguousarray(tau_h.astype(cdt))
    prof_h = np.ascontiguousarray(p.prof)
    t0_gevp = min(2, p.nt - 1)

    # pinned host copies for the end-to-end leg
    v_pin = torch.from_numpy(v_h).pin_memory()
    tau_pin = torch.from_numpy(tau_h).pin_memory()
    prof_pin = torch.from_numpy(prof_h).pin_memory()
    v = v_pin.to(dev)
    tau = tau_pin.to(dev)
    prof = prof_pin.to(dev)
    stream = torch.cuda.current_stream()

    T3 = p.T3
    tdt = torch.complex64 if mode == "fp32" else torch.complex128   # tensor-core modes keep c128 elementals
    phi = torch.empty((p.nt, p.np_, T3), dtype=tdt, device=dev)
    C = torch.empty((p.np_, p.nb, p.nb, p.nt), dtype=torch.complex128, device=dev)
    lam = torch.empty((p.np_, p.nt, p.nb), dtype=torch.complex128, device=dev)
    ws_e = distil.elementals_workspace(p.L, p.nt, p.nv, p.np_, mode)
    ws_c = distil.correlate_workspace(p.nt, p.nv, p.np_, p.nb, mode)
    ws = torch.empty(max(ws_e, ws_c, 1), dtype=torch.uint8, device=dev)

    def step(vv, tt, pp):
        distil.elementals(vv, p.L, p.mom, mode, out=phi, workspace=ws)
        distil.correlate(phi, phi[0], tt, pp, mode, out=C, workspace=ws)
        distil.gevp(C, t0_gevp, out=lam)

    def barrier():
        if world > 1:
            dist.barrier()

    for i in range(args.warmup):
        step(v, tau, prof)
        torch.cuda.synchronize()
        log(f"warm-up step {i} done")

    # ---------------- timed region (device-resident inputs)
    distil.profile_enable(timing=True, device=local)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly the timed launches
    for _ in range(args.steps):
        step(v, tau, prof)
    torch.cuda.nvtx.range_pop()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    log(f"timed region: {ms / args.steps:.1f} ms per step")
    kstats = distil.profile_read(device=local)
    distil.profile_enable(timing=False, device=local)
    entries = p.np_ * p.nb * p.nb * p.nt
    value, all_entries, ms = job_throughput(entries, ms, args.steps, dist if world > 1 else None, dev)
    ms_step = ms / args.steps

    # ---------------- end to end through the public API (host in, host out)
    C_host = torch.empty(C.shape, dtype=C.dtype).pin_memory()
    lam_host = torch.empty(lam.shape, dtype=lam.dtype).pin_memory()
    vin = torch.empty_like(v)
    tin = torch.empty_like(tau)
    pin_ = torch.empty_like(prof)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        vin.copy_(v_pin, non_blocking=True)
        tin.copy_(tau_pin, non_blocking=True)
        pin_.copy_(prof_pin, non_blocking=True)
        step(vin, tin, pin_)
        C_host.copy_(C, non_blocking=True)
        lam_host.copy_(lam, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = e0.elapsed_time(e1)
    e2e_value, _, ms_e2e = job_throughput(entries, ms_e2e, e2e_steps, dist if world > 1 else None, dev)
    h2d = v_h.nbytes + tau_h.nbytes + prof_h.nbytes
    d2h = C_host.numel() * 16 + lam_host.numel() * 16

    # ---------------- the plain CUDA-core paths on the same GPU (rank 0), one timeslice
    plain = None
    if rank == 0 and not args.no_plain and mode not in ("fp64", "fp32"):
        plain = plain_paths(distil, p, v_h, tau_h, prof, dev)

    # ---------------- parity of this run against the oracle on one slice (rank 0)
    out = None
    if rank == 0:
        flops = algorithmic_flops(p)
        pk = peaks()
        dom = max(kstats.items(), key=lambda kv: kv[1][1])[0] if kstats else None
        roof = roofline(dom, kstats, p, mode, pk, args.steps)
        launches = sum(l for l, _ in kstats.values())
        parity = parity_slice(p, v_h, tau_h, C.cpu().numpy(), mode) if not args.no_parity else None
        cpu = None if args.no_cpu_baseline else cpu_baseline(cid, args.cpu_budget)
        out = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32"}.get(mode, mode + "(f32 accumulate)"),
            "data": "synthetic (seeded orthonormal eigenvectors, Gaussian perambulators)",
            "config": {"workload": p.name, "L": p.L, "nt": p.nt, "nv": p.nv, "np": p.np_, "nb": p.nb,
                       "mode": mode, "cfg_per_rank": 1, "parallelism": f"weak x{world} (cfg = rank)",
                       "l2": "inputs larger than L2 (v is %.1f GB)" % (v_h.nbytes / 1e9)},
            "tflops_algorithmic": flops["total"] * world / (ms_step / 1e3) / 1e12,
            "e2e": {"value": e2e_value, "unit": "entries/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "kernels": {k: {"launches": l, "ms": round(t, 3)} for k, (l, t) in sorted(kstats.items(),
                                                                                  key=lambda kv: -kv[1][1])},
            "roofline": roof,
            "kernel_rooflines": kernel_rooflines(kstats, p, mode, pk, args.steps),
            "clocks": clk,
            "parity": parity,
            "cpu_baseline": cpu,
            "plain_paths": plain,
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def plain_paths(distil, p, v_h, tau_h, prof, dev):
    """The plain FP32 and FP64 CUDA-core paths of the library on the same GPU
    and inputs, on the first timeslice (all momenta, the source at t = 0 is
    that timeslice): elementals + correlator, entries/s, for comparison with
    the tensor-core mode."""
    import torch
    out = {}
    for mode, cdt in (("fp32", np.complex64), ("fp64", np.complex128)):
        v1 = torch.from_numpy(np.ascontiguousarray(v_h[:1].astype(cdt))).to(dev)
        t1 = torch.from_numpy(np.ascontiguousarray(tau_h[:1].astype(cdt))).to(dev)
        ms = []
        for rep in range(2):   # the first run loads the kernels
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            phi = distil.elementals(v1, p.L, p.mom, mode)
            C = distil.correlate(phi, phi[0], t1, prof, mode)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        entries = p.np_ * p.nb * p.nb
        out[mode] = {"value": entries / (ms[-1] / 1e3), "unit": "entries/s", "ms": ms[-1],
                     "sample": f"t = 0 slice: elementals of {p.np_} momenta + C_ab(0)"}
        del v1, t1, phi, C
    log("plain paths: " + ", ".join(f"{m} {r['value']:.1f} entries/s" for m, r in out.items()))
    return out


def run_ensemble(args):
    """Workload 4: an ensemble of configurations with uneven N_v (N_v drawn
    from {64, 96, 128} per configuration), sharded over ranks (configuration
    c goes to rank c mod N), all of a rank's configurations in one
    graph-captured plan (elementals -> correlator -> GEVP per
    configuration) with autotuned tensor-core kernel variants."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    workers = min(32, os.cpu_count() or 1)
    mine = shard_configs(args.ncfg, rank, world)
    log(f"ensemble of {args.ncfg} configurations, rank {rank} takes {mine}")
    host = [make_inputs(4, c, workers, args.nt) for c in mine]   # before any CUDA call
    log("inputs ready: v %.2f GB" % (sum(h[1].nbytes for h in host) / 1e9))

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_2609_37723_b300 import distil
    mode = args.mode
    if mode == "auto":
        mode = next((m for m in ("fp16x6", "bf16x6") if distil.mode_available(m)), "fp32")
    cdt = np.complex128 if mode == "fp64" else np.complex64
    cfgs, pins = [], []
    for p, v_h, tau_h in host:
        v_pin = torch.from_numpy(np.ascontiguousarray(v_h.astype(cdt))).pin_memory()
        tau_pin = torch.from_numpy(np.ascontiguousarray(tau_h.astype(cdt))).pin_memory()
        prof_pin = torch.from_numpy(np.ascontiguousarray(p.prof)).pin_memory()
        pins.append((v_pin, tau_pin, prof_pin))
        cfgs.append({"nv": p.nv, "v": v_pin.to(dev), "tau": tau_pin.to(dev), "prof": prof_pin.to(dev),
                     "C": torch.empty((p.np_, p.nb, p.nb, p.nt), dtype=torch.complex128, device=dev),
                     "lam": torch.empty((p.np_, p.nt, p.nb), dtype=torch.complex128, device=dev)})
    del host
    p0 = synth.config(4, mine[0]) if mine else synth.config(4, 0)
    if args.nt > 0:
        p0 = dataclasses.replace(p0, nt=min(p0.nt, args.nt))
    t0_gevp = min(2, p0.nt - 1)
    plan = distil.Plan(p0.L, p0.nt, p0.mom, p0.nb, t0_gevp, mode, cfgs, autotune=True)
    variants, kernels = plan.info()
    log(f"plan: {len(cfgs)} configurations, {kernels} kernels per run, variants {variants}")
    s = plan.stream
    for i in range(args.warmup):
        plan.run()
        s.synchronize()
        log(f"warm-up step {i} done")
    entries = sum(p0.np_ * p0.nb * p0.nb * p0.nt for _ in cfgs)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(s)
    for _ in range(args.steps):
        plan.run()
    ev1.record(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    log(f"timed region: {ms / args.steps:.1f} ms per step")
    value, all_entries, ms_max = job_throughput(entries, ms, args.steps, dist if world > 1 else None, dev)

    # end to end: host inputs in, C and lambda out, through the same plan
    C_host = [torch.empty(c["C"].shape, dtype=c["C"].dtype).pin_memory() for c in cfgs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    e2e_steps = max(1, min(args.steps, 3))
    with torch.cuda.stream(s):
        for _ in range(e2e_steps):
            for c, (vp, tp, pp) in zip(cfgs, pins):
                c["v"].copy_(vp, non_blocking=True)
                c["tau"].copy_(tp, non_blocking=True)
                c["prof"].copy_(pp, non_blocking=True)
            plan.run(s)
            for c, ch in zip(cfgs, C_host):
                ch.copy_(c["C"], non_blocking=True)
    e1.record(s)
    torch.cuda.synchronize()
    e2e_value, _, ms_e2e = job_throughput(entries, e0.elapsed_time(e1), e2e_steps, dist if world > 1 else None, dev)
    # every configuration's C on rank 0 (outside the timed regions)
    gathered = gather_C({c: ch for c, ch in zip(mine, C_host)}, args.ncfg,
                        dist if world > 1 else None)
    h2d = sum(vp.nbytes + tp.nbytes + pp.nbytes for vp, tp, pp in pins)
    d2h = sum(ch.numel() * 16 for ch in C_host)
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32"}.get(mode, mode + "(f32 accumulate)"),
            "data": "synthetic (seeded orthonormal eigenvectors, Gaussian perambulators)",
            "config": {"workload": f"L32_Nt64_ensemble{args.ncfg}", "L": p0.L, "nt": p0.nt,
                       "nv": [c["nv"] for c in cfgs], "np": p0.np_, "nb": p0.nb, "mode": mode,
                       "ncfg": args.ncfg, "parallelism": f"weak x{world} (configuration c on rank c mod N)",
                       "graph": {"kernels_per_run": kernels, "variants": variants},
                       "C_gathered_on_rank0": len(gathered) if gathered is not None else 0,
                       "l2": "inputs larger than L2"},
            "e2e": {"value": e2e_value, "unit": "entries/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(kernels * args.steps),
            "clocks": clk, "parity": None, "cpu_baseline": None,
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def kernel_bytes(name, p):
    """Algorithmic HBM bytes one step asks of the memory-side kernel
    families: what they must read and write at least."""
    n, nb, tp = p.nv, p.nb, p.nt * p.np_
    P2 = n * (n - 1) // 2
    table = {
        # V (nb x 6 spin pairs x n^3) and X (nb x 5 x P2 x n), complex double-float, read once
        "dot": ((96.0 * nb * n ** 3 + 80.0 * nb * P2 * n) * tp, "V + X per (t,p), 16 B each"),
        # the cross-product planes written once: P2 x 3 V3 x 12 B per timeslice
        "split_pairs": (12.0 * P2 * 3 * p.V3 * p.nt, "C(N_v,2) x 3 V3 x 12 B per t written"),
    }
    return table.get(name)


def kernel_rooflines(kstats, p, mode, pk, steps):
    """Every contraction kernel against the tensor peak (issued split
    products) and the memory-side kernels against the measured HBM copy
    bandwidth; achieved from the summed CUDA-event time over `steps` steps."""
    out = []
    if mode in ("fp64", "fp32"):
        return out
    prod = {"bf16x6": 6, "bf16x3": 3, "fp16x3": 3, "fp16x6": 6}[mode]
    tpeak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or 1400.0
    hpeak = pk.get("hbm_gbs") or 6400.0
    for name, (launches, ms) in sorted(kstats.items(), key=lambda kv: -kv[1][1]):
        if ms <= 0:
            continue
        c = kernel_cmacs(name, p)
        if c is not None and name.startswith("tc_gemm"):
            ach = 8.0 * prod * c[0] * steps / (ms / 1e3) / 1e12
            out.append({"kernel": name, "bound": "tensor", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s",
                        "frac": ach / tpeak, "ms_per_step": ms / steps})
            continue
        b = kernel_bytes(name, p)
        if b is not None:
            ach = b[0] * steps / (ms / 1e3) / 1e9
            out.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": hpeak, "unit": "GB/s",
                        "frac": ach / hpeak, "ms_per_step": ms / steps, "per_unit": b[1]})
    return out


def kernel_cmacs(name, p):
    """Complex MACs one step asks of a kernel family (the per-unit counts of
    the contraction each family runs, times the units per step)."""
    n, nb, tp = p.nv, p.nb, p.nt * p.np_
    P2 = n * (n - 1) // 2
    table = {
        "tc_gemm_step_i": (12.0 * nb * n ** 4 * tp, "12 N_B N_v^4 per (t,p): i contraction, 12 spin blocks, all (k,j)"),
        "tc_gemm_step_j": (24.0 * nb * n ** 4 * tp, "24 N_B N_v^4 per (t,p): j contraction, 6 spin pairs, K = 4 N_v"),
        "tc_gemm_source": (5.0 * nb * P2 * n * n * tp, "5 N_B C(N_v,2) N_v^2 per (t,p): k' contraction"),
        "tc_gemm_elementals": (3.0 * p.V3 * p.T3 * tp, "3 V3 C(N_v,3) per (t,p): useful i<j<k MACs"),
        "elementals_simt_f32": (3.0 * p.V3 * p.T3 * tp, "3 V3 C(N_v,3) per (t,p)"),
        "elementals_simt_f64": (3.0 * p.V3 * p.T3 * tp, "3 V3 C(N_v,3) per (t,p)"),
        "simt_gemm_f32": ((36.0 * nb * n ** 4 + 5.0 * nb * P2 * n * n) * tp, "38.5 N_B N_v^4 per (t,p)"),
        "simt_gemm_f64": ((36.0 * nb * n ** 4 + 5.0 * nb * P2 * n * n) * tp, "38.5 N_B N_v^4 per (t,p)"),
    }
    return table.get(name)


# DRAM bytes (read + write) per launch from ncu's dram__bytes_* counters of
# each tensor-core kernel family on the workload L32_Nt64_Nv128 (profiles/,
# first two timeslices: the per-launch units are those of the full size).
# Only valid for that workload and these kernels.
TRAFFIC_L32_NV128 = {
    "tc_gemm_elementals": 476.6e6 + 0.4e6,
    "tc_gemm_step_i": 696.4e6 + 1939.9e6,
    "tc_gemm_step_j": 625.1e6 + 353.5e6,
    "tc_gemm_source": 78.5e6 + 442.0e6,
    "dot": 1698.1e6 + 1.2e6,
}


def roofline(dom, kstats, p, mode, pk, steps):
    """Roofline of the dominant kernel family over the timed region."""
    if dom is None:
        return None
    launches, ms = kstats[dom]
    ent = kernel_cmacs(dom, p)
    if ent is None:
        return {"kernel": dom, "note": "no flop model"}
    cm, what = ent
    flop = 8.0 * cm * steps
    achieved = flop / (ms / 1e3) / 1e12
    if mode in ("fp64", "fp32"):
        peak = None
        bound = "alu"
        note = "CUDA-core path; peak FP32/FP64 SIMT not in MEASURED_PEAKS"
    else:
        prod = {"bf16x6": 6, "bf16x3": 3, "fp16x3": 3, "fp16x6": 6}[mode]
        peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or 1400.0
        achieved *= prod   # issued 16-bit tensor flops
        bound = "tensor"
        note = (f"achieved = 8 x {prod} split products x complex MACs / event time: tensor flops the "
                f"kernel must issue; peak = measured bf16 sustained (fp16 runs at the same rate)")
    traffic = TRAFFIC_L32_NV128.get(dom) if (p.L, p.nv, p.np_, p.nb) == (32, 128, 5, 6) and mode == "fp16x6" else None
    return {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if peak else None, "traffic": traffic, "per_unit": what,
            "launches": launches, "ms": ms, "note": note}


def parity_slice(p, v_h, tau_h, C_gpu, mode):
    """FP64 oracle on (t=1, p=0), source profile b = 0, of this run's inputs
    vs the benchmarked C (column b = 0 of C_ab)."""
    try:
        from oracle import nucleon as orc
        t = 1 if p.nt > 1 else 0
        mom0 = p.mom[:1]
        phi0 = orc.elementals_t(v_h[0], p.L, mom0)[0]
        phit = orc.elementals_t(v_h[t], p.L, mom0)[0]
        ref = orc.correlator_tp(phit, phi0, tau_h[t], p.prof, p.prof, bs=[0])[:, 0]
        got = C_gpu[0, :, 0, t]
        err = np.abs(got - ref) / np.abs(ref)
        return {"slice": f"t={t}, p=0, b=0, all a", "max_rel_err": float(err.max()),
                "scaled_err": float(np.abs(got - ref).max() / np.abs(ref).max()),
                "normwise": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
    except Exception as e:  # report, never hide
        return {"error": repr(e)}


# --------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, one
    (t, p = 0) slice of the same workload per step (untimed warm-up slices
    first), entries/s = N_B^2 per slice / mean timed slice time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cid = 3 if args.workload == 4 else args.workload
    o = OracleSlices(cid, args.nt)
    p = o.p
    times = []
    for i in range(args.warmup + args.steps):
        t = 1 + i % (p.nt - 1) if p.nt > 1 else 0
        dt = o.slice(t)
        log(f"reference slice t={t}: {dt:.1f} s")
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.mean(times)
    val = p.nb * p.nb / (ms / 1e3)
    cb = {"value": val, "unit": METRIC, "cores": o.cores(), "kind": "oracle",
          "sample": f"{args.steps} timed (t, p=0) slices after {args.warmup} untimed: sink elementals + "
                    f"C_ab(t) each, plus 1/N_t of the t=0 source elementals ({o.src_s:.1f} s)"}
    return {"metric": METRIC, "value": val, "unit": "entries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": p.name, "L": p.L, "nt": p.nt, "nv": p.nv, "np": p.np_, "nb": p.nb},
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", type=int, default=3, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--mode", default="auto")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32/FP64 comparison")
    ap.add_argument("--ncfg", type=int, default=4,
                    help="workload 4: configurations in the ensemble (16 in full; each holds 3-6 GB of inputs)")
    ap.add_argument("--nt", type=int, default=0,
                    help="keep only the first NT timeslices (profiling a smaller case; not a bench number)")
    args = ap.parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    elif args.workload == 4:
        out = run_ensemble(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
