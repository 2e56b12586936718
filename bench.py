#!/usr/bin/env python
"""Throughput of the distilled-nucleon hot path on B300.

The metric is C_ab(t) entries per second; algorithmic TFLOP/s, the
end-to-end rate through the public API (host inputs in, C out), the
roofline of every kernel family and of the whole step, parity against
stored FP64 oracle values, the oracle's own rate on the host cores and the
plain FP32/FP64 CUDA-core paths are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 1..5]
                    [--mode auto|fp16x6|fp16x3|bf16x6|bf16x3|fp32|fp64]
                    [--impl ours|reference] [--ncfg K] [--nt NT]
                    [--no-cpu-baseline] [--no-parity] [--no-plain]

--meson charm times the one-meson path instead (L=24, N_t=48, N_v=200,
3 Gammas x 7 profiles, pruned to 8 x 8): one step = one configuration.
--glueball charm times the A1-+ glueball operators on the same links.

Default: workload 5 (L=48, N_t=96, N_v=256, 9 momenta, 8 profiles), mode
fp16x6, one step = one sink timeslice of it (elementals of every momentum,
C_ab(t) for every (p, a, b), the GEVP of C(t) with eigenvectors), 3 warm-up
and 3 timed steps.  Workloads 1-3 time one whole configuration per step;
workload 4 runs an ensemble of --ncfg configurations with uneven N_v as one
graph-captured plan.  --impl reference times the FP64 oracle.

--gpus N without a launcher starts N ranks under torch.distributed.run.
With N ranks, workload 5 gives rank r the timeslices t = r mod N and
workloads 1-4 the configurations c = r mod N: weak scaling, no collective
on the data path; entries are summed over ranks and the time is the
slowest rank's; C is gathered on rank 0 after the run.  Rank 0 prints one
JSON line.
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
    cid, cfg, jobs, shm_name, shape, dtype = args
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    out = np.ndarray(shape, dtype=dtype, buffer=shm.buf)
    p = synth.config(cid, cfg)
    for slot, t in jobs:
        out[slot] = p.eigvecs(t)
    del out
    shm.close()
    return len(jobs)


def make_inputs(cid: int, cfg: int, workers: int, nt: int = 0, ts=None, npm: int = 0):
    """Host inputs of one configuration (numpy, identical bytes to the tests).
    Timeslices are drawn in parallel processes straight into shared memory.
    nt > 0 keeps only the first nt timeslices (a smaller case of the same
    shapes, for profilers); ts, a list of timeslices, draws exactly those
    (v[s] and tau[s] belong to timeslice ts[s])."""
    p = synth.config(cid, cfg)
    if nt > 0:
        p = dataclasses.replace(p, nt=min(p.nt, nt))
    if npm > 0:
        p = dataclasses.replace(p, mom=p.mom[:npm])
    ts = list(range(p.nt)) if ts is None else list(ts)
    shape = (len(ts), p.nv, p.V3, 3)
    dtype = np.dtype(p.dtype)
    if workers > 1 and len(ts) > 1:
        import multiprocessing as mp
        from multiprocessing import shared_memory
        shm = shared_memory.SharedMemory(create=True, size=int(np.prod(shape)) * dtype.itemsize)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"   # one BLAS thread per worker process (inherited at spawn)
        try:
            jobs = list(enumerate(ts))
            chunks = [jobs[w::workers] for w in range(workers)]
            with mp.get_context("spawn").Pool(workers) as pool:
                pool.map(_eig_worker, [(cid, cfg, c, shm.name, shape, dtype.str) for c in chunks if c])
            v = np.array(np.ndarray(shape, dtype=dtype, buffer=shm.buf))
        finally:
            shm.close()
            shm.unlink()
    else:
        v = np.stack([p.eigvecs(t) for t in ts])
    tau = np.stack([p.perambulator(t) for t in ts])
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
    p, v_h, tau_h = make_inputs(cid, rank, workers, args.nt, npm=args.np)   # before any CUDA call
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


def shard_timeslices(nt: int, rank: int, world: int, count: int) -> list:
    """The `count` sink timeslices rank `rank` processes, one per step: its
    share t = rank, rank + world, ... of the N_t timeslices of a
    configuration (every timeslice is independent given the source
    elementals at t0 = 0, which each rank computes itself), repeated
    cyclically when count exceeds the share."""
    mine = [t for t in range(nt) if t % world == rank] or [rank % nt]
    return [mine[i % len(mine)] for i in range(count)]


def gather_columns(C_local, ts_local, dist=None):
    """Rank 0 collects the C columns (timeslices) every rank computed after
    the run: returns {t: C[..., t]} on rank 0 (None elsewhere)."""
    cols = {int(t): C_local[..., t].copy() for t in sorted(set(ts_local))}
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return cols
    parts = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(cols, parts, dst=0)
    if dist.get_rank() != 0:
        return None
    merged = {}
    for part in parts:
        merged.update(part)
    return merged


def elementals_issued_cmacs(p) -> float:
    """Complex MACs the elementals GEMM issues for one timeslice (all
    momenta): 128 x NT tiles of pairs (j-major) x (i, momentum) rows, NT =
    128 (32 or 64 for fewer than 65 rows), over K = 3 V3 (each 4096-value
    chunk padded to a multiple of 64), minus the tiles the kernel skips
    because every i of the tile is >= every j."""
    n, npm = p.nv, p.np_
    pairs = [(j, k) for j in range(n) for k in range(j + 1, n)]
    P2, R = len(pairs), n * npm
    nt_tile = 128 if R > 64 else (64 if R > 32 else 32)
    K = 3 * p.V3
    kpad = sum(-(-min(4096, K - k0) // 64) * 64 for k0 in range(0, K, 4096))
    tiles = 0
    for m in range(-(-P2 // 128)):
        jmax = pairs[min(m * 128 + 127, P2 - 1)][0]
        for nn in range(-(-R // nt_tile)):
            if (nn * nt_tile) // npm < jmax:
                tiles += 1
    return float(tiles) * 128 * nt_tile * kpad


def golden_C(name: str):
    """Stored FP64 oracle values of a workload (tests/golden, written by
    make_oracle_golden.py from the oracle alone): {(t, p): C [nb][nb]}."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    out = {}
    for smp in d["samples"]:
        c = np.asarray(smp["C"], dtype=np.float64)
        out[(smp["t"], smp["p"])] = c[..., 0] + 1j * c[..., 1]
    return out


def run_timeslices(args):
    """One step = one sink timeslice t of the workload (default L = 48,
    N_t = 96, N_v = 256, 9 momenta, 8 profiles): its elementals for every
    momentum, the correlation matrix C_ab(t) for every (p, a, b) from the
    source elementals at t0 = 0, and the GEVP of C(t) against C(t0) with
    eigenvectors.  Every timeslice costs the same, so K steps are K / N_t of
    the configuration: the source elementals are the sink elementals of
    t = 0, computed once before the warm-up like every rank's own copy
    (the GEVP reference C(t0) too).  With N ranks, rank r takes the
    timeslices t = r mod N (weak scaling, no collective on the data path);
    the C columns are gathered on rank 0 after the run."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cid = args.workload
    p = synth.config(cid, 0)
    t0_gevp = min(2, p.nt - 1)
    steps_ts = shard_timeslices(p.nt, rank, world, args.warmup + args.steps)
    setup_ts = [0, t0_gevp]
    all_ts = setup_ts + steps_ts
    uniq = sorted(set(all_ts))
    workers = min(32, os.cpu_count() or 1)
    log(f"generating {len(uniq)} timeslices of workload {cid} ({p.name}) with {workers} processes")
    p, v_h, tau_h = make_inputs(cid, 0, workers, ts=uniq)   # before any CUDA call
    slot = {t: i for i, t in enumerate(uniq)}
    log(f"inputs ready: v {v_h.nbytes / 1e9:.2f} GB for {len(uniq)} timeslices")

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
    v_pin = torch.from_numpy(np.ascontiguousarray(v_h.astype(cdt, copy=False))).pin_memory()
    del v_h
    tau_pin = torch.from_numpy(np.ascontiguousarray(tau_h.astype(cdt, copy=False))).pin_memory()
    prof_pin = torch.from_numpy(np.ascontiguousarray(p.prof)).pin_memory()
    v = v_pin.to(dev)
    tau = tau_pin.to(dev)
    prof = prof_pin.to(dev)
    stream = torch.cuda.current_stream()
    tdt = torch.complex64 if mode == "fp32" else torch.complex128
    T3 = p.T3
    phi_src = torch.empty((1, p.np_, T3), dtype=tdt, device=dev)
    phi_t = torch.empty((1, p.np_, T3), dtype=tdt, device=dev)
    C = torch.zeros((p.np_, p.nb, p.nb, p.nt), dtype=torch.complex128, device=dev)
    lam = torch.full((p.np_, p.nt, p.nb), complex("nan"), dtype=torch.complex128, device=dev)
    vecs = torch.full((p.np_, p.nt, p.nb, p.nb), complex("nan"), dtype=torch.complex128, device=dev)
    ws_e = distil.elementals_workspace(p.L, 1, p.nv, p.np_, mode)
    ws_c = distil.correlate_workspace(1, p.nv, p.np_, p.nb, mode)
    ws = torch.empty(max(ws_e, ws_c, 1), dtype=torch.uint8, device=dev)
    log(f"device: v {v.numel() * v.element_size() / 1e9:.1f} GB, workspace {ws.numel() / 1e9:.1f} GB")

    if args.tuning:
        distil.set_tuning([int(x) for x in args.tuning.split(",")], device=local)

    def step(t, vt, taut):
        distil.elementals(vt, p.L, p.mom, mode, out=phi_t, workspace=ws)
        distil.correlate_slice(phi_t[0], phi_src[0], taut, prof, prof, C, t, mode, workspace=ws)
        distil.gevp_range(C, t0_gevp, t, 1, lam=lam, vecs=vecs)

    def barrier():
        if world > 1:
            dist.barrier()

    # set-up: the source elementals (t0 = 0) and the GEVP reference C(t0)
    distil.elementals(v[slot[0]:slot[0] + 1], p.L, p.mom, mode, out=phi_src, workspace=ws)
    step(t0_gevp, v[slot[t0_gevp]:slot[t0_gevp] + 1], tau[slot[t0_gevp]])
    torch.cuda.synchronize()
    for i in range(args.warmup):
        t = steps_ts[i]
        step(t, v[slot[t]:slot[t] + 1], tau[slot[t]])
        torch.cuda.synchronize()
        log(f"warm-up step {i} (t = {t}) done")
    timed_ts = steps_ts[args.warmup:]

    # ---------------- timed region (device-resident inputs)
    distil.profile_enable(timing=True, device=local)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly the timed launches
    for t in timed_ts:
        step(t, v[slot[t]:slot[t] + 1], tau[slot[t]])
    torch.cuda.nvtx.range_pop()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    log(f"timed region: {ms / args.steps:.1f} ms per step (one timeslice)")
    kstats = distil.profile_read(device=local)
    distil.profile_enable(timing=False, device=local)
    entries = p.np_ * p.nb * p.nb          # one timeslice per step
    value, all_entries, ms_max = job_throughput(entries, ms, args.steps, dist if world > 1 else None, dev)
    ms_step = ms_max / args.steps

    # ---------------- end to end: host v(t), tau(t) in, C and lambda out, every step
    e2e_steps = max(1, min(args.steps, 3))
    v_in = torch.empty_like(v[:1])
    tau_in = torch.empty_like(tau[0])
    C_host = torch.empty(C.shape, dtype=C.dtype).pin_memory()
    lam_host = torch.empty(lam.shape, dtype=lam.dtype).pin_memory()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for t in timed_ts[:e2e_steps]:
        v_in.copy_(v_pin[slot[t]:slot[t] + 1], non_blocking=True)
        tau_in.copy_(tau_pin[slot[t]], non_blocking=True)
        step(t, v_in, tau_in)
        C_host.copy_(C, non_blocking=True)
        lam_host.copy_(lam, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_value, _, _ = job_throughput(entries, e0.elapsed_time(e1), e2e_steps, dist if world > 1 else None, dev)
    h2d = v_pin[0].numel() * v_pin.element_size() + tau_pin[0].numel() * tau_pin.element_size()
    d2h = C_host.numel() * 16 + lam_host.numel() * 16

    C_np = C.cpu().numpy()
    gathered = gather_columns(C_np, [t0_gevp] + list(steps_ts), dist if world > 1 else None)
    plain = None
    if rank == 0 and not args.no_plain and mode not in ("fp64", "fp32"):
        mid, late = p.nt // 2, p.nt - 1
        plain = plain_paths_slices(distil, p, cid, [mid, late], prof, dev)
    out = None
    if rank == 0:
        pk = peaks()
        flops = algorithmic_flops(dataclasses.replace(p, nt=1))
        dom = max(kstats.items(), key=lambda kv: kv[1][1])[0] if kstats else None
        p1 = dataclasses.replace(p, nt=1)
        roof = roofline(dom, kstats, p1, mode, pk, args.steps)
        launches = sum(l for l, _ in kstats.values())
        gold = golden_C(p.name)
        parity = None
        if gold is not None and not args.no_parity:
            errs = {}
            for (t, q), ref in gold.items():
                if t in gathered:
                    got = gathered[t][q]
                    e = np.abs(got - ref) / np.abs(ref)
                    errs[f"t={t},p={q}"] = {"max_rel_err": float(e.max()),
                                             "scaled_err": float(np.abs(got - ref).max() / np.abs(ref).max())}
            parity = {"reference": "stored FP64 oracle values (tests/golden)", "slices": errs,
                      "max_rel_err": max((x["max_rel_err"] for x in errs.values()), default=None)}
        cpu = None if args.no_cpu_baseline else cpu_baseline_sampled(cid)
        out = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32"}.get(mode, mode + "(f32 accumulate)"),
            "data": "synthetic (seeded orthonormal eigenvectors, Gaussian perambulators)",
            "config": {"workload": p.name, "L": p.L, "nt": p.nt, "nv": p.nv, "np": p.np_, "nb": p.nb,
                       "mode": mode, "step": "one sink timeslice: elementals (all momenta), C_ab(t) for all "
                                             "(p, a, b), GEVP with eigenvectors",
                       "parallelism": f"weak x{world} (timeslice t on rank t mod N)",
                       "l2": "inputs larger than L2 (v(t) is %.2f GB per timeslice)"
                             % (v[0].numel() * v.element_size() / 1e9)},
            "tflops_algorithmic": flops["total"] * world / (ms_step / 1e3) / 1e12,
            "e2e": {"value": e2e_value, "unit": "entries/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "kernels": {k: {"launches": l, "ms": round(t, 3)} for k, (l, t) in sorted(kstats.items(),
                                                                                  key=lambda kv: -kv[1][1])},
            "roofline": roof,
            "kernel_rooflines": kernel_rooflines(kstats, p1, mode, pk, args.steps),
            "whole_step": whole_step_tensor(kstats, p1, mode, pk, args.steps, ms_step),
            "tuning": distil.get_tuning(device=local),
            "clocks": clk,
            "parity": parity,
            "cpu_baseline": cpu,
            "plain_paths": plain,
            "gathered_timeslices": len(gathered) if gathered is not None else 0,
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def whole_step_tensor(kstats, p, mode, pk, steps, ms_step):
    """Tensor flops the step's contraction kernels issue (elementals tiles
    including the triangle-test waste, the three mode contractions) over the
    whole step time, against the measured sustained bf16 peak."""
    if mode in ("fp64", "fp32"):
        return None
    n, nb, P2 = p.nv, p.nb, p.nv * (p.nv - 1) // 2
    flop = 8.0 * (split_products(mode, "tc_gemm_elementals") * elementals_issued_cmacs(p) * p.nt
                  + split_products(mode) * (36.0 * nb * n ** 4 + 5.0 * nb * P2 * n * n) * p.nt * p.np_)
    peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or 1400.0
    ach = flop / (ms_step / 1e3) / 1e12
    return {"issued_tflop_per_step": flop / 1e12, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "note": "issued split-product tensor flops of every contraction kernel / step time"}


def plain_paths_slices(distil, p, cid, ts, prof, dev):
    """The plain FP32 (all momenta) and FP64 (first momentum) CUDA-core paths
    of the library on the same GPU, on the given sink timeslices with the
    source at t0 = 0: elementals + C_ab(t), entries/s per timeslice."""
    import torch
    out = {}
    _, v_h, tau_h = make_inputs(cid, 0, 1, ts=[0] + list(ts))
    for mode, cdt, moms in (("fp32", np.complex64, p.mom), ("fp64", np.complex128, p.mom[:1])):
        v1 = torch.from_numpy(np.ascontiguousarray(v_h.astype(cdt))).to(dev)
        t1 = torch.from_numpy(np.ascontiguousarray(tau_h.astype(cdt))).to(dev)
        npm = len(moms)
        src = distil.elementals(v1[:1], p.L, moms, mode)
        C = torch.zeros((npm, p.nb, p.nb, p.nt), dtype=torch.complex128, device=dev)
        res = {}
        for i, t in enumerate(ts):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            phi = distil.elementals(v1[i + 1:i + 2], p.L, moms, mode)
            distil.correlate_slice(phi[0], src[0], t1[i + 1], prof, prof, C, t, mode)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            res[f"t={t}"] = {"value": npm * p.nb * p.nb / (ms / 1e3), "ms": ms}
        out[mode] = {"unit": "entries/s", "momenta": npm, "timeslices": res,
                     "sample": f"sink timeslices {list(ts)}, {npm} momenta, source at t0 = 0"}
        del v1, t1, src, C
    log("plain paths: " + "; ".join(f"{m} " + ", ".join(f"{k} {r['value']:.2f}" for k, r in o["timeslices"].items())
                                    for m, o in out.items()))
    return out


def cpu_baseline_sampled(cid: int, m_el: int = 64, m_co: int = 96) -> dict:
    """The FP64 oracle on a bounded sample of one (t, p = 0) slice of the
    workload: the elementals of the first m_el modes (cost grows as N_v^3)
    and the correlation matrix of the first m_co modes for one source profile
    (cost grows as N_v^4 per profile), each scaled to the full N_v and N_B;
    the slice's N_B^2 entries over the scaled time."""
    from oracle import nucleon as orc
    p = synth.config(cid, 0)
    mom0 = p.mom[:1]
    v1 = p.eigvecs(1).astype(np.complex128)
    tau1 = p.perambulator(1).astype(np.complex128)
    t_a = time.perf_counter()
    orc.elementals_t(v1[:m_el], p.L, mom0)
    el_s = time.perf_counter() - t_a
    m = m_co
    sub = np.concatenate([np.arange(a * p.nv, a * p.nv + m) for a in range(4)])
    phi_m = orc.elementals_t(v1[:m], p.L, mom0)[0]
    t_b = time.perf_counter()
    orc.correlator_tp(phi_m, phi_m, tau1[np.ix_(sub, sub)], p.prof[:, :m], p.prof[:, :m], bs=[0])
    co_s = time.perf_counter() - t_b
    slice_s = el_s * (p.nv / m_el) ** 3 + co_s * (p.nv / m) ** 4 * p.nb
    return {"value": p.nb * p.nb / slice_s, "unit": METRIC, "cores": OracleSlices.cores(), "kind": "oracle",
            "sample": f"one (t=1, p=0) slice scaled from the oracle's elementals of {m_el} of {p.nv} modes "
                      f"({el_s:.1f} s, x{(p.nv / m_el) ** 3:.0f}) and its correlator of {m} modes for one of "
                      f"{p.nb} source profiles ({co_s:.1f} s, x{(p.nv / m) ** 4 * p.nb:.0f}); numpy FP64, "
                      f"BLAS threads", "seconds": el_s + co_s, "slice_seconds_scaled": slice_s}


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
        # Z (nb x P2 x n complex double-float) read once
        "dot": (16.0 * nb * P2 * n * tp, "Z per (t,p), 16 B per element"),
        # V read once (nb x 6 spin pairs x n^3 x 16 B), the W planes written (nb x P2 x 5n x 12 B)
        "split_w": ((96.0 * nb * n ** 3 + 60.0 * nb * P2 * n) * tp, "V read + W planes written per (t,p)"),
        # the cross-product planes written once: P2 x 3 V3 x 16 B (eight 16-bit planes) per timeslice
        "split_pairs": (16.0 * P2 * 3 * p.V3 * p.nt, "C(N_v,2) x 3 V3 x 16 B per t written"),
    }
    return table.get(name)


def kernel_rooflines(kstats, p, mode, pk, steps):
    """Every contraction kernel against the tensor peak (issued split
    products) and the memory-side kernels against the measured HBM copy
    bandwidth; achieved from the summed CUDA-event time over `steps` steps."""
    out = []
    if mode in ("fp64", "fp32"):
        return out
    tpeak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or 1400.0
    hpeak = pk.get("hbm_gbs") or 6400.0
    for name, (launches, ms) in sorted(kstats.items(), key=lambda kv: -kv[1][1]):
        if ms <= 0:
            continue
        c = kernel_cmacs(name, p)
        if c is not None and name.startswith("tc_gemm"):
            ach = 8.0 * split_products(mode, name) * c[0] * steps / (ms / 1e3) / 1e12
            out.append({"kernel": name, "bound": "tensor", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s",
                        "frac": ach / tpeak, "ms_per_step": ms / steps})
            continue
        b = kernel_bytes(name, p)
        if b is not None:
            ach = b[0] * steps / (ms / 1e3) / 1e9
            out.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": hpeak, "unit": "GB/s",
                        "frac": ach / hpeak, "ms_per_step": ms / steps, "per_unit": b[1]})
    return out


def split_products(mode, kernel=None) -> int:
    """Real 16-bit products per complex MAC pair the tensor-core kernels issue:
    the FP16X6 elementals keep eight split products, the other FP16X6 and
    BF16X6 contractions six, the X3 modes three.  The six-product step-j and
    T contractions run as two passes of three (leading classes, then the
    second-order terms: kernels <name> and <name>_2nd)."""
    if mode == "fp16x6" and kernel == "tc_gemm_elementals":
        return 8
    six = mode in ("fp16x6", "bf16x6")
    if six and kernel in ("tc_gemm_step_j", "tc_gemm_tcontract", "tc_gemm_step_j_2nd", "tc_gemm_tcontract_2nd"):
        return 3
    return {"bf16x6": 6, "bf16x3": 3, "fp16x3": 3, "fp16x6": 6}[mode]


def kernel_cmacs(name, p):
    """Complex MACs one step asks of a kernel family (the per-unit counts of
    the contraction each family runs, times the units per step)."""
    n, nb, tp = p.nv, p.nb, p.nt * p.np_
    P2 = n * (n - 1) // 2
    table = {
        "tc_gemm_step_i": (12.0 * nb * n ** 4 * tp, "12 N_B N_v^4 per (t,p): i contraction, 12 spin blocks, all (k,j)"),
        "tc_gemm_step_j": (24.0 * nb * n ** 4 * tp, "24 N_B N_v^4 per (t,p): j contraction, 6 spin pairs, K = 4 N_v"),
        "tc_gemm_step_j_2nd": (24.0 * nb * n ** 4 * tp, "24 N_B N_v^4 per (t,p): second-order pass of step j"),
        "tc_gemm_tcontract": (5.0 * nb * P2 * n * n * tp,
                              "5 N_B C(N_v,2) N_v^2 per (t,p): T^c contraction of W, K = 5 N_v"),
        "tc_gemm_tcontract_2nd": (5.0 * nb * P2 * n * n * tp,
                                  "5 N_B C(N_v,2) N_v^2 per (t,p): second-order pass of the T contraction"),
        "tc_gemm_elementals": (3.0 * p.V3 * p.T3 * tp, "3 V3 C(N_v,3) per (t,p): useful i<j<k MACs"),
        "elementals_simt_f32": (3.0 * p.V3 * p.T3 * tp, "3 V3 C(N_v,3) per (t,p)"),
        "elementals_simt_f64": (3.0 * p.V3 * p.T3 * tp, "3 V3 C(N_v,3) per (t,p)"),
        "simt_gemm_f32": ((36.0 * nb * n ** 4 + 5.0 * nb * P2 * n * n) * tp, "38.5 N_B N_v^4 per (t,p)"),
        "simt_gemm_f64": ((36.0 * nb * n ** 4 + 5.0 * nb * P2 * n * n) * tp, "38.5 N_B N_v^4 per (t,p)"),
    }
    return table.get(name)


# DRAM bytes (read + write) per launch of a kernel family, from one ncu
# capture of the kernels as they stand: (workload, mode, kernel) -> bytes.
# The L48_Nt96_Nv256 elementals launch is too large to capture with
# --set full; its figure is the L32_Nv128 one-timeslice capture of the
# bulk-copy kernel (539.3 MB read, 3.3 MB written,
# profiles/tc_gemm_L32_Nv128_one_timeslice.md) scaled by the operand units
# of a launch, (pairs + (i, p) rows) x K chunk: x 4.23.
TRAFFIC = {
    ("L48_Nt96_Nv256", "fp16x6", "tc_gemm_elementals"): 542.6e6 * (32640 + 2304) / (8128 + 128),
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
        prod = split_products(mode, dom)
        peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or 1400.0
        achieved *= prod   # issued 16-bit tensor flops
        bound = "tensor"
        note = (f"achieved = 8 x {prod} split products x complex MACs / event time: tensor flops the "
                f"kernel must issue; peak = measured bf16 sustained (fp16 runs at the same rate)")
    traffic = TRAFFIC.get((p.name, mode, dom))
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
    """The reference arm: the FP64 oracle as it stands on the host cores.
    Workloads 1-4: one (t, p = 0) slice of the workload per step (untimed
    warm-up slices first).  Workload 5 (one slice takes many minutes): each
    step is a bounded sample of the slice (t = 1, p = 0) -- the oracle's
    elementals of the first 40 modes and its correlator of the first 96
    modes for one source profile (cycling through the profiles), scaled to
    the full slice by N_v^3 and N_B N_v^4 (about 6 s per step on 16 cores).
    entries/s = N_B^2 per slice / mean (scaled) slice time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cid = 3 if args.workload == 4 else args.workload
    times = []
    if cid == 5:
        from oracle import nucleon as orc
        p = synth.config(cid, 0)
        if args.nt > 0:
            p = dataclasses.replace(p, nt=min(p.nt, args.nt))
        m_el, m_co = 40, 96
        mom0 = p.mom[:1]
        v1 = p.eigvecs(1).astype(np.complex128)
        tau1 = p.perambulator(1).astype(np.complex128)
        sub = np.concatenate([np.arange(a * p.nv, a * p.nv + m_co) for a in range(4)])
        tau_m = tau1[np.ix_(sub, sub)]
        phi_m = orc.elementals_t(v1[:m_co], p.L, mom0)[0]       # input of the correlator sample (untimed)
        g_m = np.ascontiguousarray(p.prof[:, :m_co])
        for i in range(args.warmup + args.steps):
            t_a = time.perf_counter()
            orc.elementals_t(v1[:m_el], p.L, mom0)
            el_s = time.perf_counter() - t_a
            t_b = time.perf_counter()
            orc.correlator_tp(phi_m, phi_m, tau_m, g_m, g_m, bs=[i % p.nb])
            co_s = time.perf_counter() - t_b
            dt = el_s * (p.nv / m_el) ** 3 + co_s * (p.nv / m_co) ** 4 * p.nb
            log(f"reference sample {i}: {el_s + co_s:.1f} s, scaled slice {dt:.0f} s")
            if i >= args.warmup:
                times.append(dt)
        sample = (f"{args.steps} timed samples after {args.warmup} untimed, each the (t=1, p=0) slice scaled from "
                  f"the oracle's elementals of {m_el} of {p.nv} modes (x{(p.nv / m_el) ** 3:.0f}) and its "
                  f"correlator of {m_co} modes for one of {p.nb} source profiles (x{(p.nv / m_co) ** 4 * p.nb:.0f})")
    else:
        o = OracleSlices(cid, args.nt)
        p = o.p
        for i in range(args.warmup + args.steps):
            t = 1 + i % (p.nt - 1) if p.nt > 1 else 0
            dt = o.slice(t)
            log(f"reference slice t={t}: {dt:.1f} s")
            if i >= args.warmup:
                times.append(dt)
        sample = (f"{args.steps} timed (t, p=0) slices after {args.warmup} untimed: sink elementals + "
                  f"C_ab(t) each, plus 1/N_t of the t=0 source elementals ({o.src_s:.1f} s)")
    ms = 1e3 * statistics.mean(times)
    val = p.nb * p.nb / (ms / 1e3)
    cb = {"value": val, "unit": METRIC, "cores": OracleSlices.cores(), "kind": "oracle", "sample": sample}
    return {"metric": METRIC, "value": val, "unit": "entries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": p.name, "L": p.L, "nt": p.nt, "nv": p.nv, "np": p.np_, "nb": p.nb},
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# --------------------------------------------------------------------------- mesons

MESON_METRIC = "meson C_ab(t) entries/s"


def _meson_eig_worker(args):
    which, cfg, jobs, shm_name, shape, dtype = args
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    out = np.ndarray(shape, dtype=dtype, buffer=shm.buf)
    m = synth.meson_config(which, cfg)
    for slot, t in jobs:
        out[slot] = m.eigvecs(t)
    del out
    shm.close()
    return len(jobs)


def meson_inputs(which: str, cfg: int, workers: int, nt: int = 0):
    """Host inputs of one meson configuration: v, U, tau (numpy, the bytes the
    tests draw); the eigenvectors in parallel spawned processes.  nt > 0
    keeps the first nt timeslices (a smaller case for profilers)."""
    m = synth.meson_config(which, cfg)
    if nt > 0:
        m.base = dataclasses.replace(m.base, nt=min(nt, m.nt))
    shape = (m.nt, m.nv, m.V3, 3)
    dtype = np.dtype(m.dtype)
    if workers > 1 and m.nt > 1:
        import multiprocessing as mp
        from multiprocessing import shared_memory
        shm = shared_memory.SharedMemory(create=True, size=int(np.prod(shape)) * dtype.itemsize)
        try:
            jobs = list(enumerate(range(m.nt)))
            chunks = [jobs[w::workers] for w in range(workers)]
            with mp.get_context("spawn").Pool(workers) as pool:
                pool.map(_meson_eig_worker, [(which, cfg, c, shm.name, shape, dtype.str) for c in chunks if c])
            v = np.array(np.ndarray(shape, dtype=dtype, buffer=shm.buf))
        finally:
            shm.close()
            shm.unlink()
    else:
        v = m.all_eigvecs()
    return m, v, m.all_links(), m.all_perambulators()


def meson_cmacs(name, m):
    """Complex MACs one configuration asks of each meson contraction family."""
    n, nops, V3 = m.nv, 3 * m.nb, m.V3
    table = {
        "tc_gemm_meson_elem": (7.0 * n * m.np_ * n * 3 * V3 * m.nt,
                               "7 N_p N_v^2 3 V3 per timeslice: all displacements d, all (i, j)"),
        "tc_gemm_meson_q": (nops * 64.0 * n ** 3 * m.np_ * m.nt,
                            "3 N_B (4 N_v)^3 per (t, p): Q_b = Phibar_b g5 tau^dagger g5, dense spin-mode"),
        "tc_gemm_meson_x": (nops * 64.0 * n ** 3 * m.np_ * m.nt, "3 N_B (4 N_v)^3 per (t, p): X_b = tau Q_b"),
    }
    return table.get(name)


def meson_split_products(name) -> int:
    return 8 if name == "tc_gemm_meson_elem" else 6


def meson_bytes(name, m):
    """Algorithmic HBM bytes per configuration of the memory-side families."""
    n, nops, V3, nt = m.nv, 3 * m.nb, m.V3, m.nt
    table = {
        "meson_nabla": ((8.0 * n * 3 * V3 + 3 * 72.0 * V3 + 3 * 16.0 * n * 3 * V3) * nt,
                        "v (8 B) and the links read, three nabla fields (16 B) written, per t"),
        "meson_bb": (2 * 3 * 16.0 * n * 3 * V3 * nt,
                     "three nabla fields read, three BB fields written (16 B per value) per t"),
        "meson_reduce": (16.0 * nops * 16 * n * n * m.np_ * nt, "X (3 N_B (4 N_v)^2 x 16 B) read per (t, p)"),
    }
    return table.get(name)


# DRAM bytes (read + write) per launch of the meson elementals GEMM, from one
# ncu capture of the L=24, N_v=200 workload cut to 4 timeslices (one 4032-long
# K chunk of 4 timeslices: 443.8 MB read, 3.9 MB written, the operand planes of
# the chunk and the accumulator) scaled by the timeslices of a bench launch
# (16 per batch): x 4.
MESON_TRAFFIC = {("L24_Nt48_Nv200_meson", "tc_gemm_meson_elem"): (443.8e6 + 3.9e6) * 16 / 4}


def meson_rooflines(kstats, m, pk, steps):
    tpeak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or 1400.0
    hpeak = pk.get("hbm_gbs") or 6400.0
    out = []
    for name, (launches, ms) in sorted(kstats.items(), key=lambda kv: -kv[1][1]):
        if ms <= 0:
            continue
        c = meson_cmacs(name, m)
        if c is not None:
            ach = 8.0 * meson_split_products(name) * c[0] * steps / (ms / 1e3) / 1e12
            out.append({"kernel": name, "bound": "tensor", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s",
                        "frac": ach / tpeak, "ms_per_step": ms / steps, "launches": launches,
                        "per_unit": c[1], "split_products": meson_split_products(name)})
            continue
        b = meson_bytes(name, m)
        if b is not None:
            ach = b[0] * steps / (ms / 1e3) / 1e9
            out.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": hpeak, "unit": "GB/s",
                        "frac": ach / hpeak, "ms_per_step": ms / steps, "launches": launches, "per_unit": b[1]})
    return out


def meson_cpu_baseline(m, v, U, tau, t: int = 1):
    """The meson oracle, as it stands, on one sink timeslice of the workload:
    its elementals and its C_ab(t) (the t = 0 source elementals computed
    first, untimed: they serve every timeslice).  Returns the baseline entry
    and the oracle's C(t) for a parity check of that column."""
    from oracle import meson as om
    src = om.elementals_t(v[0].astype(np.complex128), U[0].astype(np.complex128), m.L, m.mom)
    t0 = time.perf_counter()
    phi = om.elementals_t(v[t].astype(np.complex128), U[t].astype(np.complex128), m.L, m.mom)
    t1 = time.perf_counter()
    C = om.correlator_t(phi, src, tau[t].astype(np.complex128), m.prof)
    t2 = time.perf_counter()
    entries = m.np_ * (3 * m.nb) ** 2
    return ({"value": entries / (t2 - t0), "unit": MESON_METRIC, "cores": OracleSlices.cores(), "kind": "oracle",
             "sample": f"one sink timeslice (t = {t}) of {m.nt}: elementals {t1 - t0:.1f} s + C_ab(t) "
                       f"{t2 - t1:.1f} s, numpy FP64 with BLAS threads (source elementals untimed)",
             "seconds": t2 - t0}, C)


def run_meson(args):
    """One step = one whole meson configuration (default L = 24, N_t = 48,
    N_v = 200, p = 0, 3 Gammas x 7 profiles): the elementals of every
    timeslice and displacement, the 21 x 21 C_ab(t) for every t, the pruning
    to 8 x 8 at t_p and the GEVP of the pruned matrix.  With N ranks rank r
    runs configuration r (weak scaling, no collective on the data path)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    which = args.meson
    workers = min(32, os.cpu_count() or 1)
    log(f"generating meson workload {which}, configuration {rank}")
    m, v_h, U_h, tau_h = meson_inputs(which, rank, workers, args.nt)   # before any CUDA call
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_2609_37723_b300 import distil
    v_pin = torch.from_numpy(np.ascontiguousarray(v_h.astype(np.complex64))).pin_memory()
    U_pin = torch.from_numpy(np.ascontiguousarray(U_h.astype(np.complex64))).pin_memory()
    tau_pin = torch.from_numpy(np.ascontiguousarray(tau_h.astype(np.complex64))).pin_memory()
    v, U, tau = v_pin.to(dev), U_pin.to(dev), tau_pin.to(dev)
    prof = torch.from_numpy(np.ascontiguousarray(m.prof)).to(dev)
    nops = 3 * m.nb
    phi = torch.empty((m.nt, m.np_, 7, m.nv, m.nv), dtype=torch.complex128, device=dev)
    C = torch.empty((m.np_, nops, nops, m.nt), dtype=torch.complex128, device=dev)
    ws_e = torch.empty(distil.meson_elementals_workspace(m.L, m.nt, m.nv, m.np_), dtype=torch.uint8, device=dev)
    ws_c = torch.empty(distil.meson_correlate_workspace(m.nv, m.np_, m.nb), dtype=torch.uint8, device=dev)
    t0_gevp = 1
    stream = torch.cuda.current_stream()
    log(f"device: v {v.numel() * 8 / 1e9:.2f} GB, workspaces {ws_e.numel() / 1e9:.2f} + {ws_c.numel() / 1e9:.2f} GB")
    res = {}

    def step(vv, UU, tt):
        distil.meson_elementals(vv, UU, m.L, m.mom, out=phi, workspace=ws_e)
        distil.meson_correlate(phi, phi[0], tt, prof, out=C, workspace=ws_c)
        Ct, Un, sv = distil.meson_prune(C, m.t_prune, m.nkeep)
        res["lam"] = distil.gevp(Ct, t0_gevp)
        res["sv"] = sv

    def barrier():
        if world > 1:
            dist.barrier()

    for i in range(args.warmup):
        step(v, U, tau)
        torch.cuda.synchronize()
        log(f"warm-up step {i} done")
    distil.profile_enable(timing=True, device=local)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        step(v, U, tau)
    torch.cuda.nvtx.range_pop()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    kstats = distil.profile_read(device=local)
    distil.profile_enable(timing=False, device=local)
    entries = m.np_ * nops * nops * m.nt
    value, _, ms_max = job_throughput(entries, ms, args.steps, dist if world > 1 else None, dev)
    ms_step = ms_max / args.steps
    log(f"timed region: {ms_step:.1f} ms per configuration")

    # end to end: host v, U, tau in and C, lambda out every step, through the same calls
    e2e_steps = max(1, min(args.steps, 2))
    v_in, U_in, tau_in = torch.empty_like(v), torch.empty_like(U), torch.empty_like(tau)
    C_host = torch.empty(C.shape, dtype=C.dtype).pin_memory()
    lam_host = torch.empty(res["lam"].shape, dtype=res["lam"].dtype).pin_memory()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        v_in.copy_(v_pin, non_blocking=True)
        U_in.copy_(U_pin, non_blocking=True)
        tau_in.copy_(tau_pin, non_blocking=True)
        step(v_in, U_in, tau_in)
        C_host.copy_(C, non_blocking=True)
        lam_host.copy_(res["lam"], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_value, _, _ = job_throughput(entries, e0.elapsed_time(e1), e2e_steps, dist if world > 1 else None, dev)
    h2d = sum(x.numel() * x.element_size() for x in (v_pin, U_pin, tau_pin))
    d2h = C_host.numel() * 16 + lam_host.numel() * 16
    out = None
    if rank == 0:
        pk = peaks()
        roofs = meson_rooflines(kstats, m, pk, args.steps)
        tens = [r for r in roofs if r["bound"] == "tensor"]
        dom = max(tens, key=lambda r: r["ms_per_step"]) if tens else None
        issued = sum(8.0 * meson_split_products(k) * meson_cmacs(k, m)[0]
                     for k in ("tc_gemm_meson_elem", "tc_gemm_meson_q", "tc_gemm_meson_x"))
        tpeak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops") or 1400.0
        cpu, parity = None, None
        if not args.no_cpu_baseline:
            cpu, C_ref = meson_cpu_baseline(m, v_h, U_h, tau_h, 1)
            if not args.no_parity:
                import importlib
                sys.path.insert(0, os.path.join(ROOT, "tests"))
                par = importlib.import_module("parity")
                got = C[..., 1:2].cpu().numpy()
                parity = {"reference": "FP64 oracle, sink timeslice t = 1 (the cpu_baseline sample)",
                          "max_operator_scaled_err": par.max_c_operator_scaled_error(got, C_ref[..., None]),
                          "max_matrix_scaled_err": par.max_c_scaled_error(got, C_ref[..., None]),
                          "max_rel_err": par.max_c_error(got, C_ref[..., None]),
                          "gate": "operator-scaled error (|dC_ab| / sqrt(R_a R_b), R = largest |C| of an "
                                  "operator's row or column) < 1e-6"}
        out = {
            "metric": MESON_METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp16x6(f32 accumulate)",
            "data": "synthetic (seeded orthonormal eigenvectors, Haar SU(3) links, Gaussian perambulators)",
            "config": {"workload": m.name, "L": m.L, "nt": m.nt, "nv": m.nv, "np": m.np_, "nb": m.nb,
                       "operators": nops, "nkeep": m.nkeep, "t_prune": m.t_prune, "t0_gevp": t0_gevp,
                       "step": "one configuration: elementals (7 displacements, all t), C_ab(t) for all t, "
                               "SVD pruning, GEVP of the pruned matrix",
                       "parallelism": f"weak x{world} (configuration r on rank r)",
                       "l2": "inputs larger than L2 (v is %.2f GB)" % (v.numel() * 8 / 1e9)},
            "e2e": {"value": e2e_value, "unit": "entries/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(sum(l for l, _ in kstats.values())),
            "kernels": {k: {"launches": l, "ms": round(t, 3)} for k, (l, t) in sorted(kstats.items(),
                                                                                  key=lambda kv: -kv[1][1])},
            "roofline": None if dom is None else {**dom, "traffic": MESON_TRAFFIC.get((m.name, dom["kernel"]))},
            "kernel_rooflines": roofs,
            "whole_step": {"issued_tflops": issued / (ms_step / 1e3) / 1e12,
                           "frac": issued / (ms_step / 1e3) / 1e12 / tpeak, "peak": tpeak,
                           "note": "split products the three contraction families issue per configuration "
                                   "over the whole step time"},
            "clocks": clk,
            "parity": parity,
            "cpu_baseline": cpu,
            "singular_values": res["sv"][0].cpu().numpy().tolist()[:12],
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


# --------------------------------------------------------------------------- glueballs

GLUE_METRIC = "glueball O_n(t) values/s"
FP64_NOMINAL_GFLOPS = 1250.0   # B300 FP64, nominal (no measured FP64 peak in the peaks file)


def glue_flops(name, L, nt):
    """FP64 flops (8 per complex multiply-add of 3 x 3 products) one
    configuration asks of each glueball kernel family, per site: clover
    3 planes x 4 plaquettes x 3 products x 27; 39 derivative fields x 4
    products x 27; traces 4 x 6 x 9 + 6 x 27 + 12 x 9."""
    V3 = L ** 3
    table = {
        "glue_clover": (8.0 * 3 * 4 * 3 * 27 * V3 * nt, "3 planes x 4 plaquettes x 3 products per site"),
        "glue_deriv": (8.0 * 39 * 4 * 27 * V3 * nt, "39 adjoint derivatives x 4 products per site"),
        "glue_trace": (8.0 * (4 * 6 * 9 + 6 * 27 + 12 * 9) * V3 * nt, "the five traces per site"),
    }
    return table.get(name)


def run_glueball(args):
    """One step = the five A1-+ glueball operators of every timeslice of one
    configuration (links of the meson workload: L = 24, N_t = 48)."""
    m = synth.meson_config(args.glueball, 0)
    if args.nt > 0:
        m.base = dataclasses.replace(m.base, nt=min(args.nt, m.nt))
    log(f"generating links of {m.name}")
    U_h = m.all_links().astype(np.complex64)
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    from paper_2609_37723_b300 import distil
    U_pin = torch.from_numpy(np.ascontiguousarray(U_h)).pin_memory()
    U = U_pin.to(dev)
    O = torch.empty((m.nt, 5), dtype=torch.complex128, device=dev)
    ws = torch.empty(distil.glueball_workspace(m.L, m.nt), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(UU):
        distil.glueball_operators(UU, m.L, out=O, workspace=ws)

    for _ in range(args.warmup):
        step(U)
    torch.cuda.synchronize()
    distil.profile_enable(timing=True, device=0)
    clocks = ClockSampler(0)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        step(U)
    torch.cuda.nvtx.range_pop()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    kstats = distil.profile_read(device=0)
    distil.profile_enable(timing=False, device=0)
    ms_step = ms / args.steps
    values = 5 * m.nt
    U_in = torch.empty_like(U)
    O_host = torch.empty(O.shape, dtype=O.dtype).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        U_in.copy_(U_pin, non_blocking=True)
        step(U_in)
        O_host.copy_(O, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e = values * e2e_steps / (e0.elapsed_time(e1) / 1e3)
    roofs = []
    for name, (launches, kms) in sorted(kstats.items(), key=lambda kv: -kv[1][1]):
        f = glue_flops(name, m.L, m.nt)
        if f is None or kms <= 0:
            continue
        ach = f[0] * args.steps / (kms / 1e3) / 1e9
        roofs.append({"kernel": name, "bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_GFLOPS,
                      "unit": "GFLOP/s (FP64)", "frac": ach / FP64_NOMINAL_GFLOPS, "ms_per_step": kms / args.steps,
                      "launches": launches, "per_unit": f[1], "peak_kind": "of nominal"})
    dom = max(roofs, key=lambda r: r["ms_per_step"]) if roofs else None
    cpu, parity = None, None
    if not args.no_cpu_baseline:
        from oracle import glueball as og
        t0 = time.perf_counter()
        ref = og.operators_t(U_h[1].astype(np.complex128), m.L)
        sec = time.perf_counter() - t0
        cpu = {"value": 5 / sec, "unit": GLUE_METRIC, "cores": OracleSlices.cores(), "kind": "oracle",
               "sample": f"one timeslice (t = 1) of {m.nt}: {sec:.1f} s, numpy FP64", "seconds": sec}
        got = O[1].cpu().numpy()
        parity = {"reference": "FP64 oracle, timeslice t = 1",
                  "max_err_rel_to_largest": float(np.abs(got - ref).max() / np.abs(ref).max())}
    return {
        "metric": GLUE_METRIC, "value": values / (ms_step / 1e3), "unit": "values/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Haar SU(3) links of the meson workload)",
        "config": {"workload": m.name.replace("meson", "glueball"), "L": m.L, "nt": m.nt,
                   "step": "one configuration: B_i, 39 adjoint derivative fields and O_1..O_5 of every timeslice",
                   "parallelism": "single GPU", "l2": "derivative fields (113 MB per timeslice) larger than L2"},
        "e2e": {"value": e2e, "unit": "values/s", "h2d_bytes_per_step": int(U_pin.numel() * 8),
                "d2h_bytes_per_step": int(O_host.numel() * 16)},
        "gpu_launches": int(sum(l for l, _ in kstats.values())),
        "kernels": {k: {"launches": l, "ms": round(t, 3)} for k, (l, t) in kstats.items()},
        "roofline": None if dom is None else {**dom, "traffic": None},
        "kernel_rooflines": roofs,
        "clocks": clk, "parity": parity, "cpu_baseline": cpu,
    }


def spawn_ranks(n: int) -> int:
    """bench.py --gpus N run without a launcher: start N ranks of this script
    under torch.distributed.run on this node (127.0.0.1) and return its exit
    status."""
    import socket
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", type=int, default=5, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--mode", default="auto")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32/FP64 comparison")
    ap.add_argument("--ncfg", type=int, default=4,
                    help="workload 4: configurations in the ensemble (16 in full; each holds 3-6 GB of inputs)")
    ap.add_argument("--tuning", default="",
                    help="kernel variants of the three contraction sites, e.g. 0,0,0 (default: the library's)")
    ap.add_argument("--nt", type=int, default=0,
                    help="keep only the first NT timeslices (profiling a smaller case; not a bench number)")
    ap.add_argument("--meson", default=None, choices=["charm", "small"],
                    help="time the one-meson path on this workload instead (charm: L=24, N_t=48, N_v=200)")
    ap.add_argument("--glueball", default=None, choices=["charm", "small", "tiny"],
                    help="time the A1-+ glueball operators on the links of this meson workload")
    ap.add_argument("--np", type=int, default=0,
                    help="workloads 1-3: keep only the first NP momenta (profiling a smaller case; not a bench number)")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args.gpus))
    if args.warmup < 3 and args.impl == "ours" and (args.workload == 5 or args.meson):
        ap.error("--warmup must be >= 3")
    if args.glueball and args.impl == "ours":
        out = run_glueball(args)
    elif args.meson and args.impl == "ours":
        out = run_meson(args)
    elif args.impl == "reference":
        out = run_reference(args)
    elif args.workload == 4:
        out = run_ensemble(args)
    elif args.workload == 5:
        out = run_timeslices(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
