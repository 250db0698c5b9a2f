#!/usr/bin/env python
"""Benchmark: Hubbard-Stratonovich field updates per second of the BSS-DQMC
sweep on one GB300, 16x16 cluster, mixed precision against plain FP64.

Workload (one "step" = one sweep of every chain over all L slices, with the
Metropolis pass, delayed rank-k updates, slice wraps, UDV stack products,
FP64 QR stabilisation and G recompute at every stabilisation point,
equal-time observables, the left-stack rebuild and the unequal-time G(k, tau)
of every chain): 16x16 periodic cluster, t = 0.25, U = 2, beta = 20,
dtau = 0.125 (L = 160), 64 independent chains, delay k = 32, stabilisation
every 10 slices.  Updates counted = chains * N * L proposals per sweep.

The working set (UDV stacks of 64 chains, 2.2 GB) is far larger than the
129 MB L2, so no L2 flush is needed between steps.

`--impl reference` times the CPU oracle (oracle/, plain FP64 numpy) on the
host cores instead: each step sweeps one chain per worker process.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HS-field updates/s on 1 GB300 at 16x16; mixed/batched vs plain FP64 at equal G error"
UNIT = "updates/s"
W = dict(Lx=16, Ly=16, t=0.25, U=2.0, beta=20.0, dtau=0.125, chains=64, ns=10, k=32)
WORKLOAD = ("16x16 periodic Hubbard, t=0.25, U=2, beta=20, dtau=0.125 (L=160), 64 chains, "
            "k=32, n_s=10, G(k,tau) every sweep")


def n_sites():
    return W["Lx"] * W["Ly"]


def n_slices():
    return int(round(W["beta"] / W["dtau"]))


def updates_per_sweep(chains):
    return chains * n_sites() * n_slices()


# ---------------------------------------------------------------------------
# Several GPUs (torchrun, one rank per GPU): replicas only.  Every rank runs
# the whole workload on its own chains: rank r holds the global chains
# r C .. (r + 1) C - 1 of one seed (the chain id is the Philox counter word),
# so N ranks sample exactly the chains of one N C-chain run, whatever the
# split.  No data exchange; the step time is the maximum over ranks and the
# value counts the updates of all ranks (weak scaling).
# ---------------------------------------------------------------------------
def rank_chain_offset(rank):
    return rank * W["chains"]


def max_over_ranks(x, dist, device):
    """Maximum of a float over the ranks of `dist` (None: one rank)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, ms_per_step):
    """HS-field updates per second of the whole job."""
    return world * updates_per_sweep(W["chains"]) / (ms_per_step / 1e3)


# ---------------------------------------------------------------------------
# CPU oracle timing (host cores): one worker process per core, each sweeps
# one chain of the workload once; started with `spawn` before any CUDA call.
# ---------------------------------------------------------------------------
def _oracle_chain_sweep(chain):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import dqmc as o
    p = o.Params(W["Lx"], W["Ly"], W["t"], W["U"], W["beta"], W["dtau"], n_s=W["ns"])
    ch = o.Chain(p, seed=0, chain=chain)
    t0 = time.perf_counter()
    out = ch.sweep(measure=True)
    ch.gtau()
    return time.perf_counter() - t0, out["accepted"]


def _pool(workers):
    import multiprocessing as mp
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"  # inherited by the spawned workers: one core each
    return mp.get_context("spawn").Pool(workers)


def oracle_step(pool, workers, first_chain):
    t0 = time.perf_counter()
    pool.map(_oracle_chain_sweep, range(first_chain, first_chain + workers))
    return time.perf_counter() - t0


def cpu_baseline(workers):
    with _pool(workers) as pool:
        wall = oracle_step(pool, workers, 0)
    return {"value": updates_per_sweep(workers) / wall, "unit": UNIT, "cores": workers,
            "kind": "oracle",
            "sample": "%d chains of the workload, one full sweep each incl. G(tau), one "
                      "single-threaded process per core, %.1f s wall" % (workers, wall)}


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            self.p.wait(timeout=10)

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm.
# ---------------------------------------------------------------------------
def make_sim(pkg, precision, chain_offset):
    g = pkg.Group(Lx=W["Lx"], Ly=W["Ly"], t=W["t"], U=W["U"], beta=W["beta"], dtau=W["dtau"],
                  n_chains=W["chains"], stab_interval=W["ns"], delay_k=W["k"], precision=precision)
    return pkg.DQMC([g], seed=0, chain_offset=chain_offset)


def step_device(sim, gbuf):
    sim.sweep(1, measure=True)
    sim.gtau(out=gbuf)


def time_arm(pkg, torch, precision, steps, warmup, chain_offset, dist):
    sim = make_sim(pkg, precision, chain_offset)
    gbuf = torch.empty(int(pkg.lib().dqmc_gtau_size(sim._h)), dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        step_device(sim, gbuf)
    sim.reset_stats()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sim.launch_count()
    with Clocks(torch.cuda.current_device()) as clk:
        e0.record(st)
        for _ in range(steps):
            step_device(sim, gbuf)
        e1.record(st)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / steps
    launches = sim.launch_count() - l0
    drift, acc = sim.stats()
    return sim, gbuf, {"ms": ms, "launches": launches, "drift": float(drift.max()),
                       "acceptance": float(acc.sum()) / (updates_per_sweep(W["chains"]) * steps),
                       "clocks": clk.summary()}


def kernel_profile(sim, gbuf, steps, torch):
    """Per-class device time (CUDA events around every launch) over `steps` sweeps."""
    sim.timing(True)
    sim.timing_reset()
    for _ in range(steps):
        step_device(sim, gbuf)
    torch.cuda.synchronize()
    t = sim.timing_read()
    sim.timing(False)
    return t


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


# Peaks.  FP64 pipe: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz (unit counts and
# the maximum SM clock).  FP32 pipe: 152 x 128 FMA/clk x 2 x 2070 MHz; a float-pair
# (df32) multiply-add of the sweep kernels costs 14 FP32 instructions (TwoProd,
# TwoSum, operand loads), so the df32 arithmetic ceiling is 2 x 152 x 128 x 2.07e9 / 14.
FP64_PEAK = 152 * 2 * 2 * 2.07e9 / 1e12
DF32_PEAK = 2 * 152 * 128 * 2.07e9 / 14 / 1e12

# DRAM bytes per class launch (dram__bytes_read.sum + dram__bytes_write.sum,
# summed over the kernels of one launch of the class) from one ncu capture on
# the 64-chain 16x16 case (`bench.py --profile-case`), whose launches do the
# same work as the benchmark's (one slice of 64 chains; 64 QRs of order 256;
# one stack step of 64 chains), keyed by (class, precision).  Each entry names
# the source files of its kernels and the SHA-256 prefix they had when the
# counters were taken: if a file has changed since, the entry is stale and the
# roofline line reports null.  (profiles/launches_profile_case_16x16.md)
TRAFFIC = {
    # panel x 8, fused rank-32 products x 30, finalize: one blocked QR launch
    ("qr_pivot", None): (687.4e6, ("k_qr_blocked.cu", "k_ozaki.cu"), "aadad93db001c3cb"),
    ("metropolis", "df32"): (33.71e6, ("k_sweep.cu",), "e10916f2f31b97b5"),
    ("stack_kron", None): (34.07e6, ("k_kron_tc.cu",), "5046ac778a31eae9"),
}


def _source_sha16(files):
    import hashlib
    h = hashlib.sha256()
    try:
        for rel in files:
            with open(os.path.join(ROOT, "paper_1504_05090_gb300", "csrc", rel), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return h.hexdigest()[:16]


def traffic_bytes(cls, precision):
    """Measured DRAM bytes per launch of the class, or None when there is no
    capture of the current source."""
    ent = TRAFFIC.get((cls, precision), TRAFFIC.get((cls, None)))
    if ent is None:
        return None
    nbytes, files, sha = ent
    return int(nbytes) if _source_sha16(files) == sha else None


def class_work(cls, acceptance, precision):
    """Algorithmic work of one sweep of the benchmark workload for a kernel
    class: (units, amount, bound).  Counted from the formulas of the method,
    not from what the kernels execute."""
    N, L, ns, C = n_sites(), n_slices(), W["ns"], W["chains"]
    Lx, Ly = W["Lx"], W["Ly"]
    nc = -(-L // ns)
    g3 = 2.0 * N ** 3
    if cls == "gemm_f64":
        # T updates (2 nc), recompute Mid + W1 + G (4 per point, nc points),
        # G(tau) Mid + W1 + G(l,0) + W2 + Y (6 per point, nc + 1); on the tensor
        # cores each FP64 product is 36 BF16 digit products.
        fp64eq = C * g3 * (2 * nc + 4 * nc + 6 * (nc + 1))
        return "tensor", 36 * fp64eq
    if cls == "qr_pivot":
        # Householder R and explicit Q, both stacks, counted as FP64 flops:
        # the panels run on the FP64 pipe, the trailing updates and the
        # accumulation of Q (about 90 % of the flops) on the tensor cores
        return "alu64", C * 2 * nc * (8.0 / 3.0) * N ** 3
    if cls == "gj_inverse":  # nc recomputes + (nc + 1) stabilisation points for G(tau)
        # (float-pair groups invert the G(tau) points in float pairs, the class below)
        return "alu64", C * (nc if precision == "df32" else 2 * nc + 1) * g3
    if cls == "gj_inverse_pair":  # G(tau) points of float-pair groups
        return "alu32x2", C * (nc + 1) * g3
    if cls in ("stack_kron", "gtau_propagate"):
        # two matrices (right and left stack; G(l,0) and Y) x L slices x N vectors
        # x 2N(Lx+Ly) flops per Kronecker application.  The stack products (and
        # the G(tau) propagation of FP64 groups) run on the tensor cores as 36
        # BF16 digit products per FP64 product; float-pair groups propagate
        # G(tau) in float pairs on the FP32 pipe
        fp64eq = C * 2 * L * N * 2 * N * (Lx + Ly)
        if cls == "gtau_propagate" and precision == "df32":
            return "alu32x2", fp64eq
        return "tensor", 36 * fp64eq
    if cls == "metropolis":  # rank-1 Sherman-Morrison update per accepted flip
        return ("alu32x2" if precision == "df32" else "alu"), acceptance * C * N * L * 2.0 * N * N
    if cls == "wrap":  # B G B^-1 by Kronecker factors: 2 sides x N vectors x 2N(Lx+Ly)
        return ("alu32x2" if precision == "df32" else "alu"), C * L * 2 * N * 2 * N * (Lx + Ly)
    return None, None


def roofline(profile, steps, acceptance, precision="df32"):
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained")
    rows = {}
    for cls, (ms, n) in profile.items():
        bound, work = class_work(cls, acceptance, precision)
        if bound is None or n == 0 or ms <= 0:
            continue
        ach = work * steps / (ms / 1e3) / 1e12
        if bound == "tensor":
            peak, src = (bf16, "measured bf16 GEMM, sustained (MEASURED_PEAKS.json)") if bf16 else \
                (1700.0, "fallback 1.7 PFLOP/s bf16 sustained")
        elif bound == "alu64":
            peak, src = FP64_PEAK, "derived FP64 pipe: 152 SMs x 2 FMA/clk x 2 x 2070 MHz"
        elif bound == "alu32x2":
            peak, src = DF32_PEAK, "derived df32: FP32 pipe 152 x 128 FMA/clk x 2 x 2070 MHz / 14 instr"
        else:
            peak, src = 2 * 152 * 128 * 2.07e9 / 1e12, "derived FP32 pipe: 152 x 128 FMA/clk x 2 x 2070 MHz"
        traffic = traffic_bytes(cls, precision)
        rows[cls] = {"bound": "tensor" if bound == "tensor" else "alu", "kernel": cls,
                     "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                     "traffic": traffic, "peak_source": src,
                     "flops_per_launch": work * steps / n, "avg_launch_ms": ms / n, "launches": n}
    dom = max(profile.items(), key=lambda kv: kv[1][0])[0]
    return rows.get(dom, {"bound": "alu", "kernel": dom, "achieved": None, "peak": None,
                          "unit": "TFLOP/s", "frac": None, "traffic": None}), rows


def e2e_arm(pkg, torch, sim, steps):
    """Same metric through the public API with host outputs: every step copies
    G(k, tau) of all chains, the observables and the spin correlation to host
    memory."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nbytes = 0
    for _ in range(steps):
        sim.sweep(1, measure=True)
        gt = sim.gtau()
        ob = sim.observables()
        sc = sim.spin_correlation()
        nbytes = sum(a.nbytes for a in gt) + ob.nbytes + sum(a.nbytes for a in sc)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    return {"ms": dt * 1e3, "unit": UNIT, "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": int(nbytes)}


def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_workers or min(os.cpu_count() or 1, 16))
    import torch
    import paper_1504_05090_gb300 as pkg
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    offset = rank_chain_offset(rank)  # this rank's global chains (weak scaling)

    # Mixed arm: float-pair (df32) Metropolis / delayed update / wrap on the FP32
    # pipe with FP64 stabilisation -- the same G drift as plain FP64 (see
    # --scan-ns).  Plain FP64 and FP32 working precision are timed beside it.
    sim, gbuf, mixed = time_arm(pkg, torch, "df32", args.steps, args.warmup, offset, dist)
    prof = kernel_profile(sim, gbuf, args.steps, torch)
    e2e = e2e_arm(pkg, torch, sim, max(1, min(args.steps, 3)))
    sim.close()
    arms = {}
    for prec in ("fp64", "fp32"):
        s2, b2, res = time_arm(pkg, torch, prec, args.steps, args.warmup, offset, dist)
        res["kernel_ms_per_step"] = {k: v[0] / args.steps
                                     for k, v in kernel_profile(s2, b2, args.steps, torch).items()}
        s2.close()
        arms[prec] = res
    plain = arms["fp64"]

    def slowest(ms):
        return max_over_ranks(ms, dist, "cuda")

    ms = slowest(mixed["ms"])
    roof, roof_rows = roofline(prof, args.steps, mixed["acceptance"], "df32")
    ms64 = slowest(plain["ms"])
    ms32 = slowest(arms["fp32"]["ms"])  # every rank joins every reduction
    e2e_ms = slowest(e2e.pop("ms"))
    e2e["value"] = job_value(world, e2e_ms)
    value = job_value(world, ms)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "df32+f64", "data": "synthetic",
            "config": bench_config(),
            "drift": mixed["drift"], "acceptance": mixed["acceptance"],
            "fp64_plain": {"value": job_value(world, ms64),
                           "ms_per_step": ms64, "drift": plain["drift"],
                           "speedup_mixed_over_fp64": ms64 / ms,
                           "kernel_ms_per_step": plain["kernel_ms_per_step"]},
            "fp32_working": {"value": job_value(world, ms32),
                             "ms_per_step": ms32, "drift": arms["fp32"]["drift"],
                             "kernel_ms_per_step": arms["fp32"]["kernel_ms_per_step"]},
            "roofline": roof,
            "roofline_by_class": roof_rows,
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "e2e": e2e, "gpu_launches": mixed["launches"], "clocks": mixed["clocks"],
        }
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_scan_ns(args):
    """Drift of the working G at the stabilisation points against n_s, per
    working precision (8 chains of the workload, 2 warm-up + 2 measured sweeps)."""
    import torch
    import paper_1504_05090_gb300 as pkg
    import numpy as np
    for prec, nss in (("fp64", (10, 15, 20, 25, 30)), ("df32", (10, 15, 20, 25)),
                      ("fp32", (2, 3, 5, 10))):
        for ns in nss:
            g = pkg.Group(Lx=W["Lx"], Ly=W["Ly"], t=W["t"], U=W["U"], beta=W["beta"],
                          dtau=W["dtau"], n_chains=8, stab_interval=ns, delay_k=W["k"],
                          precision=prec)
            with pkg.DQMC([g], seed=0) as sim:
                sim.sweep(2)
                sim.reset_stats()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sim.sweep(2)
                torch.cuda.synchronize()
                dt = (time.perf_counter() - t0) / 2
                d, _ = sim.stats()
                print(json.dumps({"precision": prec, "n_s": ns, "drift_max": float(d.max()),
                                  "drift_median": float(np.median(d)),
                                  "s_per_sweep_8_chains": dt}), flush=True)


def run_profile_case(args):
    """Small case for ncu captures: the 16x16 kernels on 64 chains with L = 20
    (beta = 2.5), one initialisation and one sweep with G(tau); about 0.4 GB."""
    import torch
    import paper_1504_05090_gb300 as pkg
    g = pkg.Group(Lx=W["Lx"], Ly=W["Ly"], t=W["t"], U=W["U"], beta=2.5, dtau=W["dtau"],
                  n_chains=W["chains"], stab_interval=W["ns"], delay_k=W["k"],
                  precision=args.precision)
    with pkg.DQMC([g], seed=0) as sim:
        buf = torch.empty(int(pkg.lib().dqmc_gtau_size(sim._h)), dtype=torch.float64,
                          device="cuda")
        step_device(sim, buf)
        torch.cuda.synchronize()
        d, a = sim.stats()
        print(json.dumps({"profile_case": "16x16 L=20 64 chains", "drift": float(d.max()),
                          "launches": sim.launch_count()}))


def config_groups(pkg, name, precision):
    """Parameter sets of the other benchmark configurations."""
    G = pkg.Group
    if name == "c1":   # 4x4, U = 1, beta = 10, dtau = 0.25 (L = 40), 1 chain, n_s = 10
        return [G(Lx=4, Ly=4, t=0.25, U=1.0, beta=10.0, dtau=0.25, n_chains=1, stab_interval=10,
                  delay_k=8, precision=precision)]
    if name == "c2":   # 8x8, U = 2, beta = 20, dtau in {0.4, 0.2, 0.1}, 256 chains each, k = 16, n_s = 8
        return [G(Lx=8, Ly=8, t=0.25, U=2.0, beta=20.0, dtau=dt, n_chains=256, stab_interval=8,
                  delay_k=16, precision=precision) for dt in (0.4, 0.2, 0.1)]
    if name == "c4":   # uneven batch: six lattices x 32 chains, U / beta / dtau round robin
        sides = (6, 8, 10, 12, 14, 16)
        Us, betas, dts = (1.0, 2.0, 3.0), (10.0, 15.0, 20.0), (0.2, 0.125, 0.1)
        return [G(Lx=L, Ly=L, t=0.25, U=Us[i % 3], beta=betas[i % 3], dtau=dts[i % 3], n_chains=32,
                  stab_interval=10, delay_k=16, precision=precision) for i, L in enumerate(sides)]
    if name == "c5":   # 8x8, U = 2, beta = 10, dtau = 0.125 (L = 80), 512 chains, FP64, gradients
        return [G(Lx=8, Ly=8, t=0.25, U=2.0, beta=10.0, dtau=0.125, n_chains=512, stab_interval=10,
                  delay_k=16, precision="fp64")]
    raise ValueError(name)


def time_extrapolation(pkg, torch, groups, gbuf, reps, M=400):
    """dtau -> 0 extrapolation of G_k(tau) over the groups' runs (one group per
    dtau, same lattice and beta), from the device buffer dqmc_measure_Gtau
    filled; L2 is flushed before every timed call.  Bound: HBM, the chain
    data read once (the chain average dominates)."""
    views, off = [], 0
    for g in groups:
        n = g.n_chains * (g.L + 1) * g.N
        views.append(gbuf[off:off + n].view(g.n_chains, g.L + 1, g.N))
        off += n
    dts = [g.dtau for g in groups]
    beta = groups[0].beta
    # L2 flush by reading 2x the 129 MB L2 (a written buffer would leave dirty
    # lines whose write-back the timed kernel would pay for)
    flush = torch.zeros(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        pkg.trotter_extrapolate(dts, views, beta, M)
    ms, kms = [], []
    for _ in range(reps):
        flush.sum()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pkg.trotter_extrapolate(dts, views, beta, M)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        kms.append(pkg.trotter_timing())
    med = lambda v: sorted(v)[len(v) // 2]
    ms = med(ms)
    k_mean, k_spline, k_fit = (med([k[q] for k in kms]) for q in range(3))
    in_bytes = off * 8  # the chain data, read once by the chain average
    nbytes = in_bytes + (M + 1) * groups[0].N * 8
    peak = measured_peaks().get("hbm_gbs")
    gbs = in_bytes / (k_mean / 1e3) / 1e9  # dominant kernel: the chain average
    return {"workload": "%d runs, dtau %s, %d chains x (L+1) x %d momenta each, M = %d"
                        % (len(groups), "/".join("%g" % d for d in dts), groups[0].n_chains,
                           groups[0].N, M),
            "call_ms_median": ms, "call_gbs": nbytes / (ms / 1e3) / 1e9,
            "kernel_ms_median": {"chain_mean": k_mean, "spline": k_spline, "fit": k_fit},
            "roofline": {"kernel": "chain_mean", "bound": "hbm", "achieved": gbs, "unit": "GB/s",
                         "peak": peak, "frac": gbs / peak if peak else None,
                         "traffic": None, "bytes_per_launch": in_bytes,
                         "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"
                         if peak else None},
            "l2": "flushed before every call (256 MB read)"}


def time_matsubara(pkg, torch, fine, g, beta, reps, n_freq=200):
    """Matsubara transform and Dyson self-energy of the extrapolated G_k(tau)
    (device tensor [M + 1, N]) for n_freq frequencies.  Bound: the FP64 pipe;
    the transform does 8 FP64 flops per (frequency, momentum, knot): the
    sums of z_j y_j and z_j M_j, four FMAs."""
    M = fine.shape[0] - 1
    for _ in range(3):
        pkg.matsubara_sigma(fine, beta, g.Lx, g.Ly, g.t, n_freq)
    ms, kms = [], []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pkg.matsubara_sigma(fine, beta, g.Lx, g.Ly, g.t, n_freq)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        kms.append(pkg.matsubara_timing())
    med = lambda v: sorted(v)[len(v) // 2]
    k_spline, k_transform = (med([k[q] for k in kms]) for q in range(2))
    flops = 8.0 * n_freq * g.N * M
    tf = flops / (k_transform / 1e3) / 1e12
    return {"workload": "G_k(tau) on M = %d intervals, %d momenta, %d Matsubara frequencies"
                        % (M, g.N, n_freq),
            "call_ms_median": med(ms),
            "kernel_ms_median": {"spline": k_spline, "transform_and_dyson": k_transform},
            "roofline": {"kernel": "transform_and_dyson", "bound": "alu", "achieved": tf,
                         "unit": "TFLOP/s", "peak": FP64_PEAK, "frac": tf / FP64_PEAK,
                         "flops_per_launch": flops,
                         "peak_source": "derived FP64 pipe: 152 SMs x 2 FMA/clk x 2 x 2070 MHz"}}


def run_origins(args):
    """Time-origin averaged G(tau) on the headline workload: device time of
    one dqmc_measure_Gtau_origins call with 1 and with args.origins origins,
    after warm-up sweeps.  Each extra origin is one rotation of the field,
    a rebuild of both stacks and a G(tau) pass (the kernels of the sweep)."""
    import torch
    import paper_1504_05090_gb300 as pkg
    sim = make_sim(pkg, "df32", 0)
    gbuf = torch.empty(int(pkg.lib().dqmc_gtau_size(sim._h)), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        sim.sweep(1, measure=True)
    res = {}
    for n in (1, args.origins):
        ms = []
        for _ in range(max(3, args.steps)):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sim.gtau_origins(n, out=gbuf)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[n] = sorted(ms)[len(ms) // 2]
    sim.close()
    n = args.origins
    print(json.dumps({"leg": "gtau_origins", "workload": WORKLOAD, "origins": n,
                      "ms_one_origin": res[1], "ms_origins": res[n],
                      "ms_per_extra_origin": (res[n] - res[1]) / max(1, n - 1)}), flush=True)


def run_trotter(args):
    """The dtau -> 0 extrapolation alone, on seeded synthetic runs shaped like
    the 8x8 three-dtau configuration (256 chains per run, G_k(tau) on L + 1 =
    51 / 101 / 201 slices, 64 momenta), resident on the device."""
    import torch
    import paper_1504_05090_gb300 as pkg
    groups = config_groups(pkg, "c2", "fp64")
    gen = torch.Generator(device="cuda").manual_seed(0)
    total = sum(g.n_chains * (g.L + 1) * g.N for g in groups)
    gbuf = torch.rand(total, dtype=torch.float64, device="cuda", generator=gen)
    line = {"leg": "trotter_extrapolate", "data": "synthetic"}
    line.update(time_extrapolation(pkg, torch, groups, gbuf, max(5, args.steps)))
    views, off = [], 0
    for g in groups:
        n = g.n_chains * (g.L + 1) * g.N
        views.append(gbuf[off:off + n].view(g.n_chains, g.L + 1, g.N))
        off += n
    fine = pkg.trotter_extrapolate([g.dtau for g in groups], views, groups[0].beta, 400)
    line["matsubara_sigma"] = time_matsubara(pkg, torch, fine, groups[0], groups[0].beta,
                                             max(5, args.steps))
    print(json.dumps(line), flush=True)


def run_config(args):
    """One JSON line per precision for a secondary configuration: sweeps (with
    G(tau) for c2/c4, with the gradient for c5) per second and updates/s."""
    import torch
    import paper_1504_05090_gb300 as pkg
    precs = ("fp64",) if args.config == "c5" else ("df32", "fp64", "fp32")
    for prec in precs:
        groups = config_groups(pkg, args.config, prec)
        tuned = None
        tiles = None
        if args.autotune > 0 and args.config in ("c2", "c4"):
            t0 = time.perf_counter()
            groups = pkg.autotune(groups, drift_target=args.autotune)
            tiles = pkg.autotune_tiles(groups)
            tuned = {"target": args.autotune, "seconds": time.perf_counter() - t0,
                     "n_s": [g.stab_interval for g in groups], "k": [g.delay_k for g in groups],
                     "tiles": tiles}
        with pkg.DQMC(groups, seed=0) as sim:
            if tiles:
                for gi, t in enumerate(tiles):
                    sim.set_tiles(gi, **t)
            n_up = sum(g.n_chains * g.N * g.L for g in groups)
            gbuf = torch.empty(int(pkg.lib().dqmc_gtau_size(sim._h)), dtype=torch.float64, device="cuda")
            dt = torch.empty(sim.n_chains, dtype=torch.float64, device="cuda")
            dl, lw = torch.empty_like(dt), torch.empty_like(dt)

            def step():
                sim.sweep(1, measure=True)
                if args.config in ("c2", "c4"):
                    sim.gtau(out=gbuf)
                if args.config == "c5":
                    sim.grad_device(dt, dl, lw)
            for _ in range(args.warmup):
                step()
            sim.reset_stats()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                step()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            d, a = sim.stats()
            line = {"config": args.config, "precision": prec, "ms_per_step": ms,
                    "updates_per_s": n_up / (ms / 1e3), "chains": sim.n_chains,
                    "drift_max": float(d.max()), "autotune": tuned,
                    "acceptance": float(a.sum()) / (n_up * args.steps)}
            if args.config == "c2":
                line["trotter_extrapolate"] = time_extrapolation(pkg, torch, groups, gbuf,
                                                                 max(5, args.steps))
            print(json.dumps(line), flush=True)


def bench_config():
    """The workload description both arms report."""
    return {"workload": WORKLOAD, "precision": "df32 (float pairs) Metropolis/delayed "
            "update/wrap/G(tau) propagation, fp64 UDV/QR stabilisation, G recompute, drift",
            "chains_per_gpu": W["chains"], "L2": "working set > L2 (no flush needed)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    workers = args.cpu_workers or min(os.cpu_count() or 1, 16)
    with _pool(workers) as pool:
        chain = 0
        for _ in range(args.warmup):
            oracle_step(pool, workers, chain)
            chain += workers
        t = 0.0
        for _ in range(args.steps):
            t += oracle_step(pool, workers, chain)
            chain += workers
    ms = t / args.steps * 1e3
    value = updates_per_sweep(workers) / (ms / 1e3)
    sample = ("%d chains of the workload per step (one full oracle sweep incl. G(tau) per "
              "single-threaded process)" % workers)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(),
        "reference": "the FP64 CPU oracle (oracle/dqmc.py) on the host cores: no reference "
                     "implementation exists for this paper",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-workers", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--config", default="", choices=["", "c1", "c2", "c4", "c5"],
                    help="time a secondary configuration instead of the headline workload")
    ap.add_argument("--autotune", type=float, default=0.0,
                    help="with --config c2/c4: tune n_s and k for this drift target first")
    ap.add_argument("--profile-case", action="store_true",
                    help="run the small ncu capture case (16x16, L=20) and exit")
    ap.add_argument("--precision", default="df32", choices=["df32", "fp32", "fp64"])
    ap.add_argument("--scan-ns", action="store_true",
                    help="print the G drift against the stabilisation interval and exit")
    ap.add_argument("--origins", type=int, default=0,
                    help="time the time-origin averaged G(tau) with this many origins and exit")
    ap.add_argument("--trotter", action="store_true",
                    help="time the dtau -> 0 extrapolation of G_k(tau) alone and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.config:
        run_config(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.scan_ns:
        run_scan_ns(args)
    elif args.trotter:
        run_trotter(args)
    elif args.origins > 0:
        run_origins(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
