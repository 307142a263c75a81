#!/usr/bin/env python3
"""Benchmark: site updates per second of the public goods game Monte Carlo on GB300.

Workload (one "step" = one full Monte Carlo step, L^2 elementary updates done as 16
sublattice steps): the L = 8192 bit-packed lattice of the critical-decay experiment,
K = 0.5, r = 3.744 (at the absorbing transition, r_c = 3.7443 in Section V, Fig. 4),
Bernoulli(1/2) initial state (Section III), seed 1 (+ rank). Inputs are resident in
HBM when the timed region starts; the L2 cache is flushed between timed steps (a
256 MiB write that the per-step CUDA events exclude).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--game pairwise]

Prints one JSON line. ``--impl reference`` times the CPU oracle (test
infrastructure, as it stands) on the host cores for the same metric and config.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "site updates/s at L=8192 (% HBM roofline); r_c search time, surrogate vs plain"
UNIT = "site updates/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# Per-launch counters of the dominant kernel from one ncu capture of this benchmark (see
# profiles/), keyed by a hash of the kernel's code (its sources without comments) and launch
# configuration; they are used only while that code is unchanged. alu_warp_inst / fma_warp_inst = warp instructions of the
# ALU pipe / of the FMA-heavy pipe (integer multiply-adds), dram_bytes = dram__bytes_read.sum +
# dram__bytes_write.sum.
NCU = {
    # the resident kernel (active-site and dense passes; the group game on the column-class copy):
    # means of 9 launches inside the timed window (MCS 5-7, 13-15, 22-24 of the benchmark command
    # with --no-autotune and the schedule named)
    "resident:0dd74940a8619de6:bitpack:8192:16:152:1":
        {"alu_warp_inst": 24732707, "fma_warp_inst": 16890979, "dram_bytes": 16880356},
    "resident:0dd74940a8619de6:bitpack:8192:16:152:2":
        {"alu_warp_inst": 25961540, "fma_warp_inst": 17912088, "dram_bytes": 16879474},
    "resident:0dd74940a8619de6:bitpack:8192:16:152:4":
        {"alu_warp_inst": 27730249, "fma_warp_inst": 19026971, "dram_bytes": 16883314},
    "resident-pairwise:0dd74940a8619de6:bitpack:8192:16:152:1":
        {"alu_warp_inst": 46606821, "fma_warp_inst": 31826447, "dram_bytes": 8471580},
    "resident:0dd74940a8619de6:u8:8192:16:152:2":
        {"alu_warp_inst": 28605390, "fma_warp_inst": 19541023, "dram_bytes": 101647445},
    "direct:c6f01ffbcae43cda:bitpack:8192:1:4:64":
        {"alu_warp_inst": 3675904, "fma_warp_inst": 3167136, "dram_bytes": 8444928},
}

# Integer ALU pipe of one SM: 4 sub-partitions x 16 lanes per clock (half-rate pipe).
ALU_LANES_PER_SM_CLOCK = 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=8192)
    ap.add_argument("--layout", default="bitpack", choices=["u8", "bitpack"])
    ap.add_argument("--r", type=float, default=3.744)
    ap.add_argument("--K", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--kernel", default="auto", choices=["auto", "simple", "tiled", "direct", "resident"])
    ap.add_argument("--fuse", type=int, default=1)
    ap.add_argument("--tile-x", type=int, default=0)
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--game", default="group", choices=["group", "pairwise"],
                    help="group: the public goods game (Section III); pairwise: a 2x2 matrix game "
                         "with each neighbour (Section VI)")
    ap.add_argument("--payoff", type=float, nargs=4, default=[1.0, 0.0, 1.04, 0.0],
                    metavar=("R", "S", "T", "P"), help="pairwise payoff matrix (weak prisoner's dilemma)")
    return ap.parse_args()


def game_text(args) -> str:
    if args.game == "pairwise":
        return f"pairwise game (R,S,T,P)=({', '.join(f'{x:g}' for x in args.payoff)}), K={args.K}"
    return f"PGG lattice, r={args.r}, K={args.K}"


def oracle_mcs(o, lat, args, k: int, threads: int) -> None:
    """One MCS of the oracle for the benchmark's game, from sublattice step k."""
    if args.game == "pairwise":
        o.pair_run(lat, args.payoff, args.K, args.seed, k, 1, threads=threads)
    else:
        o.run(lat, args.r, args.K, args.seed, k, 1, threads=threads)


def oracle_substep(o, lat, args, k: int) -> None:
    """One sublattice step k of the oracle for the benchmark's game, on one thread."""
    if args.game == "pairwise":
        o.pair_sublattice_step(lat, args.payoff, args.K, args.seed, k)
    else:
        o.sublattice_step(lat, args.r, args.K, args.seed, k)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def kernel_code(path: str) -> str:
    """A kernel source without its // comments, trailing blanks and empty lines (the sources hold
    no "//" inside string literals), so that an edit of comments alone keeps the hash."""
    out = []
    for line in open(path).read().splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code:
            out.append(code)
    return "\n".join(out) + "\n"


def kernel_source_hash(kernel: str) -> str:
    names = {"direct": ["pgg_kernels_direct.cu"], "tiled": ["pgg_kernels_tiled.cu"],
             "simple": ["pgg_kernels_basic.cu"], "resident": ["pgg_kernels_resident.cu"]}[kernel] + \
        ["pgg_unit.cuh", "pgg_device.cuh"]
    h = hashlib.sha256()
    for n in names:
        h.update(kernel_code(os.path.join(ROOT, "paper_1704_08098_gb300", "csrc", n)).encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlClockSampler:
    """SM clock and clock-event reasons polled every 2 ms through NVML (read-only calls),
    for timed regions far shorter than nvidia-smi's sampling period."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device: int):
        import ctypes
        import torch
        self.ok = False
        self.samples = []
        self.stop_flag = threading.Event()
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            pr = torch.cuda.get_device_properties(torch_device)
            bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0".encode()
            self.h = ctypes.c_void_p()
            if self.nvml.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(self.h)) != 0:
                return
            v = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(v)) != 0:
                return
            self.max_mhz = float(v.value)
            self.getr = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
            self.ctypes = ctypes
            self.ok = True
        except Exception:
            self.ok = False

    def _run(self):
        ct = self.ctypes
        clk, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop_flag.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(clk)) == 0 and \
                    self.getr(self.h, ct.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            time.sleep(0.002)

    def start(self):
        if self.ok:
            self.thread = threading.Thread(target=self._run, daemon=True)
            self.thread.start()

    def stop(self):
        if not self.ok:
            return None
        self.stop_flag.set()
        self.thread.join(timeout=2)
        if not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples), "source": "nvml 2 ms"}


def max_over_ranks(x: float, world: int) -> float:
    """Maximum of x over all ranks (the slowest rank sets the job's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(sites_per_step: float, steps: int, world: int, max_total_ms: float) -> float:
    """Whole-job site updates per second: every rank advances its own lattice."""
    return sites_per_step * steps * world / (max_total_ms / 1e3)


def algorithmic_bytes_per_update(layout: str, k: int) -> float:
    """Bytes a launch of k fused sublattice steps must move per site update: it reads the
    whole lattice once and writes the N/16 updated sites (k = 1, in place) or the whole
    lattice (k > 1, into the second buffer), for k N / 16 updates. b = bytes per site."""
    b = 1.0 if layout == "u8" else 1.0 / 8.0
    if k == 1:
        return 17.0 * b
    return 32.0 * b / k


def cpu_baseline(args, budget_s=12.0):
    """The CPU oracle, as it stands, on this host's cores, over the GPU arm's window: from the
    Bernoulli(1/2) start it runs the warm-up MCS untimed, then times whole MCS of the timed
    window (MCS W, W+1, ...) until about budget_s seconds of CPU work (at least one MCS, at most
    the GPU arm's step count), with a steady clock. Beside it, the same oracle on one core: the
    first four sublattice steps of MCS W on a copy of the lattice."""
    import oracle
    o = oracle.Oracle()
    threads = os.cpu_count() or 1
    L = args.L
    lat = o.init(L, args.seed, 0.5)
    for m in range(args.warmup):
        oracle_mcs(o, lat, args, 16 * m, threads)
    one = lat.copy()
    t0 = time.perf_counter()
    for j in range(4):
        oracle_substep(o, one, args, 16 * args.warmup + j)
    one_core = L * L / 16 * 4 / (time.perf_counter() - t0)
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle_mcs(o, lat, args, 16 * (args.warmup + n), threads)
        n += 1
        el = time.perf_counter() - t0
        if el * (n + 1) / n > budget_s or n >= args.steps:
            break
    return {"value": L * L * n / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"MCS {args.warmup}..{args.warmup + n - 1} of the L={L} workload after "
                      f"{args.warmup} untimed warm-up MCS from its Bernoulli(0.5) start, the GPU "
                      f"arm's timed window ({n * L * L} updates, {el:.1f} s, OpenMP over the sites "
                      f"of a step)",
            "one_core": {"value": one_core, "cores": 1,
                         "sample": f"sublattice steps {16 * args.warmup}..{16 * args.warmup + 3} "
                                   f"(the first quarter of MCS {args.warmup}), one thread"}}


def workload_config(args, world: int) -> dict:
    """The config both arms report, key for key (the same lattice, dynamics, random stream and
    timing discipline)."""
    L = args.L
    return {"workload": f"L={L} {args.layout} {game_text(args)}, Bernoulli(0.5) start, "
                        f"seed {args.seed}+rank; one step = 1 MCS = {L * L} site updates",
            "L": L, "layout": args.layout, "game": args.game, "r": args.r, "K": args.K,
            "payoff": args.payoff if args.game == "pairwise" else None,
            "window": f"MCS {args.warmup}..{args.warmup + args.steps - 1} after {args.warmup} "
                      f"untimed warm-up MCS",
            "l2": "GPU arm: L2 flushed between timed steps (256 MiB write, excluded by the "
                  "per-step CUDA events)",
            "parallelism": f"replicas x{world}"}


def refine_resident_schedule(lat, args, torch):
    """The library's autotuner times each schedule as one call of many MCS; this benchmark makes one
    call per MCS, where the per-call costs (staging, write-back, the last band to finish) weigh in.
    Untimed: time the resident kernel's halo-exchange intervals the autotuner can choose from in
    that pattern (one MCS per call over the timed window's MCS from its starting state, L2 flushed
    before each call), keep the fastest and restore the state. Returns the trial times."""
    from paper_1704_08098_gb300 import pgg
    words, step = lat.get_packed()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    best, trials = None, {}
    for spe in (1, 2, 4):
        try:
            lat.set_schedule("resident", 16, 0, spe)
        except pgg.PGGError:  # this lattice cannot take that many steps per exchange
            continue
        lat.set_packed(words, step)
        ms = 0.0
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lat.advance(1)
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        trials[spe] = ms / args.steps
        if best is None or trials[spe] < trials[best]:
            best = spe
    lat.set_packed(words, step)
    if best is None:
        return None
    lat.set_schedule("resident", 16, 0, best)
    return {"steps_per_exchange": best, "ms_per_mcs": trials}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle timed on the host cores, rank 0 only."""
    if rank != 0:
        return
    import oracle
    o = oracle.Oracle()
    threads = os.cpu_count() or 1
    L = args.L
    lat = o.init(L, args.seed, 0.5)
    k = 0
    for _ in range(args.warmup):
        oracle_mcs(o, lat, args, k, threads)
        k += 16
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_mcs(o, lat, args, k, threads)
        k += 16
    el = time.perf_counter() - t0
    value = L * L * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": workload_config(args, world),
        "implementation": "the CPU oracle (uint8 lattice in host memory, OpenMP over the sites of "
                          "a step); results identical to the GPU arm's",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} timed MCS after {args.warmup} warm-up MCS"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("PGG_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    from paper_1704_08098_gb300 import build, pgg
    build.build()
    stream = torch.cuda.current_stream()

    L = args.L
    lat = pgg.Lattice(L, args.r, args.K, layout=args.layout, stream=stream.cuda_stream)
    if args.game == "pairwise":
        lat.set_game("pairwise", args.payoff)
    lat.seed(args.seed + rank, 0.5)
    tuned = None
    if args.kernel != "auto":
        lat.set_schedule(args.kernel, args.fuse, args.tile_x, args.tile_y)
    for _ in range(args.warmup):
        lat.advance(1)
    if args.kernel == "auto" and not args.no_autotune:
        # untimed, on the state the timed window starts from and over as many MCS as the window
        # (update costs depend on how many sites can change, which falls along the window);
        # restores the lattice and step counter
        tuned = lat.autotune(max(3, min(args.steps, 1000)))
        if lat.schedule()["kernel"] == "resident":
            refined = refine_resident_schedule(lat, args, torch)
            if refined is not None:
                tuned["one_mcs_per_call"] = refined
    sched = lat.schedule()
    torch.cuda.synchronize()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    nvml = NvmlClockSampler(local)
    time.sleep(0.3)
    nvml.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        starts[i].record(stream)
        lat.advance(1)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    fine = nvml.stop()
    clocks = sampler.stop()
    if fine is not None:
        fine["nvidia_smi"] = clocks
        clocks = fine
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), world)
    # the step kernel alone, in an untimed pass of as many MCS: events around each of its launches
    # (recorded by the library; they lengthen a step by a few microseconds, so the timed region
    # above runs without them)
    lat.set_kernel_timing(True)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        lat.advance(1)
    kernel_ms, kernel_launches = lat.kernel_time()
    lat.set_kernel_timing(False)
    value = job_value(float(L) * L, args.steps, world, total_ms)

    # dominant kernel: the step kernel, 16 / k launches per MCS; its launch duration is the timed
    # MCS time / launches (launch gaps and the counts memset included, so it understates the
    # kernel's own rate a little; the event-timed pass gives the kernel alone)
    k = sched["steps_per_launch"]
    launches_per_mcs = 16 // k
    assert kernel_launches == launches_per_mcs * args.steps, (kernel_launches, launches_per_mcs)
    # other kernels of ours per MCS: the count of the simple kernel
    extra_launches_per_mcs = 1 if sched["kernel"] == "simple" else 0
    launch_s = (total_ms / args.steps) / launches_per_mcs / 1e3
    updates_per_launch = L * L / 16.0 * k
    pk, pk_kind = peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or pk.get("sm_max_mhz") or 2070.0
    kname = sched["kernel"] + ("-pairwise" if args.game == "pairwise" else "")
    key = f"{kname}:{kernel_source_hash(sched['kernel'])}:{args.layout}:{L}:" \
          f"{k}:{sched['tile_x']}:{sched['tile_y']}"
    ncu = NCU.get(key)
    alu_peak = sm_count * ALU_LANES_PER_SM_CLOCK * sm_mhz * 1e6 / 1e12  # Tops/s
    bpu = algorithmic_bytes_per_update(args.layout, k)
    hbm_achieved = bpu * updates_per_launch / launch_s / 1e9
    hbm_model = {"algorithmic_bytes_per_update": bpu, "achieved_gbs": hbm_achieved,
                 "peak_gbs": pk["hbm_gbs"], "frac": hbm_achieved / pk["hbm_gbs"],
                 "peak_kind": pk_kind}
    if ncu is not None:
        achieved = ncu["alu_warp_inst"] * 32 / launch_s / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                    "frac": achieved / alu_peak, "traffic": ncu["dram_bytes"],
                    "peak_kind": f"derived: {sm_count} SMs x {ALU_LANES_PER_SM_CLOCK} ALU lanes/clk"
                                 f" x {sm_mhz:.0f} MHz (median SM clock sampled in the run)",
                    "work_per_launch": f"{ncu['alu_warp_inst']} ALU-pipe warp instructions "
                                       f"(ncu, {updates_per_launch:.0f} updates)"}
        if ncu.get("fma_warp_inst"):
            # the integer multiply-adds the kernel issues on the FMA-heavy pipe (same lane count)
            fma = ncu["fma_warp_inst"] * 32 / launch_s / 1e12
            roofline["fma_pipe"] = {"achieved": fma, "peak": alu_peak, "frac": fma / alu_peak}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "frac": hbm_achieved / pk["hbm_gbs"], "traffic": None,
                    "peak_kind": pk_kind + " (STREAM-style copy); no ncu counters for this "
                                 "kernel source yet"}
    # the benchmark spec's HBM figure and the FMA-heavy pipe, as plain numbers beside the bound's own
    roofline["hbm_frac"] = hbm_model["frac"]
    roofline["hbm_achieved_gbs"] = hbm_achieved
    roofline["hbm_bytes_per_update"] = bpu
    if "fma_pipe" in roofline:
        roofline["fma_frac"] = roofline["fma_pipe"]["frac"]
    roofline.update({"kernel": f"{sched['kernel']} (k={k}, tile {sched['tile_x']}x"
                               f"{sched['tile_y']})", "launch_ms": launch_s * 1e3,
                     "ncu_key": key, "hbm_model": hbm_model,
                     "launch_timing": "timed MCS time / launches per MCS (CUDA events on the "
                                      "launching stream, L2 flushed between steps)",
                     "kernel_events_ms": kernel_ms / kernel_launches,
                     "kernel_events": "the step kernel alone: CUDA events recorded by the library "
                                      f"around each of {kernel_launches} launches in an untimed "
                                      "pass after the timed region"})

    # end to end through the public API with host buffers: every step uploads its input lattice
    # from pinned memory (in its bit-packed host form, L*L/8 bytes, for either device layout),
    # runs one MCS and reads its cooperator count back to the host. The inputs are the timed
    # window's own states (MCS W .. W+K-1, regenerated untimed from the same seed), taken in turn,
    # so the end-to-end figure covers the same work as `value`
    e2e = None
    if not args.no_e2e:
        h2d = L * L // 8
        lat.seed(args.seed + rank, 0.5)
        lat.advance(args.warmup)
        states, want = [], []
        for i in range(args.steps):
            words, step = lat.get_packed()
            states.append((torch.from_numpy(words.reshape(-1).view(np.int32)).pin_memory(), step))
            want.append(int(lat.step_mcs(1)[0]))
        reps = max(50, args.steps)
        # serial: synchronous upload, one MCS, the count read back by the same call
        counts = np.zeros(1, dtype=np.uint64)
        lat.set_packed_from_pointer(states[0][0].data_ptr(), states[0][1])   # untimed: first-use buffers
        lat.step_mcs(1, counts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r_ in range(reps):
            host, step = states[r_ % args.steps]
            lat.set_packed_from_pointer(host.data_ptr(), step)
            lat.step_mcs(1, counts)
        serial = L * L * reps / (time.perf_counter() - t0)
        # overlapped: step i+1's input is staged on the context's copy stream while step i runs;
        # each count goes to pinned host memory and the host reads count i-1 once step i is queued
        dev_counts = torch.zeros(reps, dtype=torch.int64, device="cuda")
        host_counts = torch.zeros(reps, dtype=torch.int64).pin_memory()
        done = [torch.cuda.Event() for _ in range(reps)]
        read = []
        lat.stage_packed_from_pointer(states[0][0].data_ptr(), states[0][1])   # untimed: copy stream
        lat.step_mcs(1, dev_counts[0].data_ptr())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(reps):
            host, step = states[i % args.steps]
            lat.stage_packed_from_pointer(host.data_ptr(), step)
            lat.step_mcs(1, dev_counts[i].data_ptr())
            host_counts[i].copy_(dev_counts[i], non_blocking=True)
            done[i].record(stream)
            if i > 0:
                done[i - 1].synchronize()
                read.append(int(host_counts[i - 1]))
        done[-1].synchronize()
        read.append(int(host_counts[-1]))
        el = time.perf_counter() - t0
        # every step reproduces the count of its window MCS
        assert read == [want[i % args.steps] for i in range(reps)], "end-to-end steps disagree"
        e2e = {"value": L * L * reps / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 8, "steps": reps,
               "path": "pgg_stage_lattice_packed(pinned host, L*L/8 bytes) + pgg_step_mcs(1, device "
                       "count) + count copied to pinned host memory and read each step; the upload "
                       "of step i+1 overlaps step i; the inputs are the timed window's states "
                       "(MCS W .. W+K-1) in turn",
               "serial": {"value": serial, "path": "pgg_set_lattice_packed (synchronous) + "
                                                   "pgg_step_mcs(1, host count)"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u1" if args.layout == "bitpack" else "u8", "data": "synthetic",
        "config": workload_config(args, world),
        "schedule": sched, "autotuned": tuned,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": (launches_per_mcs + extra_launches_per_mcs) * args.steps,
        "clocks": clocks, "wall_s": wall, "step_ms": step_ms,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    lat.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
