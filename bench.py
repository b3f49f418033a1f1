#!/usr/bin/env python3
"""Benchmark of the RSI hot path on GB300: one step = the full-image chain of
the 2^16-point piston / 2^18-point 80 x 80 mm interface / 512 x 512 image
workload at 2.25, 5 and 10 MHz (points, piston stage, transmission, RSI
stage, image), i.e. 2.58e11 source x target pair terms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is pair terms per second over the K timed
steps (CUDA events on the launching stream, L2 flushed before every step);
`e2e` repeats the measurement through the public API with the image read
back into pinned host memory each step; `roofline` relates the dominant
kernel's pair rate to the FP32-issue / MUFU limits measured by the
library's own throughput probes; `cpu_baseline` times the FP64 oracle on a
bounded sample of the same workload on the host cores.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Per-pair work of the FP32C kernels as formulated (far path, Newton update of
# r, counted from csrc/stage_fp32_body.cuh): FP32-pipe instructions, MUFU
# operations, and shared-memory loads per pair at 2 targets per thread (two
# 16-byte records per source shared by the thread's 2 targets).
OPS = {
    # FP32-pipe warp instructions, MUFU operations and shared loads per pair of
    # the default kernel (two sources per packed f32x2 instruction): RSI 18
    # packed per two pairs (10 for r - R and the phase, 4 for the obliquity
    # and the factors g, g/r of the polar amplitude, 4 accumulations) plus one
    # scalar scaling of the sincos argument per pair; piston 13 packed per two
    # pairs plus the same scaling
    "rsi": {"fp32": 10, "mufu": 3, "lds": 1.0, "fma_pipe": 19},
    "piston": {"fp32": 7.5, "mufu": 3, "lds": 1.0, "fma_pipe": 14},
    # ray-tracing pair (Sec. 2.2), two transducer points per f32x2
    # instruction: linear prediction of the crossing from the tile's reference
    # ray, 1 Newton step (15 packed FP32 per two points, 3 MUFU per point) and
    # its error bound (3 packed), ~97 packed FP32 per two pairs in all plus 5
    # scalar (the products of the fast divisions, the sincos scaling), ~13
    # compares, selects and clamps, 11 MUFU (the path differences by a Newton
    # step, T12 inside the amplitude's rsqrt); safeguarded steps not counted
    "raytrace": {"fp32": 53.5, "alu": 13, "mufu": 11, "lds": 2.0, "fma_pipe": 102},
}
# "fma_pipe": FP32-pipe lane cycles per pair: a packed f32x2 instruction keeps
# the pipe two cycles (two FMAs per lane), a scalar one cycle.
L2_FLUSH_BYTES = 256 << 20
METRIC = "rsi_pair_terms_per_s"
UNIT = "pair-terms/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target duration of the oracle CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nf", type=int, default=1,
                    help="--case stage: frequencies per stage (2-4: the multi-frequency stage at 10, 5, 2.25, 1 MHz)")
    ap.add_argument("--no-multi", action="store_true",
                    help="run frequencies that share their points one by one instead of together")
    ap.add_argument("--small", action="store_true",
                    help="f2: 2^14 transducer points onto 256^2 pixels (a profiling case)")
    ap.add_argument("--case", choices=["chain", "stage", "gemm", "infer", "train"], default="chain",
                    help="stage: only the RSI interface -> image kernel of the 10 MHz c2 chain "
                         "on a 256 x 256 image (small case for profiler captures)")
    ap.add_argument("--variant", type=int, default=0, help="FP32C distance update (0 auto)")
    ap.add_argument("--curved", action="store_true",
                    help="--case stage: c3's curved bottom surface (per-point normals) onto its image")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--tpt", type=int, default=0)
    ap.add_argument("--config", choices=["c1", "c2", "c3", "c4", "c5", "f1", "f2", "f3", "f4"], default="c2",
                    help="c4: the batched broadband scan (2048 instances in one CUDA graph); "
                         "c5: the learned surrogate (train on RSI fields, compare)")
    ap.add_argument("--fields", type=int, default=20000, help="c5: training fields")
    ap.add_argument("--instances", type=int, default=0, help="c4: first N instances only (0 = all)")
    ap.add_argument("--c5-steps", type=int, default=400000, help="c5: training steps")
    ap.add_argument("--c5-rows", type=int, default=32768, help="c5: rows (field, pixel pairs) per step")
    ap.add_argument("--c5-freq", type=int, default=248, help="c5: Fourier frequencies (2F + 16 % 128 == 0)")
    ap.add_argument("--c5-width", type=int, default=512, help="c5: hidden width")
    ap.add_argument("--c5-depth", type=int, default=5, help="c5: hidden layers")
    ap.add_argument("--c5-piston-log2", type=int, default=16, help="c5: log2 QMC points on the piston")
    ap.add_argument("--c5-iface-log2", type=int, default=18, help="c5: log2 QMC points on the interface")
    ap.add_argument("--lr", type=float, default=1e-3, help="c5: peak learning rate")
    ap.add_argument("--c5-train-tilt-max", type=float, default=13.0,
                    help="c5: train on fields with |tilt| below this (degrees; the gate serves the rest by RSI)")
    ap.add_argument("--gemm-shape", default="1024,32768,512",
                    help="--case gemm: M,N,K (default: the surrogate's output layer at batch 1024)")
    ap.add_argument("--engine", choices=["tcgen05", "mma_sync"], default="tcgen05", help="c5: GEMM engine")
    ap.add_argument("--sweep", action="store_true",
                    help="with --case stage: time every tile / targets-per-thread / variant")
    return ap.parse_args()


DESCRIPTION = {
    "c1": "c1 plain RSI in FP64: 4096 piston x 4096 interface (60 mm) x 64^2 image, 5 MHz, "
          "water -> steel at 50 mm",
    "c2": "c2 full-image RSI: 2^16 piston x 2^18 interface (80 mm) x 512^2 image, "
          "f = 2.25/5/10 MHz, water -> steel at 50 mm",
    "c3": "c3 multilayer RSI: 5 mm piston, 30 mm water, 8 layers of 0.5 mm (9 interfaces of 2^16 "
          "points), 256^2 image below; flat and concentric-cylinder variants",
}


def workload(name: str = "c2"):
    from paper_2408_06765_gb300 import workloads as W
    cfgs = {"c1": lambda: [W.c1_plain_fp64()], "c2": W.c2_all,
            "c3": lambda: [W.c3_multilayer(False), W.c3_multilayer(True)]}[name]()
    pairs = sum(W.pairs_of(c) for c in cfgs)
    pixels = sum(int(c["grid"]["nx"]) * int(c["grid"]["nz"]) for c in cfgs)
    return cfgs, pairs, pixels


def config_block(cfgs, n_gpus, name="c2"):
    return {"workload": DESCRIPTION[name],
            "frequencies_mhz": [c["freq"] / 1e6 for c in cfgs],
            "n_piston": cfgs[0]["piston"]["n"], "n_interface": cfgs[0]["interfaces"][0]["n"],
            "interfaces": len(cfgs[0]["interfaces"]),
            "image": [cfgs[0]["grid"]["nz"], cfgs[0]["grid"]["nx"]],
            "precision": ("fp64" if cfgs[0]["precision"] == "fp64"
                          else "fp32 pairs, double-float phase, compensated sums"),
            "l2": "flushed (256 MiB write) before every timed step",
            "parallelism": (f"target-sharded chain x{n_gpus} (stage targets split over the ranks, one "
                            "all-gather per interface and one of the image rows)" if n_gpus > 1 else "1 GPU")}


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# throughput probes -> ALU roofline
# ---------------------------------------------------------------------------
def recorded_traffic(kernel: str = "stage_fp32_kernel"):
    """DRAM bytes per RSI-stage launch of `kernel` from the committed ncu
    summary, if the kernel source is still the one the counters were taken
    on; else None."""
    import hashlib
    import re
    name, srcs = {"stage_fp32_kernel": ("traffic_stage_fp32_rsi_c2.md", ("stage_fp32_body.cuh", "stage_fp32.cu")),
                  "stage_multi_kernel": ("traffic_stage_multi_rsi_c2.md", ("stage_fp32_body.cuh", "stage_multi.cu"))}[
        kernel]
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    m = re.search(kernel + r"_rsi_dram_bytes_per_launch (\d+) source_sha256_16 (\w+)", open(path).read())
    if not m:
        return None
    h = hashlib.sha256()
    for f in srcs:
        h.update(open(os.path.join(ROOT, "paper_2408_06765_gb300", "csrc", f), "rb").read())
    return int(m.group(1)) if h.hexdigest()[:16] == m.group(2) else None


def recorded_fp64_ops():
    """FP64-pipe thread instructions per pair of the FP64 piston stage kernel
    from the committed ncu summary, if the kernel source is still the one the
    counters were taken on; else None."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "stage_fp64_c1_fp64_ops.md")
    if not os.path.exists(path):
        return None
    m = re.search(r"stage_fp64_kernel_fp64_ops_per_pair ([0-9.]+) source_sha256_16 (\w+)", open(path).read())
    if not m:
        return None
    h = hashlib.sha256()
    for f in ("stage_fp64.cu",):
        h.update(open(os.path.join(ROOT, "paper_2408_06765_gb300", "csrc", f), "rb").read())
    return float(m.group(1)) if h.hexdigest()[:16] == m.group(2) else None


def measure_unit_rates(rsi, torch, kinds=("ffma", "rsqrt", "sin")):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, iters = sms * 8, 65536
    sink = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    rates = {}
    for kind in kinds:
        if kind == "dfma":
            iters = 4096  # the FP64 pipe is slow: keep the probe short
        rsi.ubench(kind, blocks, 64, sink)  # warm-up
        best = float("inf")
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rsi.ubench(kind, blocks, iters, sink)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        rates[kind] = blocks * 256 * iters * 8 / best  # lane operations per second
    return rates


# sm_100-family unit counts per SM per clock: 4 schedulers x 32 lanes issue
# (FP32 FMA rate), 16 MUFU lanes; the probes in rsi_ubench confirm them.
ISSUE_LANES_PER_SM, MUFU_LANES_PER_SM = 128, 16


def multi_ops(kind: str, nf: int, harmonic: bool = False) -> dict:
    """Per pair-term counts of the multi-frequency stage kernel (nf frequencies
    on shared points, two sources per packed f32x2 instruction, one target per
    thread): the shared geometry once per source pair, phase, sincos and
    epilogue per frequency, plus one scalar scaling of each sincos argument;
    of the packed record of a source pair, 2 + nf float4 (RSI: geometry and
    the polar amplitudes) or 4 (piston) are read once per target.  harmonic:
    three frequencies, the third formed from the first by the double angle
    (no sincos): RSI 14 packed for it (e^{2iu} 6, the product with the
    source's constant 4, four accumulations) and the padding float4 read;
    piston 6 packed (e^{2iu} 4, two accumulations)."""
    if harmonic:
        assert nf == 3
        if kind == "rsi":  # per source pair: shared 14, two frequencies 7 + 2 scalar each, derived 14
            return {"fp32": (14.0 + 2 * 9.0 + 14.0) / 6, "mufu": 5.0 / 3, "lds": 6.0 / 6,
                    "fma_pipe": (14.0 + 2 * 8.0 + 14.0) / 3}
        return {"fp32": (10.0 + 2 * 5.0 + 6.0) / 6, "mufu": 5.0 / 3, "lds": 4.0 / 6,
                "fma_pipe": (10.0 + 2 * 4.0 + 6.0) / 3}
    if kind == "rsi":  # per source pair: shared 14 packed, per f 7 packed
        return {"fp32": 14.0 / (2 * nf) + 3.5 + 1.0, "mufu": 2.0 + 1.0 / nf, "lds": (2.0 + nf) / (2.0 * nf),
                "fma_pipe": 14.0 / nf + 7.0 + 1.0}
    return {"fp32": 10.0 / (2 * nf) + 1.5 + 1.0, "mufu": 2.0 + 1.0 / nf, "lds": 4.0 / (2.0 * nf),
            "fma_pipe": 10.0 / nf + 3.0 + 1.0}


def alu_roofline(kind: str, n_sm: int, clock_hz: float, ops: dict | None = None):
    """Peak pairs/s of a stage kernel at `clock_hz`: the tightest of the issue
    limit (one warp instruction per scheduler per clock), the MUFU limit and
    the FP32-pipe limit (128 FMA lanes per SM per clock; a packed f32x2
    instruction takes two of its cycles)."""
    o = ops or OPS[kind]
    lim = {"issue": (o["fp32"] + o.get("alu", 0) + o["mufu"] + o["lds"]) / (ISSUE_LANES_PER_SM * n_sm * clock_hz),
           "mufu": o["mufu"] / (MUFU_LANES_PER_SM * n_sm * clock_hz),
           "fma": o.get("fma_pipe", 0.0) / (ISSUE_LANES_PER_SM * n_sm * clock_hz)}
    worst = max(lim, key=lim.get)
    return 1.0 / lim[worst], worst


# ---------------------------------------------------------------------------
# CPU oracle sample
# ---------------------------------------------------------------------------
def oracle_sample(cfg, seconds: float, seed: int = 0):
    """Time the FP64 oracle on a bounded sample of one chain: all piston
    points onto m1 interface points, and all interface points onto m2 image
    pixels; m1, m2 sized for about `seconds` of work."""
    import numpy as np
    import oracle
    oracle.build()
    pc = cfg["piston"]
    it = cfg["interfaces"][0]
    last = cfg["interfaces"][-1]
    piston = oracle.make_points(dict(pc, kind="disk"), cfg["seed"], pc["set_id"], pc["n"])
    iface = oracle.make_points(it, cfg["seed"], it["set_id"], it["n"])
    lface = oracle.make_points(last, cfg["seed"], last["set_id"], last["n"])
    grid = oracle.grid_points(cfg["grid"])
    k1 = oracle.wavenumber(cfg["freq"], cfg["media"][0]["c"])
    kl = oracle.wavenumber(cfg["freq"], cfg["media"][len(cfg["interfaces"])]["c"])
    rng = np.random.default_rng(seed)
    sig = np.ones(last["n"], np.complex128)

    def run(m1, m2):
        s1 = rng.choice(it["n"], min(m1, it["n"]), replace=False)
        s2 = rng.choice(grid["x"].shape[0], min(m2, grid["x"].shape[0]), replace=False)
        t0 = time.perf_counter()
        phi1 = oracle.piston_field(piston, {k: iface[k][s1] for k in ("x", "y", "z")}, k1)
        oracle.rsi_field(lface, sig, {k: grid[k][s2] for k in ("x", "y", "z")}, kl)
        dt = time.perf_counter() - t0
        return dt, pc["n"] * len(s1) + last["n"] * len(s2), s1, phi1

    # rate probe with enough targets to keep every thread busy, then size the
    # sample for `seconds` of work at that rate
    m0 = 4 * oracle.default_threads()
    dt, pairs, _, _ = run(m0, m0)
    rate = pairs / dt
    m = max(16, int(seconds * rate / (pc["n"] + last["n"])))
    dt, pairs, s1, phi1 = run(m, m)
    return {"seconds": dt, "pairs": pairs, "rate": pairs / dt, "m": m,
            "iface_slots_natural": s1, "phi1": phi1, "threads": oracle.default_threads()}


GOLDEN = os.path.join(ROOT, "tests", "golden")


def image_error(got, want) -> dict:
    """Relative L2 error over the values and the worst value's error relative
    to the largest reference value."""
    import numpy as np
    got, want = np.asarray(got, np.complex128).ravel(), np.asarray(want, np.complex128).ravel()
    return {"rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
            "max_abs_over_max_ref": float(np.max(np.abs(got - want)) / np.max(np.abs(want))),
            "values": int(want.size)}


def golden_error(img, name: str):
    """image_error at the stored FP64-oracle pixels tests/golden/<name>.json
    (written by tests/golden/make_golden.py, which calls only the oracle)."""
    import numpy as np
    path = os.path.join(GOLDEN, name + ".json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    got = img.reshape(-1).cpu().numpy()[np.asarray(rec["pixels"])]
    return image_error(got, np.asarray(rec["re"]) + 1j * np.asarray(rec["im"]))


def single_core_rate(cfg, seconds: float = 4.0) -> float:
    """FP64 oracle pair rate on ONE host thread: all piston points onto m
    interface points of the workload, m sized for about `seconds`."""
    import numpy as np
    import oracle
    oracle.build()
    pc, it = cfg["piston"], cfg["interfaces"][0]
    piston = oracle.make_points(dict(pc, kind="disk"), cfg["seed"], pc["set_id"], pc["n"])
    iface = oracle.make_points(it, cfg["seed"], it["set_id"], it["n"])
    k1 = oracle.wavenumber(cfg["freq"], cfg["media"][0]["c"])

    def run(m):
        tg = {k: iface[k][:m] for k in ("x", "y", "z")}
        t0 = time.perf_counter()
        oracle.piston_field(piston, tg, k1, nthreads=1)
        return pc["n"] * m / (time.perf_counter() - t0)

    rate = run(8)
    m = int(min(it["n"], max(8, seconds * rate / pc["n"])))
    return run(m)


def cpu_leg_and_error(args, cfgs, pairs_step, images):
    """Rank 0: the FP64 oracle on the host cores (cpu_baseline) and the error
    of the timed step's own images against it.
      c2  the images of all three frequencies at the 1024 stored oracle pixels
          of each; the oracle timed on a bounded sample of the chain;
      c1, c3  the oracle runs the whole workload (timed in full), and the
          images are compared on every pixel.
    Each cpu_baseline also carries the oracle's rate on one thread."""
    import oracle
    name = args.config
    fp64 = cfgs[0]["precision"] == "fp64"
    err = {"tolerance": 1e-5 if fp64 else 1e-4}
    cpu = None
    if name == "c2":
        err["what"] = "the timed step's images, each frequency at its 1024 stored FP64-oracle pixels"
        for cfg, img in zip(cfgs, images):
            err[f"{cfg['freq'] / 1e6:g}MHz"] = golden_error(img, f"c2_{cfg['freq'] / 1e6:g}MHz")
        if not args.no_cpu_baseline:
            cfg = cfgs[min(1, len(cfgs) - 1)]
            smp = oracle_sample(cfg, args.cpu_seconds)
            cpu = {"value": smp["rate"], "unit": UNIT, "cores": smp["threads"], "kind": "oracle",
                   "sample": f"c2 at {cfg['freq'] / 1e6:g} MHz: all {cfg['piston']['n']} piston points "
                             f"onto {smp['m']} random interface points + all "
                             f"{cfg['interfaces'][0]['n']} interface points onto {smp['m']} random "
                             f"pixels ({smp['pairs']:.3g} pairs, {smp['seconds']:.1f} s), FP64",
                   "single_core_rate": single_core_rate(cfg)}
        return cpu, err
    labels = {"c1": ["5MHz"], "c3": ["flat", "curved"]}[name]
    if args.no_cpu_baseline:
        if name == "c3":
            err["what"] = "the timed step's images at 1024 stored FP64-oracle pixels each"
            for lab, img in zip(labels, images):
                err[lab] = golden_error(img, f"c3_{lab}")
            return None, err
    t0 = time.perf_counter()
    want = [oracle.field_image(c) for c in cfgs]
    dt = time.perf_counter() - t0
    err["what"] = "the timed step's images against the FP64 oracle's whole images, every pixel"
    for lab, img, w in zip(labels, images, want):
        err[lab] = image_error(img.cpu().numpy(), w)
    if not args.no_cpu_baseline:
        cpu = {"value": pairs_step / dt, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
               "sample": f"the whole {name} workload ({pairs_step:.3g} pairs, {dt:.1f} s), FP64",
               "single_core_rate": single_core_rate(cfgs[0])}
    return cpu, err


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def reduce_max(v: float, world: int):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(world: int, units_per_step_per_rank: float, steps: int, local_seconds: float):
    """Whole-job rate: units of all ranks over the slowest rank's time."""
    total_s = reduce_max(local_seconds, world)
    return total_s, world * units_per_step_per_rank * steps / total_s


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_ours(args):
    import torch
    from paper_2408_06765_gb300 import build, rsi
    world, rank, local = dist_setup()
    build.build()
    rsi.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfgs, pairs_step, pixels_step = workload(args.config)
    ws = rsi.Workspace(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    opts = {"variant": args.variant} if args.variant else None
    multi = (not args.no_multi and not args.variant and rsi.same_geometry(cfgs) and len(cfgs) <= 4
             and cfgs[0].get("precision", "fp32c") == "fp32c")

    sharded = world > 1
    if sharded:
        # one chain split over the ranks: every stage's targets divided among
        # them, one all-gather of the transmitted amplitudes per interface and
        # one of the image rows (shard.py); total work fixed as N grows
        from paper_2408_06765_gb300 import shard
        be = shard.LibrsiBackend(cfgs[0].get("precision", "fp32c"), device=dev)
        gather = shard.torch_allgather(world)
        counts = shard.row_counts(cfgs, world)
        groups = [cfgs] if multi else [[c] for c in cfgs]

        def step():
            out = []
            for grp in groups:
                _, rows = shard.run_rank(grp, rank, world, be, gather)
                local = (rows.reshape(len(grp), -1) if rows is not None else
                         torch.empty((len(grp), 0), dtype=torch.complex128, device=dev))
                full = gather(local, sum(counts), counts)
                out += [full[f].view(c["grid"]["nz"], c["grid"]["nx"]) for f, c in enumerate(grp)]
            return out
    else:
        def step():
            if multi:  # the frequencies share every point: one pass over the pair geometry
                return rsi.run_chain_multi(cfgs, fmt="c64", workspace=ws, device=dev)
            fmt = "c128" if cfgs[0]["precision"] == "fp64" else "c64"  # FP64 images keep their digits
            return [rsi.run_chain(c, fmt=fmt, workspace=ws, device=dev, stage_opts=opts).image for c in cfgs]

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    rsi.sync_status()

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    rsi.timing_enable(True)
    n0 = rsi.launch_count()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = rsi.launch_count() - n0
    barrier(world)
    clk = clocks.stop()
    rates = measure_unit_rates(rsi, torch)  # cross-check of the unit counts, GPU warm
    rsi_ms, rsi_n, rsi_pairs = rsi.timing_read(rsi.STAGE_RSI)
    pis_ms, pis_n, pis_pairs = rsi.timing_read(rsi.STAGE_PISTON)
    rsi.timing_enable(False)
    rsi.sync_status()
    # the job's work per step is one chain (2.58e11 pair terms for c2) whatever
    # the number of ranks: the rate is that over the slowest rank's time
    total_s = reduce_max(sum(step_ms) * 1e-3, world)
    value = pairs_step * args.steps / total_s
    last_images = step()
    torch.cuda.synchronize()

    # dominant kernel: the RSI stage kernel (interface -> image dominates)
    avg_s = rsi_ms * 1e-3 / max(1, rsi_n)
    achieved = (rsi_pairs / max(1, rsi_n)) / avg_s
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_hz = (clk["sm_mhz"] if clk and clk.get("sm_mhz") else
              rates["ffma"] / (ISSUE_LANES_PER_SM * n_sm) / 1e6) * 1e6
    nf = len(cfgs) if multi else 1
    # does the kernel form one frequency from another by the double angle?
    harm = multi and nf == 3 and rsi.stage_multi_shared_harmonic(
        rsi.stage_struct(rsi.STAGE_RSI, "fp32c", 1.0, 1.0),
        [rsi.wavenumber(c["freq"], c["media"][-1]["c"]) for c in cfgs])
    rsi_ops = multi_ops("rsi", nf, harm) if multi else OPS["rsi"]
    pis_ops = multi_ops("piston", nf, harm) if multi else OPS["piston"]
    peak, limiter = alu_roofline("rsi", n_sm, clk_hz, rsi_ops)
    pis_avg = pis_ms * 1e-3 / max(1, pis_n)
    pis_peak, _ = alu_roofline("piston", n_sm, clk_hz, pis_ops)
    roof = {"bound": "alu", "kernel": f"stage_multi_kernel<RSI, nf={nf}>" if multi else "stage_fp32_kernel<RSI>",
            "achieved": achieved / 1e9,
            "peak": peak / 1e9, "unit": "Gpair/s", "frac": achieved / peak, "traffic": None,
            "limiter": limiter,
            "ops_per_pair": rsi_ops, "harmonic_shared": bool(harm),
            "peak_source": "unit counts (4 issue slots of 32 lanes and 16 MUFU lanes per SM per clock) x "
                           f"{n_sm} SMs x the median SM clock of the timed region "
                           f"({clk_hz / 1e6:.0f} MHz)",
            "probe_rates_tops": {k: v / 1e12 for k, v in rates.items()},
            "probe_lanes_per_sm_clock": {k: v / (n_sm * clk_hz) for k, v in rates.items()},
            "avg_launch_ms": avg_s * 1e3, "launches": rsi_n,
            "piston_kernel": {"achieved": (pis_pairs / max(1, pis_n)) / max(pis_avg, 1e-12) / 1e9,
                              "peak": pis_peak / 1e9, "avg_launch_ms": pis_avg * 1e3,
                              "launches": pis_n}}
    if cfgs[0]["precision"] == "fp64":
        # FP64 pipe bound: the measured DFMA rate over the FP64-pipe thread
        # instructions per pair that ncu counted on the piston stage kernel
        # (sqrt, division and sincos in double are sequences of DFMA/DMUL/DADD)
        dfma = measure_unit_rates(rsi, torch, ("dfma",))["dfma"]
        ops64 = recorded_fp64_ops()
        pis_achieved = (pis_pairs / max(1, pis_n)) / max(pis_avg, 1e-12)
        peak64 = dfma / ops64 if ops64 else None
        roof = {"bound": "fp64", "kernel": "stage_fp64_kernel<PISTON> (the RSI stage's kernel is the same "
                                           "arithmetic plus the obliquity)",
                "achieved": pis_achieved / 1e9, "peak": peak64 / 1e9 if peak64 else None, "unit": "Gpair/s",
                "frac": pis_achieved / peak64 if peak64 else None, "traffic": None,
                "fp64_ops_per_pair": ops64, "dfma_rate_tops": dfma / 1e12,
                "dfma_lanes_per_sm_clock": dfma / (n_sm * clk_hz),
                "peak_source": "rsi_ubench DFMA probe (measured in this run) / FP64-pipe thread instructions "
                               "per pair counted by ncu (profiles/stage_fp64_c1_fp64_ops.md)",
                "rsi_kernel": {"achieved": achieved / 1e9, "avg_launch_ms": avg_s * 1e3, "launches": rsi_n},
                "avg_launch_ms": pis_avg * 1e3, "launches": pis_n}
    if cfgs[0]["precision"] != "fp64" and args.config == "c2":
        roof["traffic"] = recorded_traffic("stage_multi_kernel" if multi else "stage_fp32_kernel")

    e2e = None
    if not args.no_e2e:
        host = [torch.empty(tuple(im.shape), dtype=im.dtype, pin_memory=True) for im in last_images]
        d2h = sum(h.numel() * h.element_size() for h in host)
        e2e_s = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            imgs = step()
            for h, im in zip(host, imgs):
                h.copy_(im, non_blocking=True)
            torch.cuda.synchronize()
            e2e_s.append(time.perf_counter() - t0)
        e2e_value = pairs_step * args.steps / reduce_max(sum(e2e_s), world)
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
               "note": "inputs are scalar workload parameters passed by value through the "
                       "C ABI (no array inputs); the step's images are read back each step"}

    cpu, err = None, None
    if rank == 0:
        cpu, err = cpu_leg_and_error(args, cfgs, pairs_step, last_images)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None,
                "dtype": "f64" if cfgs[0]["precision"] == "fp64" else "f32",
                "data": "synthetic (seeded scrambled-Sobol points; workload parameters only)",
                "config": config_block(cfgs, world, args.config),
                "field_pts_per_s": pixels_step * args.steps / total_s,
                "rel_l2_err": err,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches, "gpu": torch.cuda.get_device_name(dev)}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 CPU oracle as the reference arm, on the host cores (rank 0)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfgs, _, _ = workload(args.config if args.config in DESCRIPTION else "c2")
    cfg = cfgs[min(1, len(cfgs) - 1)]
    per_step = max(2.0, min(20.0, 90.0 / max(1, args.steps + args.warmup)))
    for _ in range(max(1, args.warmup)):
        oracle_sample(cfg, 1.0, seed=99)
    rates, secs, pairs = [], 0.0, 0
    for s in range(args.steps):
        smp = oracle_sample(cfg, per_step, seed=s)
        rates.append(smp["rate"])
        secs += smp["seconds"]
        pairs += smp["pairs"]
    value = pairs / secs
    cpu = {"value": value, "unit": UNIT, "cores": smp["threads"], "kind": "oracle",
           "sample": f"per step: all piston points onto {smp['m']} interface points + all "
                     f"interface points onto {smp['m']} pixels of {cfg['name']}, FP64"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(1, args.warmup),
            "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block(cfgs, 1, args.config if args.config in DESCRIPTION else "c2"),
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_stage_case(args):
    """One RSI stage (2^18 interface points -> 65 536 pixels), `steps` times."""
    import torch
    from paper_2408_06765_gb300 import build, rsi
    from paper_2408_06765_gb300 import workloads as W
    build.build()
    cfg = W.c2_full_image(10e6)
    cfg["grid"] = dict(cfg["grid"], nx=256, nz=256)
    it = cfg["interfaces"][0]
    normals, c_img = rsi.NORMALS_Z, 5900.0
    if args.curved:  # c3's curved bottom surface (per-point normals) onto its 256^2 image in water
        cfg = W.c3_multilayer(curved=True)
        it = cfg["interfaces"][-1]
        normals, c_img = rsi.NORMALS_POINTS, cfg["media"][-1]["c"]
    pts = rsi.make_qmc_points(it, 0, it["set_id"], it["n"])
    grid = rsi.grid_points(cfg["grid"])
    sigma = torch.ones(it["n"], dtype=torch.complex128, device="cuda")
    ws = rsi.Workspace()
    shapes = [(args.tile, args.tpt, args.variant)]
    if args.sweep:
        shapes = [(t, q, v) for t in (64, 128, 256, 512) for q in (2, 4) for v in (1, 2, 3)]
    nf = args.nf
    if nf > 1:
        shapes = [(args.tile, 2, 0)]
        ks = [rsi.wavenumber(f, 5900.0) for f in (10e6, 5e6, 2.25e6, 1e6)[:nf]]
        sigma = torch.ones((nf, it["n"]), dtype=torch.complex128, device="cuda")
    for tile, tpt, variant in shapes:
        st = rsi.stage_struct(rsi.STAGE_RSI, "fp32c", rsi.wavenumber(cfg["freq"], c_img),
                              normals=normals, tile=tile, tpt=tpt, variant=variant)
        out = None
        times = []
        for _ in range(args.warmup + args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if nf > 1:
                out = rsi.propagate_stage_multi(st, ks, pts, sigma, grid, workspace=ws)
            else:
                out = rsi.propagate_stage(st, pts, sigma, grid, workspace=ws)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        rsi.sync_status()
        ms = min(times[args.warmup:])
        pairs = it["n"] * grid.n * nf
        print(json.dumps({"case": "stage", "curved": bool(args.curved), "nf": nf, "ms": ms,
                          "gpair_per_s": pairs / ms / 1e6,
                          "variant": variant, "tile": tile, "tpt": tpt,
                          "checksum": float(out.abs().sum().item())}), flush=True)


def run_batch_c4(args):
    """c4: 64 frequencies x 32 scan positions, uneven QMC counts, one graph."""
    import numpy as np
    import torch
    from paper_2408_06765_gb300 import build, rsi
    from paper_2408_06765_gb300 import workloads as W
    build.build()
    cfgs = W.c4_all()
    if args.instances:
        cfgs = cfgs[:args.instances]
    pairs = sum(W.pairs_of(c) for c in cfgs)
    pixels = sum(c["grid"]["nx"] * c["grid"]["nz"] for c in cfgs)
    b = rsi.Batch(cfgs, seed=0)
    for _ in range(max(3, args.warmup)):
        b.run()
    torch.cuda.synchronize()
    rsi.sync_status()
    clocks = ClockSampler(0)
    clocks.start()
    n0 = rsi.launch_count()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    rsi.sync_status()
    graph_launches = rsi.launch_count() - n0
    total_s = sum(ms) * 1e-3
    # batched vs the plain per-instance loop on the same GPU, on a seeded subset
    rng = np.random.default_rng(0)
    sub = sorted(rng.choice(len(cfgs), min(32, len(cfgs)), replace=False).tolist())
    sub_cfgs = [cfgs[i] for i in sub]
    sb = rsi.Batch(sub_cfgs, seed=0)
    sb.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sb.run()
    e1.record()
    e1.synchronize()
    batch_sub_ms = e0.elapsed_time(e1)
    ws = rsi.Workspace()
    plain = [rsi.run_chain(c, fmt="c64", workspace=ws).image for c in sub_cfgs]
    torch.cuda.synchronize()
    e0.record()
    plain = [rsi.run_chain(c, fmt="c64", workspace=ws).image for c in sub_cfgs]
    e1.record()
    e1.synchronize()
    plain_sub_ms = e0.elapsed_time(e1)
    errs = []
    for j, i in enumerate(sub):
        g = b.image(i).cpu().numpy().astype(np.complex128)
        p = plain[j].cpu().numpy().astype(np.complex128)
        errs.append(float(np.linalg.norm(g - p) / np.linalg.norm(p)))
    sub_pairs = sum(W.pairs_of(c) for c in sub_cfgs)
    # the FP64 oracle on 64 seeded instances (timed on the host cores) and
    # the batched images of those instances against it
    cpu, oracle_err = None, None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        pick = sorted(np.random.default_rng(64).choice(len(cfgs), min(64, len(cfgs)), replace=False).tolist())
        t0 = time.perf_counter()
        want = [oracle.field_image(cfgs[i]) for i in pick]
        dt = time.perf_counter() - t0
        opairs = sum(W.pairs_of(cfgs[i]) for i in pick)
        e = [image_error(b.image(i).cpu().numpy(), w) for i, w in zip(pick, want)]
        oracle_err = {"instances": len(pick), "max_rel_l2": max(x["rel_l2"] for x in e),
                      "median_rel_l2": float(np.median([x["rel_l2"] for x in e])),
                      "max_abs_over_max_ref": max(x["max_abs_over_max_ref"] for x in e), "tolerance": 1e-4}
        cpu = {"value": opairs / dt, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
               "sample": f"{len(pick)} seeded instances of the scan, whole chains ({opairs:.3g} pairs, "
                         f"{dt:.1f} s), FP64",
               "single_core_rate": single_core_rate(cfgs[pick[0]])}
    # step-level bound: every piston and RSI pair at its kernel's ALU (MUFU)
    # limit, at the median SM clock of the timed region; everything else in
    # the graph (points, transmission, prep, reduce, images) counts as overhead
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    clk_hz = (clk["sm_mhz"] if clk and clk.get("sm_mhz") else 2070.0) * 1e6
    pk_pis, _ = alu_roofline("piston", n_sm, clk_hz)
    pk_rsi, _ = alu_roofline("rsi", n_sm, clk_hz)
    pis_pairs = sum(int(c["piston"]["n"]) * int(c["interfaces"][0]["n"]) for c in cfgs)
    t_bound = pis_pairs / pk_pis + (pairs - pis_pairs) / pk_rsi
    t_step = total_s / args.steps
    line = {"metric": METRIC, "value": pairs * args.steps / total_s, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c4 batched broadband scan: 64 frequencies (1-10 MHz) x 32 "
                                   "x-positions, QMC counts round(2^(12+4U)), 128^2 image each, "
                                   "one CUDA graph with persistent stage kernels",
                       "instances": len(cfgs), "pairs_per_step": pairs},
            "field_pts_per_s": pixels * args.steps / total_s,
            "batched_vs_plain": {"instances": len(sub), "batch_ms": batch_sub_ms,
                                 "plain_loop_ms": plain_sub_ms,
                                 "batch_gpair_per_s": sub_pairs / batch_sub_ms / 1e6,
                                 "plain_gpair_per_s": sub_pairs / plain_sub_ms / 1e6,
                                 "max_rel_l2": max(errs), "tolerance": 1e-3},
            "rel_l2_err": oracle_err, "cpu_baseline": cpu,
            "roofline": {"bound": "alu", "kernel": "whole batched step: piston and RSI pairs at their "
                                                    "stage kernels' MUFU limits",
                         "achieved": pairs / t_step / 1e9, "peak": pairs / t_bound / 1e9, "unit": "Gpair/s",
                         "frac": t_bound / t_step, "traffic": None,
                         "peak_source": f"unit counts x {n_sm} SMs x the median SM clock of the timed region"},
            "graph_launches": graph_launches, "clocks": clk, "gpu": torch.cuda.get_device_name(0)}
    print(json.dumps(line), flush=True)
    sb.close()
    b.close()


def run_two_medium_f1(args):
    """f1: both media of c2's interface at 5 MHz with a 10 degree tilt
    (incident + reflected field in the water, transmitted field in the
    steel), timed like the c2 step; error against the stored oracle pixels."""
    import numpy as np
    import torch
    from paper_2408_06765_gb300 import build, rsi
    from paper_2408_06765_gb300 import workloads as W
    build.build()
    rsi.load()
    dev = torch.device("cuda", 0)
    cfg = W.f1_two_medium()
    pairs = rsi.two_medium_pairs(cfg)
    nx = int(cfg["grid_water"]["nx"])
    pixels = nx * (int(cfg["grid_water"]["nz"]) + int(cfg["grid_solid"]["nz"]))
    ws = rsi.Workspace(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    step = lambda: rsi.run_two_medium(cfg, fmt="c64", workspace=ws, device=dev)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    rsi.sync_status()
    clocks = ClockSampler(0)
    clocks.start()
    rsi.timing_enable(True)
    n0 = rsi.launch_count()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = step()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = rsi.launch_count() - n0
    clk = clocks.stop()
    rsi_ms, rsi_n, rsi_pairs = rsi.timing_read(rsi.STAGE_RSI)
    pis_ms, pis_n, pis_pairs = rsi.timing_read(rsi.STAGE_PISTON)
    rsi.timing_enable(False)
    rsi.sync_status()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_hz = (clk["sm_mhz"] if clk and clk.get("sm_mhz") else 2070.0) * 1e6
    peak, limiter = alu_roofline("rsi", n_sm, clk_hz)
    achieved = rsi_pairs / (rsi_ms * 1e-3)
    err = None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "f1_5MHz.json")
    if os.path.exists(path):
        rec = json.load(open(path))
        got = res.image.reshape(-1).cpu().numpy().astype(np.complex128)[np.asarray(rec["pixels"])]
        want = np.asarray(rec["re"]) + 1j * np.asarray(rec["im"])
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    total_s = sum(ms) * 1e-3
    line = {"metric": METRIC, "value": pairs * args.steps / total_s, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scrambled-Sobol points; workload parameters only)",
            "config": {"workload": "f1 two-medium image: 6.35 mm piston tilted 10 deg, 5 MHz, water -> "
                                   "steel at 50 mm, 2^16 piston x 2^18 interface (80 mm); 512 x 256 "
                                   "pixels of incident + reflected field in the water and 512 x 256 "
                                   "of transmitted field in the steel",
                       "pairs_per_step": pairs, "l2_flush": "256 MiB write before every step"},
            "field_pts_per_s": pixels * args.steps / total_s,
            "rel_l2_err": {"image_vs_stored_fp64_oracle_1024_pixels": err, "tolerance": 1e-4},
            "roofline": {"bound": "alu", "kernel": "stage_fp32_kernel<RSI> (reflected + transmitted)",
                         "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
                         "frac": achieved / peak, "traffic": None, "limiter": limiter,
                         "launches": rsi_n,
                         "piston_kernel_gpair_s": pis_pairs / max(pis_ms * 1e-3, 1e-12) / 1e9},
            "clocks": clk, "gpu_launches": launches, "gpu": torch.cuda.get_device_name(dev)}
    print(json.dumps(line), flush=True)


def run_raytrace_f2(args):
    """f2: the ray-tracing model (Sec. 2.2) on c2's geometry with a 10 degree
    tilt at 5 MHz: 2^16 transducer points onto a 512^2 image in the steel;
    error against the stored oracle pixels."""
    import numpy as np
    import torch
    from paper_2408_06765_gb300 import build, rsi
    from paper_2408_06765_gb300 import workloads as W
    build.build()
    rsi.load()
    dev = torch.device("cuda", 0)
    cfg = W.f2_ray_tracing(n_piston=1 << 14, nx=256, nz=256) if args.small else W.f2_ray_tracing()
    g = cfg["grid"]
    pixels = int(g["nx"]) * int(g["nz"])
    pairs = int(cfg["piston"]["n"]) * pixels
    ws = rsi.Workspace(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    step = lambda: rsi.run_raytrace(cfg, fmt="c64", workspace=ws, device=dev)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    rsi.sync_status()
    clocks = ClockSampler(0)
    clocks.start()
    rsi.timing_enable(True)
    n0 = rsi.launch_count()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        img = step()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = rsi.launch_count() - n0
    clk = clocks.stop()
    rt_ms, rt_n, rt_pairs = rsi.timing_read(rsi.TIMING_RAYTRACE)
    rsi.timing_enable(False)
    rsi.sync_status()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_hz = (clk["sm_mhz"] if clk and clk.get("sm_mhz") else 2070.0) * 1e6
    peak, limiter = alu_roofline("raytrace", n_sm, clk_hz)
    achieved = rt_pairs / (rt_ms * 1e-3)
    err = None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "f2_5MHz.json")
    if os.path.exists(path) and not args.small:
        rec = json.load(open(path))
        got = img.reshape(-1).cpu().numpy().astype(np.complex128)[np.asarray(rec["pixels"])]
        want = np.asarray(rec["re"]) + 1j * np.asarray(rec["im"])
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    total_s = sum(ms) * 1e-3
    line = {"metric": METRIC, "value": pairs * args.steps / total_s, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scrambled-Sobol points; workload parameters only)",
            "config": {"workload": "f2 ray-tracing model: 6.35 mm piston tilted 10 deg, 2^16 points, 5 MHz, "
                                   "water -> steel at 50 mm, 512^2 image over 80 x 60 mm in the steel",
                       "pairs_per_step": pairs, "l2_flush": "256 MiB write before every step"},
            "field_pts_per_s": pixels * args.steps / total_s,
            "rel_l2_err": {"image_vs_stored_fp64_oracle_1024_pixels": err, "tolerance": 1e-4},
            "roofline": {"bound": "alu", "kernel": "raytrace_kernel", "achieved": achieved / 1e9,
                         "peak": peak / 1e9, "unit": "Gpair/s", "frac": achieved / peak, "traffic": None,
                         "limiter": limiter, "ops_per_pair": OPS["raytrace"], "launches": rt_n},
            "clocks": clk, "gpu_launches": launches, "gpu": torch.cuda.get_device_name(dev)}
    print(json.dumps(line), flush=True)


def run_gemm_case(args):
    """The surrogate's dominant kernel alone: the output-layer GEMM of batch-1024
    inference, [1024 x 512] x [512 x 32768] + bias with an f32 output (or the
    --gemm-shape M,N,K), on random BF16 operands (the GEMM engine of --engine);
    each of the `steps` samples averages 20 back-to-back launches."""
    import torch
    from paper_2408_06765_gb300 import build, rsi
    build.build()
    rsi.load()
    g = torch.Generator(device="cuda").manual_seed(0)
    M, N, K = (int(x) for x in args.gemm_shape.split(","))
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    out = torch.empty(M, N, device="cuda")
    reps = 20  # back-to-back launches per sample: the host's per-call work overlaps the kernels
    times = []
    for _ in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            rsi.nn_gemm("f32", A, B, out_f32=out, bias=bias, engine=args.engine)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / reps)
    rsi.sync_status()
    ms = min(times[args.warmup:])
    nbytes = 2.0 * (A.numel() + B.numel()) + 4.0 * (out.numel() + bias.numel())
    print(json.dumps({"case": "gemm", "engine": args.engine, "M": M, "N": N, "K": K, "ms": ms,
                      "tflops": 2.0 * M * N * K / ms / 1e9, "gbytes_per_s": nbytes / ms / 1e6}), flush=True)


def run_train_case(args):
    """The surrogate's training step alone (random rows, forward, backward,
    Adam, replayed from the CUDA graph) on a coordinate network of the c5
    architecture and synthetic targets (the cost does not depend on them)."""
    import numpy as np
    import torch
    from paper_2408_06765_gb300 import build, rsi, surrogate
    build.build()
    rsi.load()
    net = surrogate.CoordNet(n_freq=args.c5_freq, width=args.c5_width, depth=args.c5_depth, rows=args.c5_rows,
                             engine=args.engine)
    rng = np.random.default_rng(0)
    n = 256
    params = surrogate.LO + (surrogate.HI - surrogate.LO) * rng.random((n, 5))
    g = torch.Generator(device="cuda").manual_seed(0)
    img = torch.randn(n, 128, 128, dtype=torch.complex64, device="cuda", generator=g)
    tset = surrogate.TrainingSet(net, params, img)
    steps = args.steps + max(3, args.warmup) + 1
    lrs = [1e-4] * steps
    seeds = np.arange(steps, dtype=np.int64)
    net.rows_random(tset.params, tset.targets, tset.log_rms, seed=0)
    net.forward()
    net.backward()
    net.adam()
    net.step_count += 1
    tr = surrogate.GraphedTrainer(net, tset, lrs, seeds)
    for _ in range(max(3, args.warmup)):
        tr.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        tr.step()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"case": "train", "rows": net.rows, "width": net.width, "depth": net.depth,
                      "ms_per_step": ms, "rows_per_s": net.rows / (ms * 1e-3)}), flush=True)


def run_infer_case(args):
    """The surrogate's inference alone (rsi_nn_infer: rows, hidden layers,
    head, per-field assembly and carrier) at 1024 fields per call on a
    randomly initialised coordinate network of the c5 architecture (the cost
    does not depend on the weights), `steps` calls of seeded parameter rows
    already on the device."""
    import numpy as np
    import torch
    from paper_2408_06765_gb300 import build, rsi, surrogate
    build.build()
    rsi.load()
    net = surrogate.CoordNet(n_freq=args.c5_freq, width=args.c5_width, depth=args.c5_depth, rows=args.c5_rows,
                             engine=args.engine)
    rng = np.random.default_rng(0)
    q = torch.tensor(surrogate.LO + (surrogate.HI - surrogate.LO) * rng.random((1024, 5)), device="cuda")
    out = torch.empty(1024, surrogate.NPIX * 2, dtype=torch.float32, device="cuda")
    for _ in range(max(1, args.warmup)):
        net.infer(q, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        net.infer(q, out)
    e1.record()
    e1.synchronize()
    rsi.sync_status()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"case": "infer", "engine": args.engine, "fields_per_call": 1024, "calls": args.steps,
                      "ms_per_call": ms, "fields_per_s": 1024 / (ms * 1e-3)}), flush=True)


def run_sequences_f3(args):
    """f3: Halton (the paper's points) against scrambled Sobol, side by side:
    on-axis error of the flat piston (closed form) and of the focused cap
    (O'Neil's closed form) for N = 2^8 .. 2^18 points, FP64 stage so that
    only the QMC error shows, the fitted convergence slopes, and the point
    generation rate of both sequences."""
    import numpy as np
    import torch
    from paper_2408_06765_gb300 import build, rsi
    build.build()
    rsi.load()
    mm, f, c = 1e-3, 2.5e6, 1480.0
    k = 2 * math.pi * f / c
    a, R = 6.35 * mm, 33 * mm
    z = np.linspace(5 * mm, 60 * mm, 56)
    flat = 1.0 / (1j * k) * (np.exp(1j * k * z) - np.exp(1j * k * np.sqrt(z * z + a * a)))
    zc = np.linspace(3 * mm, 45 * mm, 43)
    zc = zc[np.abs(zc - R) > 0.5 * mm]
    r_rim = np.sqrt(R * R + (R - zc) ** 2 - 2 * R * (R - zc) * math.sqrt(1 - (a / R) ** 2))
    cap = -(R / (1j * k * (R - zc))) * (np.exp(1j * k * r_rim) - np.exp(1j * k * zc))
    surfaces = {"flat": ({"kind": "disk", "centre": (0.0, 0.0, 0.0), "a": a}, z, flat),
                "cap": ({"kind": "cap", "centre": (0.0, 0.0, 0.0), "a": a, "R": R}, zc, cap)}
    ws = rsi.Workspace()
    st = rsi.stage_struct(rsi.STAGE_PISTON, "fp64", k, 1.0)
    out = {}
    for sname, (surf, zs, exact) in surfaces.items():
        tgt = rsi.Points(len(zs))
        for key, vals in (("X", 0 * zs), ("Y", 0 * zs), ("Z", zs)):
            tgt.field(key).copy_(torch.tensor(vals, dtype=torch.float64))
        for key, vals in (("XH", 0 * zs), ("XL", 0 * zs), ("YH", 0 * zs), ("YL", 0 * zs)):
            tgt.field(key).copy_(torch.tensor(vals, dtype=torch.float32))
        tgt.field("ZH").copy_(torch.tensor(zs, dtype=torch.float32))
        tgt.field("ZL").copy_(torch.tensor(zs - zs.astype(np.float32).astype(np.float64), dtype=torch.float32))
        for seq in ("sobol", "halton"):
            rows = []
            for m in range(8, 19):
                src = rsi.make_qmc_points(dict(surf, sequence=seq), 0, 0, 1 << m)
                phi = rsi.propagate_stage(st, src, None, tgt, workspace=ws).cpu().numpy()
                rows.append([1 << m, float(np.linalg.norm(phi - exact) / np.linalg.norm(exact))])
            n = np.log([r[0] for r in rows])
            e = np.log([r[1] for r in rows])
            out[f"{sname}_{seq}"] = {"n_and_rel_l2": rows, "slope": float(np.polyfit(n, e, 1)[0])}
    # generation rate: 2^24 points of each sequence on the piston
    rates = {}
    for seq in ("sobol", "halton"):
        pts = rsi.Points(1 << 24)
        surf = {"kind": "disk", "centre": (0.0, 0.0, 0.0), "a": a, "sequence": seq}
        for _ in range(3):
            rsi.make_qmc_points(surf, 0, 0, 1 << 24, out=pts)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            rsi.make_qmc_points(surf, 0, 0, 1 << 24, out=pts)
        e1.record()
        e1.synchronize()
        rates[seq] = 10 * (1 << 24) / (e0.elapsed_time(e1) * 1e-3)
    rsi.sync_status()
    line = {"config": {"workload": "f3 QMC point sets: on-axis field of a 6.35 mm flat piston and of the "
                                   "focused cap (R = 33 mm) at 2.5 MHz in water against their closed forms, "
                                   "N = 2^8 .. 2^18 points, FP64 stage",
                       "scrambled_sobol_seed": 0},
            "convergence": out, "points_per_s": rates, "gpu": torch.cuda.get_device_name(0)}
    print(json.dumps(line), flush=True)


def run_focused_f4(args):
    """f4: the focused transducer through both models (RSI chain and ray
    tracing) at full size; errors against the stored oracle pixels."""
    import numpy as np
    import torch
    from paper_2408_06765_gb300 import build, rsi
    from paper_2408_06765_gb300 import workloads as W
    build.build()
    rsi.load()
    dev = torch.device("cuda", 0)
    cfg = W.f4_focused()
    g = cfg["grid"]
    pixels = int(g["nx"]) * int(g["nz"])
    ws = rsi.Workspace(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    models = {"rsi_chain": (lambda: rsi.run_chain(cfg, fmt="c64", workspace=ws, device=dev).image, W.pairs_of(cfg)),
              "ray_tracing": (lambda: rsi.run_raytrace(cfg, fmt="c64", workspace=ws, device=dev),
                              int(cfg["piston"]["n"]) * pixels)}
    res = {}
    clocks = ClockSampler(0)
    clocks.start()
    for name, (step, pairs) in models.items():
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            img = step()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        err = None
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                            ("f4_chain" if name == "rsi_chain" else "f4_ray") + "_2.5MHz.json")
        if os.path.exists(path):
            rec = json.load(open(path))
            got = img.reshape(-1).cpu().numpy().astype(np.complex128)[np.asarray(rec["pixels"])]
            want = np.asarray(rec["re"]) + 1j * np.asarray(rec["im"])
            err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        t = sum(ms) * 1e-3
        res[name] = {"pair_terms_per_s": pairs * args.steps / t, "ms_per_image": t * 1e3 / args.steps,
                     "pairs": pairs, "field_pts_per_s": pixels * args.steps / t,
                     "rel_l2_vs_stored_oracle_1024_pixels": err}
    clk = clocks.stop()
    rsi.sync_status()
    line = {"config": {"workload": "f4 focused transducer: spherical cap a = 6.35 mm, R = 33 mm, 2^16 points, "
                                   "2.5 MHz, 10 mm water -> steel, 2^18 interface points on 40 mm, 512^2 image "
                                   "over 20 x 30 mm of steel around the focus",
                       "l2_flush": "256 MiB write before every step"},
            "steps": args.steps, "warmup": max(3, args.warmup), "models": res, "clocks": clk,
            "gpu": torch.cuda.get_device_name(dev)}
    print(json.dumps(line), flush=True)


def measured_peaks():
    """Copy bandwidth and bf16 GEMM throughput measured on this GPU model
    (MEASURED_PEAKS.json beside this file), else the fallback figures."""
    f = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(f) as fh:
            d = json.load(fh)
        d["source"] = "measured"
        return d
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def run_surrogate_c5(args):
    """c5: generate fields with the batched RSI path, train the coordinate
    network on them, and measure its held-out error against the RSI path,
    the fraction of queries its gate serves, and the images per second it
    infers."""
    import numpy as np
    import torch
    from paper_2408_06765_gb300 import build, rsi, surrogate
    from paper_2408_06765_gb300 import workloads as W
    build.build()
    n = args.fields
    n_p, n_i = 1 << args.c5_piston_log2, 1 << args.c5_iface_log2
    params = W.c5_params(n, seed=0)
    t0 = time.perf_counter()
    imgs = surrogate.rsi_images(params, n_piston=n_p, n_iface=n_i)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    n_hold = max(256, n // 10)
    if n_hold >= n:
        raise SystemExit("c5 needs more than 256 fields")
    tr, ho = slice(0, n - n_hold), slice(n - n_hold, n)
    net = surrogate.CoordNet(n_freq=args.c5_freq, width=args.c5_width, depth=args.c5_depth, rows=args.c5_rows,
                             engine=args.engine)
    # train on the tilts the network can serve: near and past the critical
    # angle the refracted beam grazes the interface, those fields cost most of
    # the loss and the gate sends them to the RSI path anyway
    keep = np.nonzero(np.degrees(np.abs(params[tr][:, 1])) < args.c5_train_tilt_max)[0]
    tset = surrogate.TrainingSet(net, params[tr][keep], imgs[tr][torch.tensor(keep, device="cuda")])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = surrogate.train(net, tset, steps=args.c5_steps, lr=args.lr)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    hp = params[ho]
    hp_d = torch.tensor(hp, device="cuda")
    pred = net.infer(hp_d)
    torch.cuda.synchronize()
    errs = surrogate.rel_errors(pred, imgs[ho]).cpu().numpy()
    tilt = np.abs(hp[:, 1])
    pre, post = tilt < surrogate.CRIT, tilt >= surrogate.CRIT
    f_mhz = hp[:, 3] / 1e6
    # the gate: the k-nearest held-out error estimate, leave-one-out over the
    # held-out set (each query's own error excluded from its estimate)
    tmax = math.radians(args.c5_train_tilt_max)
    sur = surrogate.Surrogate(net, hp, errs, tilt_max=tmax)
    est = np.array([surrogate.Surrogate(net, np.delete(hp, i, 0), np.delete(errs, i), tilt_max=tmax)
                    .error_estimate(hp[i:i + 1])[0] for i in range(len(hp))]) if len(hp) <= 4096 \
        else sur.error_estimate(hp)
    served = est <= 1e-2
    # inference rate: batches of the network's whole-field chunk size
    per = net.rows // surrogate.NPIX
    nb = max(per, (1024 // per) * per)
    q = torch.tensor(params[:nb], device="cuda")
    out = torch.empty(nb, surrogate.NPIX * 2, dtype=torch.float32, device="cuda")
    for _ in range(2):
        net.infer(q, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 5
    for _ in range(reps):
        net.infer(q, out)
    e1.record()
    e1.synchronize()
    inf_s = e0.elapsed_time(e1) * 1e-3 / reps
    nn_fields_s = nb / inf_s
    rsi_fields_s = n / gen_s
    # the dominant kernel: one hidden layer's GEMM over a whole chunk of rows
    # (M = rows, N = K = width), timed alone
    R, Wd = net.rows, net.width
    A = torch.randn(R, Wd, device="cuda").to(torch.bfloat16)
    Bm = torch.randn(Wd, Wd, device="cuda").to(torch.bfloat16)
    bias = torch.zeros(Wd, device="cuda")
    zf = torch.empty(R, Wd, device="cuda")
    hb = torch.empty(R, Wd, dtype=torch.bfloat16, device="cuda")
    gemm = lambda: rsi.nn_gemm("bias_silu", A, Bm, out_f32=zf, out_bf16=hb, bias=bias, engine=args.engine)
    for _ in range(3):
        gemm()
    e0.record()
    for _ in range(20):
        gemm()
    e1.record()
    e1.synchronize()
    gemm_ms = e0.elapsed_time(e1) / 20
    flops = 2.0 * R * Wd * Wd
    peaks = measured_peaks()
    tf = flops / (gemm_ms * 1e-3) / 1e12
    gemm_bytes = 2.0 * (R * Wd + Wd * Wd) + 4.0 * R * Wd + 2.0 * R * Wd
    # JSON-safe statistics: outside its training tilts the network extrapolates
    # without bound (the gate never serves those queries)
    fin = lambda v: float(v) if np.isfinite(v) else None
    med = lambda m: fin(np.median(errs[m])) if m.any() else None
    trained = np.degrees(tilt) < args.c5_train_tilt_max
    # the error left after the best complex scale per field (the shape)
    pr, rf = pred.reshape(len(errs), -1), imgs[ho].reshape(len(errs), -1)
    alpha = (pr.conj() * rf).sum(1) / (pr.conj() * pr).sum(1)
    shape_errs = surrogate.rel_errors(alpha[:, None] * pr, rf).cpu().numpy()[trained]
    tdeg = np.degrees(tilt)
    line = {"config": {"workload": "c5 learned surrogate: coordinate network per pixel (9 row inputs in the "
                                   "refracted-beam frame -> Fourier features -> hidden SiLU layers -> re, im, "
                                   "log rms), BF16 weights, FP32 accumulation",
                       "fields": n, "held_out": int(len(errs)), "steps": args.c5_steps, "rows_per_step": net.rows,
                       "trained_on": f"{len(keep)} of the {n - n_hold} training fields, |tilt| < {args.c5_train_tilt_max:g} deg",
                       "n_freq": net.n_freq, "width": net.width, "depth": net.depth,
                       "rsi_points": [n_p, n_i]},
            "rsi_generation_s": gen_s, "rsi_fields_per_s": rsi_fields_s,
            "train_s": train_s, "final_train_loss": losses[-1], "train_loss_curve": losses, "lr": args.lr,
            "held_out_rel_l2": {"median": fin(np.median(errs)), "p90": fin(np.quantile(errs, 0.9)),
                                "within_training_tilts": {"fields": int(trained.sum()),
                                                          "median": med(trained),
                                                          "mean": fin(errs[trained].mean()),
                                                          "p90": fin(np.quantile(errs[trained], 0.9)),
                                                          "max": fin(errs[trained].max())}},
            "held_out_median_pre_critical": med(pre), "held_out_median_post_critical": med(post),
            "held_out_shape_only_median_within_training_tilts": fin(np.median(shape_errs)),
            "held_out_median_by_tilt_deg": {f"{a}-{b}": med((tdeg >= a) & (tdeg < b))
                                            for a, b in ((0, 5), (5, 10), (10, 13), (13, 14.5), (14.5, 15))},
            "held_out_median_by_frequency": {f"{lo}-{lo + 2}MHz": med((f_mhz >= lo) & (f_mhz < lo + 2))
                                             for lo in (2, 4, 6, 8)},
            "held_out_fraction_below": {k: float(np.mean(errs <= float(k))) for k in ("3e-3", "1e-2", "3e-2", "1e-1")},
            "gate": {"threshold": 1e-2, "estimate": "mean error of the 8 nearest held-out fields (leave-one-out)",
                     "served_fraction": float(served.mean()),
                     "served_true_error_median": float(np.median(errs[served])) if served.any() else None,
                     "served_true_error_max": float(errs[served].max()) if served.any() else None},
            "surrogate_fields_per_s": nn_fields_s, "infer_batch": nb,
            "speedup_vs_rsi": nn_fields_s / rsi_fields_s,
            # the hidden-layer GEMM does 2 width^2 flop per row against 2 width (A) + 4 width
            # (FP32 z) + 2 width (BF16 h) bytes: 128 flop per byte at width 512, below the
            # ridge of the measured peaks (~286), so HBM bounds it; both fractions reported
            "roofline": {"kernel": f"hidden-layer GEMM {R} x {Wd} x {Wd} (bias + SiLU epilogue)", "bound": "hbm",
                         "achieved": gemm_bytes / (gemm_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": gemm_bytes / (gemm_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "traffic": None,
                         "ms": gemm_ms, "algorithmic_bytes": gemm_bytes,
                         "flop_per_byte": flops / gemm_bytes,
                         "ridge_flop_per_byte": peaks["bf16_tflops"] * 1e12 / (peaks["hbm_gbs"] * 1e9),
                         "peak_source": peaks["source"] + " copy bandwidth",
                         "tensor": {"achieved": tf, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                                    "frac": tf / peaks["bf16_tflops"], "peak_source": peaks["source"] + " bf16 burst"}},
            "engine": args.engine, "gpu": torch.cuda.get_device_name(0)}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.config == "c5" and args.impl == "ours":
        run_surrogate_c5(args)
    elif args.config == "f1" and args.impl == "ours":
        run_two_medium_f1(args)
    elif args.config == "f2" and args.impl == "ours":
        run_raytrace_f2(args)
    elif args.config == "f3" and args.impl == "ours":
        run_sequences_f3(args)
    elif args.config == "f4" and args.impl == "ours":
        run_focused_f4(args)
    elif args.config == "c4" and args.impl == "ours" and args.case == "chain":
        run_batch_c4(args)
    elif args.case == "stage":
        run_stage_case(args)
    elif args.case == "gemm":
        run_gemm_case(args)
    elif args.case == "infer":
        run_infer_case(args)
    elif args.case == "train":
        run_train_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
