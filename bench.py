#!/usr/bin/env python
"""Benchmark of the far/near-field evaluation: pair interactions per second
(phi and E) of charged BEM triangles and rectangles by distance-ratio-banded
Gaussian cubature with an analytic near field (arXiv:1606.03743, Sec. 4-6).

Workload (one step): phi and E at 1,000,000 field points inside coaxial
cylinder electrodes meshed with 100,000 flat rectangles and 50,000 end-cap
triangles (150,000 elements), all rule bands in use, through the C ABI
(bem_eval) on device-resident inputs.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)

Multi-GPU (torchrun): every rank evaluates its own 1M-point batch against the
whole mesh (weak scaling, no collective on the data path); the timed region
is bracketed by barriers and the slowest rank's time is used.
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

import synth  # noqa: E402

METRIC = "pair interactions/s (phi+E) at stated rel. error vs FP64; p50/p99 query latency"
UNIT = "pairs/s"
FP32_LANES = 128  # FP32 lanes per SM (nominal; the measured rate is the denominator)
WORKLOAD = ("coaxial cylinders r=1.0/1.2 len 4: 2 x 200x250 flat rectangles + 2 end caps of 25000 triangles "
            "(150000 elements, sigma~N(1,0.2)); 1000000 field points uniform in r<0.95, |z|<1.9")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--points", type=int, default=1_000_000)
    ap.add_argument("--fp64-points", type=int, default=16384, help="batch for the FP64-path comparison line")
    ap.add_argument("--cpu-sample", type=int, default=8192, help="points of the oracle CPU baseline sample")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, FP64 comparison and CPU baseline")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving (latency) measurement")
    ap.add_argument("--no-assembly", action="store_true", help="skip the collocation-assembly measurement")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-tick", type=int, default=32768, help="points per serving tick (larger requests split)")
    ap.add_argument("--no-large", action="store_true", help="skip the 500k-element x 4M-point mixed vs FP64 run")
    ap.add_argument("--grad-points", type=int, default=16384, help="points of the FP64 field-gradient line")
    ap.add_argument("--grad-points-mixed", type=int, default=262144, help="points of the mixed field-gradient line")
    ap.add_argument("--large-points", type=int, default=4_000_000)
    ap.add_argument("--large-fp64-points", type=int, default=32768)
    ap.add_argument("--large-oracle-points", type=int, default=2048)
    ap.add_argument("--band-fit", action="store_true",
                    help="instead of the benchmark: time the far kernel with every far pair forced into one rule, "
                         "for each rule, and fit its cycles per node and per (warp, element)")
    a = ap.parse_args()
    a.warmup = max(a.warmup, 3)
    return a


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background.
    Started before the warm-up (so that nvidia-smi's own start-up stays out of
    the timed region); only the samples between mark_start() and mark_end()
    are reported."""

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None
        self.t0, self.t1 = None, None

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_end(self):
        self.t1 = time.monotonic()

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.monotonic(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = [r for t, r in self.rows
                if (self.t0 is None or t >= self.t0) and (self.t1 is None or t <= self.t1 + 0.2)]
        if not rows:  # a timed region shorter than one sampling period
            rows = [r for _, r in self.rows]
        self.rows = rows
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 8:
                for nm, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def far_traffic_from_profile():
    """DRAM bytes per far-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    src = os.path.join(ROOT, "paper_1606_03743_gb300", "csrc", "k_far.cu")
    prof = os.path.join(ROOT, "profiles", "k_far_coax150k_1M.md")
    if not os.path.exists(prof):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    txt = open(prof).read()
    m_sha = re.search(r"k_far\.cu sha256\[:16\]:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram bytes per launch \(full workload\):\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_b or m_sha.group(1) != sha:
        return None
    return float(m_b.group(1))


def measured_peaks(bem, sms: int) -> dict:
    """Throughput of the pipes that bound the far-field kernel, measured on
    this GPU by the library's own microbenchmark kernels (bem_peak_rate: every
    SM full of independent FFMA, FFMA2, MUFU.RSQ or DFMA chains, best of three
    launches timed with CUDA events, the SM clock read in the kernel).  The
    FP32 pipe peak is the better of the scalar and packed FMA rates (lane
    operations: an FMA counts once)."""
    kinds = {"ffma": bem.PEAK_FFMA, "ffma2": bem.PEAK_FFMA2, "rsqrt": bem.PEAK_RSQRT, "dfma": bem.PEAK_DFMA}
    out = {}
    for name, k in kinds.items():
        r = bem.bem_peak_rate(k)
        out[name] = {"tops": r["ops_per_s"] / 1e12, "ms": r["ms"], "sm_mhz": r["sm_mhz"],
                     "lanes_per_sm_per_clock": r["ops_per_s"] / (sms * r["sm_mhz"] * 1e6) if r["sm_mhz"] else None}
    out["fp32_tops"] = max(out["ffma"]["tops"], out["ffma2"]["tops"])
    out["sms"] = sms
    out["how"] = ("bem_peak_rate: 2048 threads per SM, 8 independent chains of one instruction per thread, "
                  "~50 ms launches, best of 3 (CUDA events); SM MHz from clock64 over %globaltimer")
    return out


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def measured_hbm_gbs() -> tuple[float, str]:
    """HBM copy bandwidth from MEASURED_PEAKS.json beside this file, else the
    fallback figure of an earlier GB300 measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s, an earlier GB300 measurement)"


def algorithmic_work_phi(stats: np.ndarray) -> float:
    """FP-pipe operations of potential-only far pairs (assembly rows, matvec):
    per pair 8 to classify it, per node 8 (r_i: 3, r^2: 3, q_i / r: 1, sum: 1)
    plus one rsqrt."""
    nodes = {0: [0, 33, 19, 12, 7, 4], 1: [0, 33, 17, 12, 7, 4]}
    return sum(float(stats[6 * t + b]) * (8 + 8 * nodes[t][b]) for t in (0, 1) for b in range(1, 6))


def algorithmic_work(stats: np.ndarray) -> tuple[float, float, float]:
    """Work the method needs for the far pairs of one step, from the pair
    counts per distance-ratio band.  FP32-pipe operations (an FMA is one
    operation): per pair 8 to classify it (P - Q_cen: 3, its square: 3,
    compare: 2), per Gaussian node 13 (r_i = P - Q_i: 3, r^2: 3, q_i / r: 1,
    phi sum: 1, 1 / r^2: 1, q_i / r^3: 1, E sum: 3) plus one rsqrt (Eq. 4.1).
    Also the same work in flops (FMA = 2): 8 + 18 per node.
    Returns (ops, rsqrts, flops)."""
    nodes = {0: [0, 33, 19, 12, 7, 4], 1: [0, 33, 17, 12, 7, 4]}
    ops = rsq = flops = 0.0
    for t in (0, 1):
        for b in range(1, 6):
            pairs = float(stats[6 * t + b])
            ops += pairs * (8 + 13 * nodes[t][b])
            flops += pairs * (8 + 18 * nodes[t][b])
            rsq += pairs * nodes[t][b]
    return ops, rsq, flops


def cores_used(n_threads: int) -> int:
    return n_threads


# ------------------------------------------------------------------ reference arm (CPU oracle)
def run_reference(a, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    mesh = synth.coax_mesh(seed=2)
    pts = synth.coax_points(seed=2, n=a.points)
    n_sample = 256
    nt = oracle.max_threads()
    sample = pts[:n_sample]
    for _ in range(min(a.warmup, 1)):
        oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, sample[:16], nthreads=nt)
    times = []
    for k in range(a.steps):
        sl = pts[(k * n_sample) % a.points:][:n_sample]
        t0 = time.perf_counter()
        oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, sl, nthreads=nt)
        times.append(time.perf_counter() - t0)
    pairs = n_sample * mesh.n
    value = pairs * a.steps / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_elements": mesh.n, "n_points": a.points,
                       "step": f"{n_sample} of the {a.points} points against all elements (bounded CPU sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": f"{n_sample} points x {mesh.n} elements per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)
    if a.band_fit:
        return band_fit(a)

    import torch
    import paper_1606_03743_gb300 as bem
    from paper_1606_03743_gb300 import shard

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    prec = bem.MIXED if a.precision == "mixed" else bem.FP64
    mesh = synth.coax_mesh(seed=2)
    pts = synth.coax_points(seed=shard.rank_seed(2, rank), n=a.points)  # each rank its own batch
    dev = torch.device("cuda", local)
    m = bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                 torch.from_numpy(mesh.sigma).to(dev), precision=prec)
    p_d = torch.from_numpy(pts).to(dev)
    phi = torch.empty(a.points, dtype=torch.float64, device=dev)
    E = torch.empty((a.points, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (126 MB)
    stream = torch.cuda.current_stream()

    def step():
        bem.bem_eval(m.handle, p_d, phi, E, stream=stream.cuda_stream)

    # band statistics of this workload and the pipe peaks (outside the timed region)
    m.set_stats(True)
    step()
    stats = m.last_stats()
    m.set_stats(False)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks(bem, sms)
    m.set_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(a.warmup):  # the timed step exactly (the first L2 flush loads its kernel: ~250 ms once)
        flush.zero_()
        step()

    barrier()
    clocks.mark_start()
    l0 = bem.bem_kernel_launches()
    far_ms = []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(a.steps):
        flush.zero_()
        step()
        far_ms.append(float(m.last_times()[1]))
    t_end.record(stream)
    barrier()
    clocks.mark_end()
    launches = bem.bem_kernel_launches() - l0
    ck = clocks.stop()
    m.set_timing(False)
    ms = t_start.elapsed_time(t_end)
    ms = shard.slowest_rank_ms(ms, dist, dev)
    pairs_step = float(a.points) * mesh.n
    value = shard.job_rate(world * pairs_step * a.steps, ms)

    # roofline of the dominant kernel (far-field cubature), from its own events:
    # the FP32 pipe bounds it (measured FMA rate), the MUFU pipe's rsqrt rate second
    ops, rsq, flops = algorithmic_work(stats)
    far_avg = statistics.mean(far_ms)
    peak_ops = peaks["fp32_tops"]  # T FP32-pipe lane ops/s, measured
    derived_ops = sms * FP32_LANES * 2070e6 / 1e12  # unit counts x maximum SM clock
    achieved = ops / (far_avg * 1e-3) / 1e12
    mufu_frac = rsq / (far_avg * 1e-3) / (peaks["rsqrt"]["tops"] * 1e12)
    flop_frac = flops / (far_avg * 1e-3) / (2 * peak_ops * 1e12)
    traffic = far_traffic_from_profile()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64 mixed" if prec == bem.MIXED else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_elements": mesh.n, "n_points_per_gpu": a.points,
                       "precision": a.precision, "parallelism": f"points sharded, {world} GPU(s)",
                       "l2": "256 MiB buffer written between steps (inside the timed region)"},
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Tops/s",
                         "frac": achieved / peak_ops, "traffic": traffic,
                         "kernel": "k_far (far-field cubature)", "kernel_ms": far_avg,
                         "peak_note": ("FP32 pipe, measured (of measured): the better of the FFMA and FFMA2 "
                                       "microbenchmark rates in lane operations per second (an FMA is one op)"),
                         "frac_of_derived_peak": achieved / derived_ops, "derived_peak": derived_ops,
                         "derived_peak_note": f"{sms} SMs x {FP32_LANES} lanes x 2070 MHz",
                         "work_note": "algorithmic FP32 ops per far pair: 8 + 13 x nodes of its rule",
                         "mufu_frac": mufu_frac,
                         "mufu_peak_note": ("MUFU rsqrt, measured: %.2f T/s = %.1f lanes per SM per clock"
                                            % (peaks["rsqrt"]["tops"], peaks["rsqrt"]["lanes_per_sm_per_clock"] or 0)),
                         "flop_frac_fma2": flop_frac},
            "peaks_measured": peaks,
            "band_pairs": {"triangle": [int(x) for x in stats[0:6]], "rectangle": [int(x) for x in stats[6:12]],
                           "order": "analytic, 33, 19|17, 12, 7, 4 points"},
            "far_kernel_work": {"warp_element_uniform": int(stats[13]), "warp_element_mixed": int(stats[14]),
                                "algorithmic_ops": ops,
                                "node_evals_executed": int(stats[15]),
                                "node_evals_algorithmic": int(rsq),
                                "executed_over_algorithmic": float(stats[15]) / rsq if rsq else None},
            "clocks": ck}

    if not a.no_extras:
        line["e2e"] = end_to_end(a, bem, torch, m, mesh, pts, stream, dist, dev, world, barrier)
    if rank == 0 and world == 1 and not a.no_extras:
        line.update(extras(a, bem, torch, m, mesh, pts, prec, stream, phi, E, peaks))
    if rank == 0 and world == 1 and not a.no_serving:
        line["serving"] = serving(a, bem, torch)
        lat = line["serving"]["mixed"]
        line["latency"] = {"p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"], "workload": line["serving"]["workload"]}
    if rank == 0 and world == 1 and not a.no_assembly:
        line["assembly"] = assembly(a, bem, torch, peaks)
    if rank == 0 and world == 1 and not a.no_extras:
        line["node_table_ablation"] = node_table_ablation(a, bem, torch, mesh, p_d, phi, E, stream, far_avg, ops,
                                                          peak_ops)
    if rank == 0 and world == 1 and not a.no_large:
        line["large_mixed_vs_fp64"] = large_mixed_vs_fp64(a, bem, torch)
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def end_to_end(a, bem, torch, m, mesh, pts, stream, dist, dev, world, barrier):
    """The metric through the C ABI with pinned host buffers, the host-to-device
    copy of the points and the device-to-host copy of phi and E inside the timed
    region; every rank times its own batch, the slowest rank counts."""
    from paper_1606_03743_gb300 import shard
    hp = torch.from_numpy(pts).pin_memory()
    hphi = torch.empty(a.points, dtype=torch.float64).pin_memory()
    hE = torch.empty((a.points, 3), dtype=torch.float64).pin_memory()
    bem.bem_eval(m.handle, hp, hphi, hE, stream=stream.cuda_stream)
    ts = []
    for _ in range(3):
        barrier()
        t0 = time.perf_counter()
        bem.bem_eval(m.handle, hp, hphi, hE, stream=stream.cuda_stream)  # returns with the results on the host
        ts.append(time.perf_counter() - t0)
    e2e_ms = shard.slowest_rank_ms(statistics.median(ts) * 1e3, dist, dev)
    return {"value": shard.job_rate(world * float(a.points) * mesh.n, e2e_ms), "unit": UNIT,
            "h2d_bytes_per_step": int(hp.numel() * 8), "d2h_bytes_per_step": int((hphi.numel() + hE.numel()) * 8),
            "ms_per_step": e2e_ms, "timing": "host clock around the call, median of 3, slowest rank"}


def extras(a, bem, torch, m, mesh, pts, prec, stream, phi_d, E_d, peaks):
    """End-to-end (host buffers), FP64-path comparison, CPU oracle baseline and accuracy."""
    out = {}
    # ---- the plain FP64 kernel on the same GPU (smaller batch: it is ~50x slower)
    dev = phi_d.device
    m64 = bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                   torch.from_numpy(mesh.sigma).to(dev), precision=bem.FP64)
    n64 = min(a.fp64_points, a.points)
    p64 = torch.from_numpy(pts[:n64]).to(dev)
    f64phi = torch.empty(n64, dtype=torch.float64, device=dev)
    f64E = torch.empty((n64, 3), dtype=torch.float64, device=dev)
    m64.set_stats(True)  # band counts of this batch (untimed)
    bem.bem_eval(m64.handle, p64, f64phi, f64E, stream=stream.cuda_stream)
    stats64 = m64.last_stats()
    m64.set_stats(False)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    m64.set_timing(True)
    calls, far64 = [], []
    for _ in range(3):
        t0.record(stream)
        bem.bem_eval(m64.handle, p64, f64phi, f64E, stream=stream.cuda_stream)
        t1.record(stream)
        torch.cuda.synchronize()
        calls.append(t0.elapsed_time(t1))
        far64.append(float(m64.last_times()[1]))
    m64.set_timing(False)
    ms64 = statistics.median(calls)
    ops64, _, _ = algorithmic_work(stats64)
    far64_ms = statistics.median(far64)
    fp64_roof = {"bound": "alu", "kernel": "k_far (FP64 path)", "kernel_ms": far64_ms,
                 "achieved": ops64 / (far64_ms * 1e-3) / 1e12, "peak": peaks["dfma"]["tops"], "unit": "Tops/s",
                 "frac": ops64 / (far64_ms * 1e-3) / 1e12 / peaks["dfma"]["tops"],
                 "peak_note": "FP64 pipe, measured DFMA rate (of measured)",
                 "work_note": ("the same algorithmic count as the mixed path (8 + 13 x nodes per far pair) on the "
                               "FP64 pipe; the FP64 reciprocal square root is a multi-instruction sequence, so "
                               "the kernel issues more FP64 operations than this count"),
                 "timing": "median of 3 calls, kernel time from the library's CUDA events"}
    mix_rate = None
    # same batch on the mixed mesh for a like-for-like ratio
    if prec == bem.MIXED:
        mphi = torch.empty(n64, dtype=torch.float64, device=dev)
        mE = torch.empty((n64, 3), dtype=torch.float64, device=dev)
        bem.bem_eval(m.handle, p64, mphi, mE, stream=stream.cuda_stream)
        t0.record(stream)
        bem.bem_eval(m.handle, p64, mphi, mE, stream=stream.cuda_stream)
        t1.record(stream)
        torch.cuda.synchronize()
        mix_rate = n64 * mesh.n / (t0.elapsed_time(t1) * 1e-3)
    out["fp64_path"] = {"value": n64 * mesh.n / (ms64 * 1e-3), "unit": UNIT, "n_points": n64, "ms": ms64,
                        "roofline": fp64_roof,
                        "mixed_same_batch": mix_rate,
                        "mixed_over_fp64": (mix_rate / (n64 * mesh.n / (ms64 * 1e-3))) if mix_rate else None}

    # ---- CPU oracle baseline on a bounded sample + accuracy of this run at those points
    import oracle
    oracle.build()
    ns = min(a.cpu_sample, a.points)
    nt = oracle.max_threads()
    t0c = time.perf_counter()
    rphi, rE, mdr, esum = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts[:ns], nthreads=nt,
                                            return_min_dr=True, return_esum=True)
    cpu_s = time.perf_counter() - t0c
    out["cpu_baseline"] = {"value": ns * mesh.n / cpu_s, "unit": UNIT, "cores": nt, "kind": "oracle",
                           "cpu_model": cpu_model(),
                           "sample": f"first {ns} of the {a.points} points x all {mesh.n} elements ({cpu_s:.1f} s)"}
    gphi = phi_d[:ns].cpu().numpy()
    gE = E_d[:ns].cpu().numpy()
    g64phi = f64phi.cpu().numpy()
    g64E = f64E.cpu().numpy()
    k = min(ns, n64)

    # ---- field gradient: the far kernel's gradient modes (FP64 mesh and mixed mesh) + analytic near field
    ngo = min(a.grad_points, a.points, 512)
    t0c = time.perf_counter()
    Gref, gsum = oracle.eval_grad(mesh.types, mesh.verts, mesh.sigma, pts[:ngo], nthreads=nt, return_gsum=True)
    kap_g = gsum / np.abs(Gref).max(axis=1)  # cancellation in G, as kappa for E
    cpu_g = time.perf_counter() - t0c
    grads = {}
    for gkey, gmesh, ng in (("f64", m64, min(a.grad_points, a.points)),
                            ("mixed", m, min(a.grad_points_mixed, a.points))):
        pg = torch.from_numpy(pts[:ng]).to(dev)
        Gd = torch.empty((ng, 6), dtype=torch.float64, device=dev)
        bem.bem_eval_grad(gmesh.handle, pg, Gd, stream=stream.cuda_stream)
        t0.record(stream)
        bem.bem_eval_grad(gmesh.handle, pg, Gd, stream=stream.cuda_stream)
        t1.record(stream)
        torch.cuda.synchronize()
        msg = t0.elapsed_time(t1)
        Gg = Gd[:ngo].cpu().numpy()
        gerr = np.abs(Gg - Gref).max(axis=1) / np.abs(Gref).max(axis=1)
        gsel = (mdr[:ngo] >= 3) & (kap_g <= 100)
        grads[gkey] = {"value": ng * mesh.n / (msg * 1e-3), "unit": UNIT, "n_points": ng, "ms": msg,
                       "max_rel_err_vs_oracle": float(gerr[gsel].max()),
                       "max_rel_err_vs_oracle_min_dr3": float(gerr[mdr[:ngo] >= 3].max()),
                       "max_rel_err_vs_oracle_all": float(gerr.max()),
                       "max_err_over_gsum": float((np.abs(Gg - Gref).max(axis=1) / gsum).max()),
                       "max_rel_trace": float((np.abs(Gg[:, :3].sum(1)) / np.abs(Gg).max(axis=1)).max())}
        del Gd, pg
    out["field_gradient"] = {**grads, "oracle_pairs_per_s": ngo * mesh.n / cpu_g, "oracle_points": ngo,
                             "error": "max over points of max |dG| / max |G| (components); gated: min DR >= 3 "
                                      "and kappa_G = sum_j max|G_j| / max|G| <= 100",
                             "kappa_g_quantiles": [float(q) for q in np.quantile(kap_g, [0.5, 0.9, 0.99, 1.0])],
                             "gated_points": int(((mdr[:ngo] >= 3) & (kap_g <= 100)).sum()),
                             "mixed_over_f64": grads["mixed"]["value"] / grads["f64"]["value"]}

    # ---- varying densities over the elements (the same mesh): linear, sigma varying by up to ~30 %
    # across each element, and quadratic, with second-order terms of a few per cent on top
    rng_d = np.random.default_rng(31)
    lin = np.stack([mesh.sigma, *(rng_d.normal(0.0, 0.15, (2, mesh.n)) * mesh.sigma)], axis=1)
    quad = np.concatenate([lin, (rng_d.normal(0.0, 0.05, (3, mesh.n)) * mesh.sigma).T], axis=1)
    varying = [("linear_density", lin, m.set_sigma_linear, oracle.eval_linear,
                "sigma = s_c + s_a alpha + s_b beta per element, s_a, s_b ~ N(0, 0.15 s_c)"),
               ("quadratic_density", quad, m.set_sigma_quadratic, oracle.eval_quad,
                "sigma = c0 + c1 alpha + c2 beta + c3 alpha^2 + c4 alpha beta + c5 beta^2, "
                "c1, c2 ~ N(0, 0.15 c0), c3, c4, c5 ~ N(0, 0.05 c0)")]
    lphi = torch.empty(a.points, dtype=torch.float64, device=dev)
    lE = torch.empty((a.points, 3), dtype=torch.float64, device=dev)
    p_all = torch.from_numpy(pts).to(dev)
    nlo = 512
    far = mdr[:nlo] >= 3
    kap = (esum / np.linalg.norm(rE, axis=1))[:nlo]
    sel = far & (kap <= 100)
    ngv = min(a.grad_points_mixed, a.points)
    pgv = torch.from_numpy(pts[:ngv]).to(dev)
    Gv = torch.empty((ngv, 6), dtype=torch.float64, device=dev)
    nvo = 256
    for key, coef, setter, ref_fn, desc in varying:
        setter(coef)
        bem.bem_eval(m.handle, p_all, lphi, lE, stream=stream.cuda_stream)
        t0.record(stream)
        bem.bem_eval(m.handle, p_all, lphi, lE, stream=stream.cuda_stream)
        t1.record(stream)
        torch.cuda.synchronize()
        msl = t0.elapsed_time(t1)
        # the field gradient with the same densities
        bem.bem_eval_grad(m.handle, pgv, Gv, stream=stream.cuda_stream)
        t0.record(stream)
        bem.bem_eval_grad(m.handle, pgv, Gv, stream=stream.cuda_stream)
        t1.record(stream)
        torch.cuda.synchronize()
        msg_v = t0.elapsed_time(t1)
        m.set_sigma(mesh.sigma)
        Gvr, gsv = oracle.eval_grad_var(mesh.types, mesh.verts, coef, pts[:nvo], nthreads=nt, return_gsum=True)
        Gvg = Gv[:nvo].cpu().numpy()
        gverr = np.abs(Gvg - Gvr).max(axis=1) / np.abs(Gvr).max(axis=1)
        gvsel = (mdr[:nvo] >= 3) & (gsv / np.abs(Gvr).max(axis=1) <= 100)
        lref_phi, lref_E = ref_fn(mesh.types, mesh.verts, coef, pts[:nlo], nthreads=nt)
        gl_phi, gl_E = lphi[:nlo].cpu().numpy(), lE[:nlo].cpu().numpy()
        out[key] = {
            "value": a.points * mesh.n / (msl * 1e-3), "unit": UNIT, "ms": msl, "precision": a.precision,
            "density": desc,
            "max_rel_phi_vs_oracle": float((np.abs(gl_phi - lref_phi) / np.abs(lref_phi))[sel].max()),
            "max_rel_E_vs_oracle": float((np.linalg.norm(gl_E - lref_E, axis=1)
                                          / np.linalg.norm(lref_E, axis=1))[sel].max()),
            "oracle_points": nlo, "gate_points": "min DR >= 3 and kappa (constant density) <= 100",
            "field_gradient": {"value": ngv * mesh.n / (msg_v * 1e-3), "unit": UNIT, "n_points": ngv, "ms": msg_v,
                               "max_rel_err_vs_oracle": float(gverr[gvsel].max()), "oracle_points": nvo,
                               "gate_points": "min DR >= 3 and kappa_G <= 100"}}

    out["accuracy_vs_oracle"] = accuracy_report(gphi, gE, g64phi[:k], g64E[:k], rphi, rE, mdr, esum)
    out["accuracy_vs_oracle"]["run_precision"] = a.precision
    out["accuracy_vs_oracle"]["points"] = ns
    m64.close()
    return out


def node_table_ablation(a, bem, torch, mesh, p_d, phi, E, stream, far_ms_fly, ops, peak):
    """The same workload with the nodes precomputed per element (the paper's
    Sec. 6 / Table 4 comparison) against the on-the-fly kernel timed above."""
    dev = p_d.device
    m = bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                 torch.from_numpy(mesh.sigma).to(dev), precision=bem.MIXED, node_table=True)
    phi2 = torch.empty_like(phi)
    E2 = torch.empty_like(E)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    bem.bem_eval(m.handle, p_d, phi2, E2, stream=stream.cuda_stream)
    m.set_timing(True)
    far = []
    for _ in range(3):
        flush.zero_()
        bem.bem_eval(m.handle, p_d, phi2, E2, stream=stream.cuda_stream)
        far.append(float(m.last_times()[1]))
    m.set_timing(False)
    torch.cuda.synchronize()
    d_phi = ((phi2 - phi).abs() / phi.abs()).max().item()
    d_E = ((E2 - E).norm(dim=1) / E.norm(dim=1)).max().item()
    ms = statistics.mean(far)
    out = {"far_kernel_ms_on_the_fly": far_ms_fly, "far_kernel_ms_node_table": ms,
           "frac_node_table": ops / (ms * 1e-3) / 1e12 / peak,
           "table_bytes": int(mesh.n * 75 * 48),  # 75 node slots x three float4 records
           "max_rel_diff_vs_on_the_fly": {"phi": d_phi, "E": d_E}}
    m.close()
    return out


def accuracy_report(gphi, gE, g64phi, g64E, rphi, rE, mdr, esum):
    """Relative errors of phi, of the vector E and of |E| against the oracle,
    grouped by the distance-ratio band of each point's nearest element
    (the default triangle limits, Sec. 4 reading: near < 4.5 <= 33-point < 12
    <= 19-point < 30 <= 12-point < 120 <= 7-point < 2250 <= 4-point), plus the
    points at DR >= 3 from every element whose field does not cancel by more
    than 100 (kappa = sum_j |E_j| / |E|)."""
    kappa = esum / np.linalg.norm(rE, axis=1)

    def errs(p, e, sel):
        n = len(p)
        sel = sel[:n]
        ep = np.abs(p - rphi[:n]) / np.abs(rphi[:n])
        nE = np.linalg.norm(rE[:n], axis=1)
        dE = np.linalg.norm(e - rE[:n], axis=1)
        eE = dE / nE
        eA = np.abs(np.linalg.norm(e, axis=1) - nE) / nE
        eEc = dE / esum[:n]  # |dE| / sum_j |E_j|: error relative to the size of the terms
        if not sel.any():
            return {"n": 0}
        return {"max_rel_phi": float(ep[sel].max()), "max_rel_E": float(eE[sel].max()),
                "max_rel_absE": float(eA[sel].max()), "mean_rel_phi": float(ep[sel].mean()),
                "mean_rel_E": float(eE[sel].mean()), "max_E_over_sum_abs_Ej": float(eEc[sel].max()),
                "n": int(sel.sum())}

    edges = [0, 4.5, 12, 30, 120, 2250, np.inf]
    names = ["near (<4.5)", "33-pt [4.5,12)", "19-pt [12,30)", "12-pt [30,120)", "7-pt [120,2250)",
             "4-pt (>=2250)"]
    groups = {"min_DR>=3,kappa<=100": (mdr >= 3) & (kappa <= 100), "min_DR>=3": mdr >= 3}
    for lo, hi, nm in zip(edges[:-1], edges[1:], names):
        groups["min_DR " + nm] = (mdr >= lo) & (mdr < hi)
    return {"bands": {b: errs(gphi, gE, s) for b, s in groups.items()},
            "fp64_path": {b: errs(g64phi, g64E, s) for b, s in groups.items()},
            "kappa": {"definition": "sum_j |E_j| / |E| (oracle)", "median": float(np.median(kappa)),
                      "p99": float(np.percentile(kappa, 99)), "max": float(kappa.max()),
                      "frac_above_100": float((kappa > 100).mean())},
            "band_of_point": "band of the smallest distance ratio D/L over all elements"}


def large_mixed_vs_fp64(a, bem, torch):
    """500000-element coaxial mesh and 4000000 field points: the mixed path
    over all points, the plain FP64 kernel on a subset, both against the
    oracle on a bounded sample, errors per distance-ratio band."""
    import oracle
    oracle.build()
    mesh = synth.coax_mesh_large(seed=4)
    pts = synth.coax_points(seed=4, n=a.large_points)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    out = {"workload": (f"{mesh.n} elements (coaxial, 400x500 rectangles per cylinder + 2 x 50000 cap triangles), "
                        f"{a.large_points} field points")}
    res = {}
    for prec, name, n in ((bem.MIXED, "mixed", a.large_points), (bem.FP64, "fp64", a.large_fp64_points)):
        m = bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                     torch.from_numpy(mesh.sigma).to(dev), precision=prec)
        p_d = torch.from_numpy(pts[:n]).to(dev)
        phi = torch.empty(n, dtype=torch.float64, device=dev)
        E = torch.empty((n, 3), dtype=torch.float64, device=dev)
        bem.bem_eval(m.handle, p_d, phi, E, stream=stream.cuda_stream)  # sizes the workspace
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        bem.bem_eval(m.handle, p_d, phi, E, stream=stream.cuda_stream)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        out[name] = {"value": n * mesh.n / (ms * 1e-3), "unit": UNIT, "n_points": n, "ms": ms}
        res[name] = (phi[: a.large_oracle_points].cpu().numpy(), E[: a.large_oracle_points].cpu().numpy())
        m.close()
        del p_d, phi, E
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    ns = a.large_oracle_points
    t0c = time.perf_counter()
    rphi, rE, mdr, esum = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts[:ns],
                                            nthreads=oracle.max_threads(), return_min_dr=True, return_esum=True)
    out["oracle_s"] = time.perf_counter() - t0c
    out["accuracy_vs_oracle"] = accuracy_report(res["mixed"][0], res["mixed"][1], res["fp64"][0], res["fp64"][1],
                                                rphi, rE, mdr, esum)
    out["accuracy_vs_oracle"]["points"] = ns
    return out


SIZE_CLASSES = ((1, 1000), (1001, 10000), (10001, 100000))


def latency_classes(ms, sizes) -> dict:
    """p50 / p99 latency per request-size class (points)."""
    out = {}
    for lo, hi in SIZE_CLASSES:
        sel = (sizes >= lo) & (sizes <= hi)
        if sel.any():
            out[f"{lo}-{hi}"] = {"n": int(sel.sum()), "p50_ms": float(np.percentile(ms[sel], 50)),
                                 "p99_ms": float(np.percentile(ms[sel], 99)), "max_ms": float(ms[sel].max())}
    return out


def run_server(bem, m, reqs, rate, n_el, tick):
    """Poisson arrivals at `rate` requests/s into a server on mesh m; returns
    latency statistics (measured by the library, submission to results on
    the host), overall and per request-size class, and throughput."""
    srv = bem.Server(m, max_points_per_tick=tick)
    rng = np.random.default_rng(55)
    gaps = rng.exponential(1.0 / rate, len(reqs))
    tickets = []
    t0 = time.perf_counter()
    t_next = t0
    for r, g in zip(reqs, gaps):
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        tickets.append(srv.submit(r))
        t_next += g
    for t in tickets:
        srv.wait(t, timeout=600)
    wall = time.perf_counter() - t0
    st = srv.stats()
    ms, sizes = srv.latencies()
    srv.close()
    pts = sum(len(r) for r in reqs)
    return {"requests": len(reqs), "points": int(pts), "rate_req_per_s": rate, "p50_ms": st["p50_ms"],
            "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "by_size": latency_classes(ms, sizes),
            "points_per_tick": int(st["points_per_tick"]), "ticks": int(st["ticks"]),
            "fallback_ticks": int(st["fallback_ticks"]), "graph_launches": int(st["graph_launches"]),
            "throughput_pairs_per_s": pts * n_el / wall, "wall_s": wall}


def serving(a, bem, torch):
    """Serving workload: the 500k-element coaxial mesh resident on the GPU,
    query batches of floor(10^U[0,5]) points (clipped to [1, 1e5]) along
    helical tracks, Poisson arrivals at 70 % of the measured capacity."""
    mesh = synth.coax_mesh_large(seed=4)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"workload": (f"{mesh.n} elements (coaxial, 400x500 rectangles per cylinder + 100000 cap triangles); "
                        f"{a.serve_requests} requests of 10^U[0,5] points on helices, Poisson arrivals at 70% "
                        "of measured capacity")}
    reqs = synth.helix_requests(seed=5, n_req=a.serve_requests)
    for prec, name in ((bem.MIXED, "mixed"), (bem.FP64, "fp64")):
        m = bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                     torch.from_numpy(mesh.sigma).to(dev), precision=prec)
        # capacity in points/s from one evaluation of a representative batch
        probe = synth.coax_points(seed=6, n=65536 if prec == bem.MIXED else 2048)
        m.eval(probe[:1024])
        t0 = time.perf_counter()
        m.eval(probe)
        cap_pts = len(probe) / (time.perf_counter() - t0)
        if prec == bem.MIXED:
            sel = reqs
        else:  # the FP64 kernel is ~30x slower: a capped subset (sizes <= 2000), compared like for like below
            sel = [r for r in reqs if len(r) <= 2000][:20]
        mean_size = float(np.mean([len(r) for r in sel]))
        rate = 0.7 * cap_pts / mean_size
        out[name] = run_server(bem, m, sel, rate, mesh.n, a.serve_tick)
        out[name]["capacity_points_per_s"] = cap_pts
        if prec == bem.FP64:
            # the same capped subset on the mixed path, at the same arrival rate
            m.close()
            m = bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                         torch.from_numpy(mesh.sigma).to(dev), precision=bem.MIXED)
            out["mixed_same_subset_as_fp64"] = run_server(bem, m, sel, rate, mesh.n, a.serve_tick)
        m.close()
    return out


def assembly(a, bem, torch, peaks):
    """Collocation assembly: 20000 elements (geodesic sphere + inner
    cylinder), the dense 20000 x 20000 FP64 matrix on the device, plus the
    matrix-free product."""
    mesh = synth.sphere_cylinder_mesh(seed=3)
    col = synth.collocation_points(mesh)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"workload": f"{mesh.n} elements (18000-triangle geodesic sphere + 2000-rectangle cylinder), "
                       f"{mesh.n} x {mesh.n} FP64 matrix; solve with the sphere at 1 V, the cylinder at 0 V"}
    c_d = torch.from_numpy(col).to(dev)
    A = torch.empty((mesh.n, mesh.n), dtype=torch.float64, device=dev)
    x = torch.from_numpy(mesh.sigma).to(dev)
    y = torch.empty(mesh.n, dtype=torch.float64, device=dev)
    hbm, hbm_note = measured_hbm_gbs()
    for prec, name in ((bem.FP64, "fp64"), (bem.MIXED, "mixed")):
        m = bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                     torch.from_numpy(mesh.sigma).to(dev), precision=prec)
        m.set_stats(True)  # band counts (untimed)
        bem.bem_assemble(m.handle, c_d, A)
        st = m.last_stats()
        m.set_stats(False)
        torch.cuda.synchronize()
        tas = []
        for _ in range(3):
            t0 = time.perf_counter()
            bem.bem_assemble(m.handle, c_d, A)
            torch.cuda.synchronize()
            tas.append(time.perf_counter() - t0)
        ta = statistics.median(tas)
        ops_a = algorithmic_work_phi(st)
        pipe = peaks["dfma"]["tops"] if prec == bem.FP64 else peaks["fp32_tops"]
        bem.bem_matvec(m.handle, x, y)
        t0 = time.perf_counter()
        bem.bem_matvec(m.handle, x, y)
        torch.cuda.synchronize()
        tm = time.perf_counter() - t0
        # the product's phases from the library's CUDA events: its far kernel does the assembly's
        # far pairs (potential only), which lean on the MUFU pipe (one rsqrt per node)
        m.set_timing(True)
        bem.bem_matvec(m.handle, x, y)
        torch.cuda.synchronize()
        ph = [float(t) for t in m.last_times()]
        m.set_timing(False)
        _, rsq_a, _ = algorithmic_work(st)
        nbytes = 8.0 * mesh.n * mesh.n
        out[name] = {"assemble_ms": ta * 1e3, "matrix_write_GBps": nbytes / ta / 1e9,
                     "hbm_frac": nbytes / ta / 1e9 / hbm, "hbm_peak_gbs": hbm, "hbm_peak_note": hbm_note,
                     "pipe_frac": ops_a / ta / 1e12 / pipe,
                     "pipe_note": ("algorithmic ops (8 per far pair + 8 per node, potential only) over the whole "
                                   "call's time, against the measured " +
                                   ("DFMA" if prec == bem.FP64 else "FP32 FMA") + " rate"),
                     "entries_per_s": mesh.n * mesh.n / ta, "matvec_ms": tm * 1e3,
                     "matvec_pairs_per_s": mesh.n * mesh.n / tm,
                     "matvec_phases_ms": {"sort": ph[0], "far": ph[1], "near": ph[2], "finalize": ph[3]},
                     "matvec_far_pipe_frac": ops_a / (ph[1] * 1e-3) / 1e12 / pipe,
                     "timing": "median of 3 calls, host clock with a device synchronize"}
        if prec == bem.MIXED:
            out[name]["matvec_far_mufu_frac"] = rsq_a / (ph[1] * 1e-3) / (peaks["rsqrt"]["tops"] * 1e12)
            out[name]["mufu_note"] = ("algorithmic rsqrt (one per node of the far pairs) over the product's far-kernel "
                                      "time, against the measured MUFU rsqrt rate: the potential-only node needs 4 "
                                      "packed FP32 operations and one rsqrt, so MUFU bounds it")
        # the electrode problem: sphere (triangles) at 1 V, inner cylinder at 0 V
        rhs = torch.from_numpy(np.where(mesh.types == 0, 1.0, 0.0)).to(dev)
        sig = torch.empty(mesh.n, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = bem.bem_solve(m.handle, rhs, sig)
        torch.cuda.synchronize()
        out[name]["solve"] = {"ms": (time.perf_counter() - t0) * 1e3, "products": info["products"],
                              "relative_residual": info["residual"], "converged": info["converged"],
                              "method": "restarted GMRES(50), Jacobi right preconditioner, matrix-free products"}
        if prec == bem.FP64:
            t0 = time.perf_counter()
            info = bem.bem_solve(m.handle, rhs, sig, refine=True)
            torch.cuda.synchronize()
            out[name]["solve_refined"] = {"ms": (time.perf_counter() - t0) * 1e3, "products": info["products"],
                                          "relative_residual": info["residual"], "converged": info["converged"],
                                          "method": "FP64 residuals, GMRES on mixed-precision products to 1e-6"}
        m.close()
    del A
    return out


def band_fit(a) -> int:
    """The far kernel (mixed, phi and E) on the benchmark workload with every
    far pair forced into one rule by the band limits (the near limit kept),
    for each of the five rules: its CUDA-event time, the (warp, element)
    pairs and node evaluations from the kernel's statistics, and a
    least-squares fit of SM sub-partition cycles per (warp, element) pair
    against the nodes per pair: slope = cycles per node (128 points of a
    warp), intercept = the per-(warp, element) work around the node loop."""
    import torch
    import paper_1606_03743_gb300 as bem

    dev = torch.device("cuda", 0)
    mesh = synth.coax_mesh(seed=2)
    p_d = torch.from_numpy(synth.coax_points(seed=2, n=a.points)).to(dev)
    phi = torch.empty(a.points, dtype=torch.float64, device=dev)
    E = torch.empty((a.points, 3), dtype=torch.float64, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    near = bem.bem_default_limits()[:, 0]
    rows = []
    for band in range(1, 6):  # band b: the rule with 33, 19|17, 12, 7, 4 nodes
        lim = np.zeros((2, 5))
        for t in range(2):
            for k in range(5):
                lim[t, k] = near[t] * (1.0 + 1e-9 * k) if k < band else 1e30 * (k + 1)
        m = bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                     torch.from_numpy(mesh.sigma).to(dev), precision=bem.MIXED, limits=lim)
        m.set_stats(True)
        bem.bem_eval(m.handle, p_d, phi, E)
        st = m.last_stats()
        m.set_stats(False)
        m.set_timing(True)
        far = []
        for _ in range(3):
            bem.bem_eval(m.handle, p_d, phi, E)
            torch.cuda.synchronize()
            far.append(float(m.last_times()[1]))
        m.close()
        wel = float(st[13] + st[14])  # (warp, element) pairs: one band, per-point bands
        nodes = float(st[15]) / (32 * 4) / wel  # node evaluations per (warp, element) pair
        cyc = statistics.median(far) * 1e-3 * 2070e6 * sms * 4 / wel  # sub-partition cycles per pair
        rows.append({"band": band, "far_ms": statistics.median(far), "warp_element_pairs": wel,
                     "nodes_per_pair": nodes, "cycles_per_pair": cyc})
    x = np.array([r["nodes_per_pair"] for r in rows])
    y = np.array([r["cycles_per_pair"] for r in rows])
    slope, icpt = np.polyfit(x, y, 1)
    print(json.dumps({"mode": "band_fit", "workload": WORKLOAD, "n_points": a.points, "rules": rows,
                      "fit": {"cycles_per_node": float(slope), "cycles_per_warp_element": float(icpt),
                              "note": "cycles of one SM sub-partition at 2070 MHz per (warp, element) pair of "
                                      "128 points; least squares over the five rules"}}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
