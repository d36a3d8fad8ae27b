#!/usr/bin/env python3
"""Benchmark of the exhaustive specular-polynomial solve on one GB300.

One step is one pass of the whole hot path over the refraction-caustics
workload: the bounding-cone cull over every (receiver, triangle) pair of a
64x64-cell heightfield (8,192 triangles, IOR 1.5) under a point light at
(0, 0, 2) seen by a 256x256 receiver grid on z = -1 (536,870,912 pairs),
then the mixed-precision solve of every surviving pair (FP64 construction,
FP32 Laplace expansion and isolation, FP64 polish and path checks), then
the read-back of the path count.  Inputs are synthetic and seeded.

metric: candidate solves/s -- (receiver, triangle) tuples whose complete
admissible path set is produced per second (all pairs of the workload; the
cull proves most of them empty).  Also reported: survivors solved per
second and admissible paths per second.

--impl reference times the FP64 CPU oracle on the same metric: each step
solves every pair of a seeded sample of receivers on all host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate solves/s & admissible paths/s on 1 GB300: learned+FP32 vs plain FP64"
UNIT = "candidates/s"
# Algorithmic FP64 flops per solved candidate in the isolation kernel:
# construction of a, b (Sec. 3.5) and the FP64 Bezout entries (Eq. eq_bezout);
# counted from the implementation.  FP32: Laplace expansion.
FP64_FLOPS = {"T": 1310, "R": 650}
FP32_LAPLACE_FLOPS = {"T": 2744, "R": 400}
# Nominal scalar peaks derived from unit counts and clocks:
# FP32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz; FP64: 1.25 TFLOP/s.
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
NOMINAL_FP64_TFLOPS = 1.25
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) per launch of the isolation kernel from the last
# ncu capture (profiles/kernels_refract_64x64_r256_mixed.md).  Reported only
# while the kernel's sources hash to the value the capture was taken on.
KERNEL_SOURCES = ["common.cuh", "polys.cuh", "laplace_gen.cuh", "k1_sys.cuh", "k1_iso.cuh", "k1_iso_f32.cu"]
TRAFFIC = {"sources_sha256": None, "bytes_per_launch": None}


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2405_13409_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["mine", "reference"], default="mine")
    p.add_argument("--workload", choices=["refract", "reflect", "glints"], default="refract")
    p.add_argument("--precision", choices=["mixed", "plain"], default="mixed")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--ref-receivers", type=int, default=16)
    return p.parse_args()


def workload(name):
    """(scene, chain mode, scattering kind, description, camera or None)."""
    from paper_2405_13409_gb300 import binding, scenes
    if name == "glints":
        s = scenes.glint_scene()
        return s, binding.CHAINS_FOOTPRINT, "R", (
            "glints: 1024x1024-cell heightfield (2,097,152 triangles, 64 sinusoids of wavelength 2-20 cells), "
            "pinhole 512x512 at (0,-2,1.5), light (1,1,2), reflection, pixel-footprint candidates"), \
            s.meta["camera"].as_array()
    if name == "refract":
        s = scenes.refract_scene()
        return s, binding.CHAINS_CONE, "T", (
            "refraction caustics: 64x64-cell sinusoid heightfield (8,192 triangles, amplitude 0.08), "
            "eta 1 -> 1.5, light (0,0,2), 256x256 receivers on z=-1, bounding-cone cull"), None
    s = scenes.reflect_scene()
    return s, binding.CHAINS_ALL, "R", (
        "reflection: 16x16-cell sinusoid heightfield (512 triangles, amplitude 0.05), light (0.3,-0.2,2), "
        "32x32 receivers on z=1, exhaustive"), None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"spoly_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
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
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.remove(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def run_oracle_sample(s, n_recv, seed):
    import oracle
    from paper_2405_13409_gb300 import scenes
    rng = np.random.default_rng(seed)
    qs = np.sort(rng.choice(s.n_queries, n_recv, replace=False)).astype(np.int32)
    chains = np.stack([np.repeat(qs, s.n_tris), np.tile(np.arange(s.n_tris, dtype=np.int32), n_recv),
                       -np.ones(n_recv * s.n_tris, np.int32)], -1).astype(np.int32)
    del scenes
    t0 = time.perf_counter()
    paths, cnt = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, chains)
    return chains.shape[0], time.perf_counter() - t0, paths.size


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    s, _, kind, desc, _cam = workload(args.workload)
    cores = os.cpu_count()
    for i in range(args.warmup):
        run_oracle_sample(s, args.ref_receivers, 1000 + i)
    tot_c, tot_t, tot_p = 0, 0.0, 0
    for i in range(args.steps):
        c, t, p = run_oracle_sample(s, args.ref_receivers, 2000 + i)
        tot_c += c
        tot_t += t
        tot_p += p
    value = tot_c / tot_t
    sample = f"all {s.n_tris} triangles x {args.ref_receivers} seeded receivers per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "precision": "plain FP64 CPU oracle"},
            "paths_per_s": tot_p / tot_t,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2405_13409_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    __graft_entry__.build_library()
    dev = torch.device(f"cuda:{local}")
    stream = torch.cuda.current_stream()
    ctx = binding.Context(local, stream.cuda_stream)
    s, mode, kind, desc, camera = workload(args.workload)
    precision = binding.MIXED if args.precision == "mixed" else binding.PLAIN_FP64
    host = [np.ascontiguousarray(a) for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
    d = [torch.from_numpy(a).to(dev) for a in host]
    mesh = ctx.mesh(d[0])
    q = ctx.queries(*d[1:])
    pairs = s.n_queries * s.n_tris

    peak32 = ctx.spoly_measure_peak(binding.PEAK_FP32_FMA)
    peak64 = ctx.spoly_measure_peak(binding.PEAK_FP64_FMA)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    state = {"chains": None, "sol": None}

    def step(m, qq):
        state["chains"] = ctx.spoly_build_chains(m, qq, mode, margin=1e-3, reuse=state["chains"], camera=camera)
        state["sol"] = ctx.spoly_solve(m, qq, state["chains"], precision=precision,
                                       flags=binding.SOLVE_TIMING, reuse=state["sol"], camera=camera)

    for _ in range(args.warmup):
        step(mesh, q)
    torch.cuda.synchronize()
    n_chains = ctx.spoly_chains_count(state["chains"])
    stats = ctx.spoly_stats(state["sol"])
    if mode == binding.CHAINS_FOOTPRINT:
        pairs = n_chains  # the footprint defines the candidate set of this workload

    # timed region: device-resident inputs, L2 flushed between steps
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms, iso_ms, pol_ms = [], [], []
    n_paths = 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(mesh, q)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        i_ms, p_ms = ctx.spoly_phase_ms(state["sol"])
        iso_ms.append(i_ms)
        pol_ms.append(p_ms)
        n_paths = ctx.spoly_stats(state["sol"])["admissible"]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    t = torch.tensor([total_ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = world * pairs * args.steps / (total_ms * 1e-3)

    # end to end: host (pinned) inputs through the C ABI, H2D and D2H inside the timed region
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(a).pin_memory() for a in host]
        hmesh = ctx.mesh(pinned[0])
        hq = ctx.queries(*pinned[1:])
        out = torch.empty(max(1, 2 * n_paths + 1024) * binding.PATH_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        for _ in range(2):
            step(hmesh, hq)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e_ms = []
        d2h = 0
        for _ in range(args.steps):
            flush.fill_(1.0)
            t0 = time.perf_counter()
            step(hmesh, hq)
            cap = out.numel() // binding.PATH_DTYPE.itemsize
            n = ctx.spoly_paths_into(state["sol"], out, cap)
            torch.cuda.synchronize()
            e_ms.append(1e3 * (time.perf_counter() - t0))
            d2h = min(n, cap) * binding.PATH_DTYPE.itemsize + 8
        te = torch.tensor([sum(e_ms)], device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        h2d = 2 * sum(a.nbytes for a in host)
        e2e = {"value": world * pairs * args.steps / (float(te.item()) * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    iso = statistics.mean(iso_ms)
    achieved64 = FP64_FLOPS[kind] * n_chains / (iso * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if precision == binding.MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": desc, "precision": args.precision, "pairs_per_step": pairs,
                   "l2": "flushed between steps (512 MiB write)", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "solved_per_s": world * n_chains * args.steps / (total_ms * 1e-3),
        "paths_per_s": world * n_paths * args.steps / (total_ms * 1e-3),
        "survivors_per_step": n_chains, "paths_per_step": n_paths, "counters": stats,
        "phase_ms": {"step": total_ms / args.steps, "isolation": iso, "polish": statistics.mean(pol_ms),
                     "chains": total_ms / args.steps - iso - statistics.mean(pol_ms)},
        "roofline": {"bound": "alu", "pipe": "fp64", "kernel": "k1_isolate_kernel<float>",
                     "achieved": achieved64, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved64 / NOMINAL_FP64_TFLOPS,
                     "traffic": TRAFFIC["bytes_per_launch"]
                     if TRAFFIC["sources_sha256"] == kernel_sources_sha256() else None,
                     "peak_measured_fp64": peak64, "peak_measured_fp32": peak32,
                     "frac_of_measured": achieved64 / peak64 if peak64 else None,
                     "fp32_laplace_tflops": FP32_LAPLACE_FLOPS[kind] * n_chains / (iso * 1e-3) / 1e12},
        "gpu_launches": 7 * args.steps,
        "clocks": clk,
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        n_recv = 64 if kind == "T" else 256
        c, tcpu, _ = run_oracle_sample(s, min(n_recv, s.n_queries), 7)
        line["cpu_baseline"] = {"value": c / tcpu, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"all {s.n_tris} triangles x {min(n_recv, s.n_queries)} seeded receivers"}
    print(json.dumps(line))
    ctx.spoly_solution_free(state["sol"])
    ctx.spoly_chains_free(state["chains"])
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
