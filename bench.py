#!/usr/bin/env python3
"""Benchmark of the exhaustive specular-polynomial solve on one GB300.

Default workload (glints): a 1024x1024-cell heightfield (2,097,152
triangles, height = sum of 64 random-phase sinusoids of wavelength 2-20
cells) seen by a 512x512 pinhole camera at (0, -2, 1.5) under a point light
at (1, 1, 2).  One step is one pass of the whole hot path: the pixel-
footprint candidate build over a uniform grid, the learned gate (features +
BF16 tensor-core MLP + compaction), the mixed-precision solve of the
surviving candidates (FP64 construction, FP32 Laplace expansion and
isolation, FP64 polish and path checks), and the read-back of the path
count.  Every pixel shares its endpoints (the pinhole and the light), so a
triangle's solutions do not depend on the pixel: the footprint's distinct
triangles are gated and solved once each, and every path goes to the pixel
its vertex projects into, which yields each (pixel, triangle) candidate's
complete path set.  The same run times the plain
FP64 path (no gate, every step in FP64) on the same candidates and reports
the recall of the gated solve against it.  The gate is trained before the
timed region on the glint generator's training seeds (its own kernels) and
calibrated on a validation seed.  Inputs are synthetic and seeded.

metric: candidate solves/s -- (pixel, triangle) candidates of the footprint
whose complete admissible path set is produced per second (the gate proves
most of them empty).  Also reported: admissible paths per second.

--workload refract / reflect time the 1-bounce caustic and reflection
workloads (bounding-cone cull / exhaustive, no gate); --workload slab the
2-bounce refraction slab; --workload corridor the 2-bounce reflection
corridor between two heightfield mirrors (--intervals sets the v1 sample
intervals of 2-bounce chains); --workload batched the batched mixed workload
(independent queries of 1 or 2 bounces with explicit candidate lists:
per-chain cone test, learned gate on the 1-bounce chains, persistent
isolation with an autotuned launch shape, 2-bounce pipeline).
--impl reference times the FP64 CPU oracle on the same metric.
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
# counted from the implementation's arithmetic.  FP32: Laplace expansion.
FP64_FLOPS = {"T": 1310, "R": 650}
FP32_LAPLACE_FLOPS = {"T": 2744, "R": 400}
# Nominal scalar peaks derived from unit counts and clocks:
# FP32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz; FP64: 1.25 TFLOP/s.
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
NOMINAL_FP64_TFLOPS = 1.25
L2_FLUSH_BYTES = 512 << 20
# Gate: algorithmic flops per candidate (24x64 + 64x64 + 64x64 + 64 MACs)
# and the measured dense BF16 peak of this GPU type (MEASURED_PEAKS.json).
GATE_FLOPS = 2 * (24 * 64 + 64 * 64 + 64 * 64 + 64)
BF16_PEAK_TFLOPS = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] \
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
# Kernel launches per step, counted from the committed ncu launch list of
# each workload.
LAUNCHES_PER_STEP = {("refract", False): 7, ("reflect", False): 4, ("glints", False): 15, ("glints", True): 16}
# 2-bounce solve: systems count + fill, then per batch of <= 16,384 systems the
# build, six FP32 sign classes, five FP64 re-sampling chunk classes and five
# re-sampling scan classes, five polish classes, the active-chain list and the
# path kernel.
TT_FIXED, TT_PER_BATCH, TT_BATCH = 2, 24, 16384
K2_KINDS = ("TT", "RR")  # 2-bounce workloads (slab, corridor)


def launches_per_step(workload, use_gate, stats):
    """Kernel launches of the library in one step (counted from the
    committed ncu launch lists of each workload)."""
    if workload in ("slab", "corridor", "batched"):
        batches = -(-int(stats.get("k2_systems", 0)) // TT_BATCH)
        tt = TT_FIXED + TT_PER_BATCH * batches
        if workload in ("slab", "corridor"):
            return 5 + 1 + tt  # cone cull (flag, shared check, forward boxes, pairs, chains), partition
        # explicit validation + cone test, gate, then the graph: partition, persistent isolation, side
        # solve, finish, and the device-driven 2-bounce pass (its 31 launches plus 3 of its scan),
        # counted from the committed launch list
        return 2 + (1 if use_gate else 0) + 4 + 31
    return LAUNCHES_PER_STEP.get((workload, use_gate), 7)
# DRAM bytes (read + write) per launch from an ncu capture of the kernel on
# the workload named, reported only while the kernel's sources hash to the
# value the capture was taken on.
TRAFFIC = {
    "gate_kernel": {"workload": "glints", "sources": ["gate.cu", "gate.cuh", "mlp.cuh", "common.cuh", "umma.cuh"],
                    "sources_sha256": "bdca7565ecb6cae7efaf372bbcd4f2309812293115c143d5b47ea000b29ffd05",
                    "bytes_per_launch": 288503808 + 3689984},
    "k1_isolate_kernel": {"workload": "refract",
                          "sources": ["common.cuh", "polys.cuh", "laplace_gen.cuh", "k1_sys.cuh", "k1_iso.cuh",
                                      "k1_iso_f32.cu"], "sources_sha256": None, "bytes_per_launch": None},
}


def kernel_sources_sha256(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2405_13409_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def traffic(kernel, workload):
    t = TRAFFIC[kernel]
    if t["workload"] != workload or t["sources_sha256"] is None:
        return None
    return t["bytes_per_launch"] if t["sources_sha256"] == kernel_sources_sha256(t["sources"]) else None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["mine", "reference"], default="mine")
    p.add_argument("--workload", choices=["glints", "refract", "reflect", "slab", "corridor", "batched"],
                   default="glints")
    p.add_argument("--corridor-receivers", type=int, default=16,
                   help="corridor: receiver grid side (16: 16x16 receivers)")
    p.add_argument("--intervals", type=int, default=0,
                   help="2-bounce chains: v1 sample intervals (0: 4096, the 2^12 + 1 samples; the paper's "
                        "2-bounce GPU timing uses 100)")
    p.add_argument("--batch-queries", type=int, default=4096, help="batched: number of queries")
    p.add_argument("--slab-receivers", type=int, default=64,
                   help="slab: receiver grid side (64: the full 64x64 grid)")
    p.add_argument("--precision", choices=["mixed", "plain"], default="mixed")
    p.add_argument("--no-gate", action="store_true", help="glints: solve every candidate (no learned gate)")
    p.add_argument("--no-plain", action="store_true", help="glints: skip the plain FP64 comparison")
    p.add_argument("--plain-steps", type=int, default=5)
    p.add_argument("--train-seeds", type=int, default=2)
    p.add_argument("--train-steps", type=int, default=3000)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--gate-file", default="",
                   help="glints: load the trained gate (and its threshold, PATH.json) from PATH if it exists, "
                        "else train it and save it there")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--ref-units", type=int, default=0,
                   help="reference arm sample per step: receivers (refract/reflect) or pixels (glints)")
    return p.parse_args()


def workload(name, slab_receivers=64, batch_queries=4096, corridor_receivers=16):
    """(scene, chain mode, scattering kind, description, camera or None)."""
    from paper_2405_13409_gb300 import binding, scenes
    if name == "corridor":
        s = scenes.corridor_scene(n_recv=corridor_receivers)
        return s, binding.CHAINS_CONE, "RR", (
            f"2-bounce reflection corridor: 16x16-cell floor (z=0, normals up) and ceiling (z=1, normals down) "
            f"heightfield mirrors (512 triangles each, amplitude 0.05), light (-0.6,0.1,0.5), "
            f"{corridor_receivers}x{corridor_receivers} receivers on z=0.5 over [-0.8,0.8]^2, forward+backward "
            f"cone cull"), None
    if name == "batched":
        s = scenes.batched_scene(n_queries=batch_queries)
        return s, binding.CHAINS_EXPLICIT_CONE, "mixed", (
            f"batched mixed workload: {batch_queries} queries, bounce count uniform in {{1,2}}, candidate counts "
            f"log-uniform in 1e2..1e5 ({s.chains.shape[0]:,} explicit chains), per-query geometry from the "
            f"refraction generator (1 bounce) or the 16x16-cell slab (2 bounces); per-chain cone test, learned "
            f"gate on 1-bounce chains, persistent isolation with an autotuned launch shape"), None
    if name == "slab":
        s = scenes.slab_scene(n_recv=slab_receivers)
        return s, binding.CHAINS_CONE, "TT", (
            f"2-bounce refraction slab: 16x16-cell top (z=0) and bottom (z=-0.3) heightfields (512 triangles "
            f"each, amplitude 0.05), eta 1 -> 1.5 -> 1, light (0.2,0.1,2), {slab_receivers}x{slab_receivers} "
            f"receivers on z=-1, forward+backward cone cull, 4097 v1 samples"), None
    if name == "glints":
        s = scenes.glint_scene()
        return s, binding.CHAINS_FOOTPRINT_UNIQUE, "R", (
            "glints: 1024x1024-cell heightfield (2,097,152 triangles, 64 sinusoids of wavelength 2-20 cells), "
            "pinhole 512x512 at (0,-2,1.5), light (1,1,2), reflection, pixel-footprint candidates; the "
            "footprint's distinct triangles gated and solved once, each path assigned to its pixel"), \
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
    """SM clock and throttle-reason samples taken DURING the timed region by a
    thread reading NVML every 5 ms (through ctypes; read-only queries), with
    nvidia-smi at 100 ms as the fallback when NVML cannot be loaded."""

    # NVML clock-event reason bits
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown", 0x4: "sw_power_cap"}

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.thread = None
        self.proc = None
        self.stop_flag = False
        self.nvml = None
        try:
            import ctypes
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(h)) == 0:
                    self.nvml, self.h, self.ct = lib, h, ctypes
        except OSError:
            self.nvml = None

    def _sample_nvml(self):
        ct, lib = self.ct, self.nvml
        clk, mx, rs = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_flag:
            if (lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(clk)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ct.byref(mx)) == 0 and
                    get_reasons(self.h, ct.byref(rs)) == 0):
                self.rows.append((float(clk.value), float(mx.value), int(rs.value)))
            time.sleep(0.005)

    def start(self):
        import threading
        if self.nvml is not None:
            self.thread = threading.Thread(target=self._sample_nvml, daemon=True)
            self.thread.start()
            return
        self.path = os.path.join("/tmp", f"spoly_clocks_{os.getpid()}.csv")
        fields = ("index,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                  "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                  "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={fields}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag = True
            self.thread.join()
            rows = self.rows
            src = "nvml 5 ms"
        elif self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            rows = []
            bits = [0x8, 0x40, 0x20, 0x4]
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                try:
                    r = sum(b for b, v in zip(bits, f[3:7]) if v.lower() == "active")
                    rows.append((float(f[1]), float(f[2]), r))
                except (ValueError, IndexError):
                    continue
            os.remove(self.path)
            src = "nvidia-smi 100 ms"
        else:
            return None
        if not rows:
            return None
        reasons = sorted({n for _, _, r in rows for b, n in self.REASONS.items() if r & b})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "source": src}


def footprint_sample(s, camera, n_pixels, seed):
    """Host (numpy) footprint candidates of seeded 16x16-pixel blocks (about
    n_pixels pixels in all), for the CPU legs: the triangles whose xy
    bounding box meets the pixel's footprint box (its four corner rays
    between the mesh's z bounds)."""
    w, h = int(camera[14]), int(camera[15])
    side = 16
    n_blocks = max(1, n_pixels // (side * side))
    rng = np.random.default_rng(seed)
    T = s.tri
    xs, ys, zs = T[[0, 3, 6]], T[[1, 4, 7]], T[[2, 5, 8]]
    txl, txh, tyl, tyh = xs.min(0), xs.max(0), ys.min(0), ys.max(0)
    zlo, zhi = zs.min(), zs.max()
    o, f, r, u = camera[0:3], camera[3:6], camera[6:9], camera[9:12]
    th, asp = camera[12], camera[13]

    def box(ixa, ixb, iya, iyb):
        pts = []
        for ix in (ixa, ixb):
            for iy in (iya, iyb):
                d = f + (-1 + 2 * ix / w) * th * asp * r + (1 - 2 * iy / h) * th * u
                for z in (zlo, zhi):
                    pts.append(o + (z - o[2]) / d[2] * d)
        pts = np.array(pts)
        return pts[:, 0].min(), pts[:, 0].max(), pts[:, 1].min(), pts[:, 1].max()

    rows = []
    for _ in range(n_blocks):
        x0, y0 = int(rng.integers(0, w - side + 1)), int(rng.integers(0, h - side + 1))
        bx = box(x0, x0 + side, y0, y0 + side)
        near = np.where(~((txh < bx[0]) | (txl > bx[1]) | (tyh < bx[2]) | (tyl > bx[3])))[0]
        for iy in range(y0, y0 + side):
            for ix in range(x0, x0 + side):
                b = box(ix, ix + 1, iy, iy + 1)
                t = near[~((txh[near] < b[0]) | (txl[near] > b[1]) | (tyh[near] < b[2]) | (tyl[near] > b[3]))]
                rows.append(np.stack([np.full(t.size, iy * w + ix), t, -np.ones(t.size, np.int64)], -1))
    return np.concatenate(rows).astype(np.int32), n_blocks


def run_oracle_sample(s, camera, n_units, seed, kind="R", n_intervals=0):
    """One CPU-oracle step: all triangles x n_units seeded receivers, the
    footprint candidates of a block of about n_units pixels (glints), or
    (slab) n_units (receiver, top, bottom) tuples pairing a seeded top
    triangle with the bottom triangle of the same cell."""
    import oracle
    if kind == "mixed":
        # a seeded sample of the explicit list per bounce count; the rate is
        # weighted by the list's own 1/2-bounce mix
        from oracle import tt
        rng = np.random.default_rng(seed)
        two = s.chains[:, 2] >= 0
        i1 = rng.choice(np.where(~two)[0], min(n_units * 256, int((~two).sum())), replace=False)
        i2 = rng.choice(np.where(two)[0], min(n_units, int(two.sum())), replace=False)
        t0 = time.perf_counter()
        p1, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, s.chains[np.sort(i1)])
        t1 = time.perf_counter()
        p2, _ = tt.solve(s.tri, s.x_first, s.x_last, s.eta, s.chains[np.sort(i2)], tt.fit_sqrt_pieces())
        t2 = time.perf_counter()
        n1, n2 = int((~two).sum()), int(two.sum())
        per_chain = (n1 * (t1 - t0) / max(1, i1.size) + n2 * (t2 - t1) / max(1, i2.size)) / (n1 + n2)
        return 1, per_chain, 0, (f"{i1.size} seeded 1-bounce and {i2.size} seeded 2-bounce chains of the explicit list; "
                                 f"time per chain weighted by the list's {n1:,}/{n2:,} mix")
    if kind == "RR":
        from oracle import rr
        rng = np.random.default_rng(seed)
        half = s.n_tris // 2
        qs = rng.integers(0, s.n_queries, n_units)
        t1 = rng.integers(0, half, n_units)
        chains = np.stack([qs, t1, t1 + half], -1).astype(np.int32)
        t0 = time.perf_counter()
        paths = rr.solve(s.tri, s.x_first, s.x_last, chains, n_intervals or rr.N_INTERVALS)
        return chains.shape[0], time.perf_counter() - t0, paths.size, \
            f"{n_units} seeded (receiver, floor triangle, ceiling triangle of the same cell) tuples"
    if kind == "TT":
        from oracle import tt
        rng = np.random.default_rng(seed)
        half = s.n_tris // 2
        qs = rng.integers(0, s.n_queries, n_units)
        t1 = rng.integers(0, half, n_units)
        chains = np.stack([qs, t1, t1 + half], -1).astype(np.int32)
        table = tt.fit_sqrt_pieces()
        t0 = time.perf_counter()
        paths, _ = tt.solve(s.tri, s.x_first, s.x_last, s.eta, chains, table)
        return chains.shape[0], time.perf_counter() - t0, paths.size, \
            f"{n_units} seeded (receiver, top triangle, bottom triangle of the same cell) tuples"
    if camera is not None:
        chains, nb = footprint_sample(s, camera, n_units, seed)
        desc = f"footprint candidates of {nb} 16x16-pixel blocks at seeded positions"
    else:
        rng = np.random.default_rng(seed)
        qs = np.sort(rng.choice(s.n_queries, n_units, replace=False)).astype(np.int32)
        chains = np.stack([np.repeat(qs, s.n_tris), np.tile(np.arange(s.n_tris, dtype=np.int32), n_units),
                           -np.ones(n_units * s.n_tris, np.int32)], -1).astype(np.int32)
        desc = f"all {s.n_tris} triangles x {n_units} seeded receivers"
    t0 = time.perf_counter()
    paths, cnt = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, chains)
    return chains.shape[0], time.perf_counter() - t0, paths.size, desc


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    s, _, kind, desc, cam = workload(args.workload, args.slab_receivers, args.batch_queries, args.corridor_receivers)
    units = args.ref_units or (16384 if cam is not None else (8 if kind in K2_KINDS + ("mixed",) else 16))
    cores = os.cpu_count()
    for i in range(args.warmup):
        run_oracle_sample(s, cam, units, 1000 + i, kind, args.intervals)
    tot_c, tot_t, tot_p, sample = 0, 0.0, 0, ""
    for i in range(args.steps):
        c, t, p, sample = run_oracle_sample(s, cam, units, 2000 + i, kind, args.intervals)
        tot_c += c
        tot_t += t
        tot_p += p
    value = tot_c / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "precision": "plain FP64 CPU oracle, no gate"},
            "paths_per_s": tot_p / tot_t,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def job_rate(local_ms, units_per_rank, steps, world, device="cpu"):
    """Replicas (one per rank, no data exchange): the job's time is the
    slowest rank's, and the rate counts the units of every rank.  Returns
    (max over ranks of local_ms, units per second of the whole job)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * units_per_rank * steps / (ms * 1e-3)


def match_paths(got, ref, tol=1e-5):
    """Paths of `ref` with a path of `got` on the same (pixel, triangle)
    within tol in (u, v); returns (matched, max |delta(u, v)| over matches)."""
    from collections import defaultdict
    g = defaultdict(list)
    for qq, t, uv in zip(got["query"].tolist(), got["tri"][:, 0].tolist(), got["uv"][:, :2]):
        g[(qq, t)].append(uv)
    matched, worst = 0, 0.0
    for qq, t, uv in zip(ref["query"].tolist(), ref["tri"][:, 0].tolist(), ref["uv"][:, :2]):
        ds = [float(np.max(np.abs(uv - x))) for x in g.get((qq, t), [])]
        if ds and min(ds) <= tol:
            matched += 1
            worst = max(worst, min(ds))
    return matched, worst


class Pipeline:
    """One step of the hot path through the C ABI: candidate build, optional
    gate, solve.  Handles are reused across steps (grow-only buffers)."""

    def __init__(self, ctx, mode, precision, camera, mlp=None, tau=0.0, ranges=None, explicit=None, flags=0,
                 n_intervals=0):
        self.ctx, self.mode, self.precision, self.camera = ctx, mode, precision, camera
        self.n_intervals = n_intervals  # 2-bounce v1 sample intervals (0: the library's 4096)
        self.mlp, self.tau = mlp, tau
        self.ranges = ranges  # 2-bounce cone: ((first range), (second range))
        self.explicit = explicit  # explicit chain list (device tensor [n, 3])
        self.flags = flags
        self.chains = self.gated = self.sol = None
        self.ev = None

    def step(self, mesh, q, stream=None, torch=None):
        from paper_2405_13409_gb300 import binding
        ev = None
        if torch is not None:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
        if self.explicit is not None:
            self.chains = self.ctx.spoly_build_chains(mesh, q, self.mode, margin=1e-3, reuse=self.chains,
                                                      explicit=self.explicit)
        elif self.ranges:
            self.chains = self.ctx.spoly_build_chains(mesh, q, self.mode, margin=1e-3, reuse=self.chains,
                                                      tri_range=self.ranges[0], second_range=self.ranges[1])
        else:
            self.chains = self.ctx.spoly_build_chains(mesh, q, self.mode, margin=1e-3, reuse=self.chains,
                                                      camera=self.camera)
        if ev:
            ev[1].record(stream)
        solve_on = self.chains
        if self.mlp is not None:
            self.gated = self.ctx.spoly_gate(self.mlp, mesh, q, self.chains, self.tau, reuse=self.gated)
            solve_on = self.gated
        if ev:
            ev[2].record(stream)
        self.sol = self.ctx.spoly_solve(mesh, q, solve_on, precision=self.precision,
                                        flags=binding.SOLVE_TIMING | self.flags, reuse=self.sol, camera=self.camera,
                                        n_intervals=self.n_intervals)
        self.ev = ev

    def phase_ms(self):
        """(candidate build, gate) milliseconds of the last timed step."""
        self.ev[2].synchronize()
        return self.ev[0].elapsed_time(self.ev[1]), self.ev[1].elapsed_time(self.ev[2])

    def free(self):
        for h in (self.sol,):
            if h is not None:
                self.ctx.spoly_solution_free(h)
        for h in (self.chains, self.gated):
            if h is not None:
                self.ctx.spoly_chains_free(h)


def timed_steps(pipe, mesh, q, steps, flush, stream, torch):
    """steps timed with CUDA events on the launching stream, L2 flushed
    before each; returns per-step dicts."""
    out = []
    for _ in range(steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pipe.step(mesh, q, stream, torch)
        b.record(stream)
        b.synchronize()
        c_ms, g_ms = pipe.phase_ms()
        i_ms, p_ms, tt_ms, sign_ms = pipe.ctx.spoly_phase_ms(pipe.sol)
        out.append({"step": a.elapsed_time(b), "chains": c_ms, "gate": g_ms, "isolation": i_ms, "polish": p_ms,
                    "k2": tt_ms, "k2_sign": sign_ms,
                    "paths": pipe.ctx.spoly_stats(pipe.sol)["admissible"]})
    return out


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
    # a non-default stream, current for torch and the library (graph capture needs one)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    ctx = binding.Context(local, stream.cuda_stream)
    s, mode, kind, desc, camera = workload(args.workload, args.slab_receivers, args.batch_queries, args.corridor_receivers)
    precision = binding.MIXED if args.precision == "mixed" else binding.PLAIN_FP64
    batched = kind == "mixed"
    host = [np.ascontiguousarray(a) for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
    if batched:
        host.append(np.ascontiguousarray(s.chains))
    d = [torch.from_numpy(a).to(dev) for a in host]
    mesh = ctx.mesh(d[0])
    q = ctx.queries(*d[1:6])
    explicit = d[6] if batched else None

    peak32 = ctx.spoly_measure_peak(binding.PEAK_FP32_FMA)
    peak64 = ctx.spoly_measure_peak(binding.PEAK_FP64_FMA)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # learned gate: trained and calibrated before the timed region
    use_gate = (camera is not None or batched) and precision == binding.MIXED and not args.no_gate
    mlp, tau, gate_info = None, 0.0, None
    if use_gate and args.gate_file and os.path.exists(args.gate_file) and os.path.exists(args.gate_file + ".json"):
        mlp = ctx.spoly_mlp_load(args.gate_file)
        gate_info = json.load(open(args.gate_file + ".json"))
        gate_info["loaded_from"] = args.gate_file
        tau = gate_info["tau_logit"]
    elif use_gate:
        from paper_2405_13409_gb300 import gate_train, scenes
        t0 = time.perf_counter()
        if batched:
            # the gate covers the 1-bounce (refraction) chains, whose meshes
            # have 64 to 224 cells a side: training and validation scenes
            # span that range, and the threshold keeps a wider margin
            cells = [64 + (160 * i) // max(1, args.train_seeds - 1) for i in range(args.train_seeds)]
            train = [scenes.refract_scene(seed=1000 + i, n_cells=c, n_recv=128) for i, c in enumerate(cells)]
            val = [scenes.refract_scene(seed=2000 + i, n_cells=c, n_recv=128) for i, c in enumerate((64, 144, 224))]
            gmode, margin = binding.CHAINS_CONE, 2.0
        else:
            train = [scenes.glint_scene(seed=1000 + i) for i in range(args.train_seeds)]
            val = [scenes.glint_scene(seed=2000)]
            gmode, margin = mode, 1.0
        gen_s = time.perf_counter() - t0
        mlp, tau, gate_info = gate_train.train_gate(ctx, torch, train, val, gmode, camera, margin=margin,
                                                    steps=args.train_steps, seed=args.seed)
        gate_info["scene_generation_s"] = gen_s
        gate_info["train_seeds"] = [1000 + i for i in range(args.train_seeds)]
        gate_info["val_seeds"] = [2000 + i for i in range(len(val))]
        del train, val
        torch.cuda.empty_cache()
        if args.gate_file:
            ctx.spoly_mlp_save(mlp, args.gate_file)
            json.dump(gate_info, open(args.gate_file + ".json", "w"))

    ranges = ((0, s.n_tris // 2), (s.n_tris // 2, s.n_tris)) if kind in K2_KINDS else None
    tune = None
    if batched:
        # launch shape of the persistent isolation, tuned on the 1-bounce chains
        one = torch.from_numpy(np.ascontiguousarray(s.chains[s.chains[:, 2] < 0])).to(dev)
        ch1 = ctx.spoly_build_chains(mesh, q, mode, margin=1e-3, explicit=one)
        best, table = ctx.spoly_autotune(mesh, q, ch1, precision)
        tune = {"block": best[0], "blocks_per_sm": best[1], "chunk": best[2], "ms": best[3], "shapes": len(table)}
        ctx.spoly_chains_free(ch1)
        del one
    footprint = mode in (binding.CHAINS_FOOTPRINT, binding.CHAINS_FOOTPRINT_UNIQUE)
    assign = binding.SOLVE_PIXEL_ASSIGN if mode == binding.CHAINS_FOOTPRINT_UNIQUE else 0
    # the batched solve (both bounce depths) is captured once into a CUDA graph
    # and replayed every step
    pipe = Pipeline(ctx, mode, precision, camera, mlp, tau, ranges, explicit,
                    ((binding.SOLVE_PERSISTENT | binding.SOLVE_GRAPH) if batched else 0) | assign,
                    n_intervals=args.intervals)
    for _ in range(args.warmup):
        pipe.step(mesh, q)
    torch.cuda.synchronize()
    n_cand = ctx.spoly_chains_count(pipe.chains)
    n_solved = ctx.spoly_chains_count(pipe.gated) if use_gate else n_cand
    stats = ctx.spoly_stats(pipe.sol)
    if footprint:
        pairs = ctx.spoly_chains_footprint_pairs(pipe.chains)  # (pixel, triangle) candidates of the step
    elif batched:
        pairs = int(s.chains.shape[0])  # every explicit chain of the step
    elif kind in K2_KINDS:
        pairs = s.n_queries * (s.n_tris // 2) ** 2  # every (receiver, top, bottom) tuple the cull stands for
    else:
        pairs = s.n_queries * s.n_tris

    # timed region: device-resident inputs, L2 flushed between steps
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    rec = timed_steps(pipe, mesh, q, args.steps, flush, stream, torch)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms, value = job_rate(sum(r["step"] for r in rec), pairs, args.steps, world, dev)
    n_paths = rec[-1]["paths"]
    got_paths = ctx.spoly_paths(pipe.sol)

    # the path phase's last steps on the final step's paths (outside the
    # metric's step): visibility, contributions and the glint image
    render = None
    if camera is not None and n_paths > 0:
        ra, rb, rc = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        img = torch.zeros(s.n_queries, dtype=torch.float64, device=dev)
        ra.record(stream)
        n_vis = ctx.spoly_visibility(mesh, q, pipe.sol)
        rb.record(stream)
        ctx.spoly_contributions(mesh, q, pipe.sol, 1.0, image=img)
        rc.record(stream)
        rc.synchronize()
        render = {"visible_paths": n_vis, "occluded_paths": n_paths - n_vis, "visibility_ms": ra.elapsed_time(rb),
                  "contributions_ms": rb.elapsed_time(rc), "lit_pixels": int((img > 0).sum().item()),
                  "image_sum": float(img.sum().item())}
        got_paths = ctx.spoly_paths(pipe.sol)

    # plain FP64 path on the same candidates: no gate, every step in FP64
    plain = None
    if (camera is not None or batched) and not args.no_plain and precision == binding.MIXED:
        pp = Pipeline(ctx, mode, binding.PLAIN_FP64, camera, explicit=explicit, flags=assign)
        pp.step(mesh, q)
        torch.cuda.synchronize()
        k = max(1, min(args.steps, args.plain_steps))
        prec = timed_steps(pp, mesh, q, k, flush, stream, torch)
        pms = sum(r["step"] for r in prec) / k
        ref_paths = ctx.spoly_paths(pp.sol)
        matched, worst = match_paths(got_paths, ref_paths)
        plain = {"ms_per_step": pms, "value": pairs / (pms * 1e-3), "steps": k, "paths_per_step": int(ref_paths.size),
                 "isolation_ms": statistics.mean(r["isolation"] for r in prec),
                 "recall_of_plain_paths": matched / max(1, ref_paths.size), "max_abs_delta_uv": worst,
                 "speedup": pms / (total_ms / args.steps)}
        pp.free()

    # end to end through the public API: every step hands the library its
    # inputs in pinned host memory (spoly_upload copies them to the device and
    # checks them there; an explicit chain list is copied by the chain
    # builder), runs the pipeline and reads the paths back into pinned host
    # memory, all inside the timed region
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(a).pin_memory() for a in host]
        hmesh, hq = ctx.mesh(pinned[0]), ctx.queries(*pinned[1:6])
        out = torch.empty(max(1, 2 * n_paths + 1024) * binding.PATH_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        cap = out.numel() // binding.PATH_DTYPE.itemsize
        if batched:
            pipe.explicit = pinned[6]

        def e2e_step():
            emesh, eq = ctx.spoly_upload(hmesh, hq)
            pipe.step(emesh, eq)
            return ctx.spoly_paths_into(pipe.sol, out, cap)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e_ms = []
        d2h = 0
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n = e2e_step()
            torch.cuda.synchronize()
            e_ms.append(1e3 * (time.perf_counter() - t0))
            d2h = min(n, cap) * binding.PATH_DTYPE.itemsize + 8
        e_total, e_value = job_rate(sum(e_ms), pairs, args.steps, world, dev)
        e2e = {"value": e_value, "unit": UNIT, "h2d_bytes_per_step": sum(a.nbytes for a in host),
               "d2h_bytes_per_step": d2h, "ms_per_step": e_total / args.steps}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    ph = {k: statistics.mean(r[k] for r in rec) for k in ("chains", "gate", "isolation", "polish", "k2", "k2_sign")}
    ph["step"] = total_ms / args.steps
    iso = ph["isolation"]
    achieved64 = FP64_FLOPS.get(kind, 0) * n_solved / (iso * 1e-3) / 1e12 if iso > 0 else 0.0
    roof_iso = {"bound": "alu", "pipe": "fp64", "kernel": "k1_isolate_kernel<float>",
                "achieved": achieved64, "peak": peak64, "unit": "TFLOP/s", "frac": achieved64 / peak64,
                "peak_source": "measured FP64 FMA microbenchmark (spoly_measure_peak)",
                "traffic": traffic("k1_isolate_kernel", args.workload),
                "nominal_fp64_tflops": NOMINAL_FP64_TFLOPS, "measured_fp32_tflops": peak32,
                "fp32_laplace_tflops": FP32_LAPLACE_FLOPS.get(kind, 0) * n_solved / (iso * 1e-3) / 1e12 if iso > 0
                else 0.0}
    roofline = roof_iso
    if kind in K2_KINDS or (batched and ph["k2"] >= max(ph["gate"], iso, ph["chains"])):
        # the FP32 sign kernels (tt_sign_kernel<float, N, G>, all size
        # classes), timed by the library with CUDA events around their
        # launches.  Work per determinant evaluation: elimination n^3/3 FMA,
        # the Bezout row recurrence 2 n^2 FMA, ~1,900 flop of Horner
        # evaluation of the coefficients (n from the library's counters of
        # the FP32 pass).
        ev = stats.get("k2_evals32", 0)
        n3 = stats.get("k2_eval32_n3", 0)
        nbar = (n3 / ev) ** (1.0 / 3.0) if ev else 0.0
        tt_flops = 2.0 / 3.0 * n3 + (4.0 * nbar * nbar + 1900.0) * ev
        sign_ms = ph["k2_sign"]
        ach = tt_flops / (sign_ms * 1e-3) / 1e12 if sign_ms > 0 else 0.0
        roofline = {"bound": "alu", "pipe": "fp32", "kernel": "tt_sign_kernel<float, N, G> (FP32 sign pass)",
                    "achieved": ach, "peak": peak32, "unit": "TFLOP/s", "frac": ach / peak32 if peak32 else None,
                    "peak_source": "measured FP32 FMA microbenchmark (spoly_measure_peak)", "traffic": None,
                    "flop_model": "2/3 n^3 + 4 n^2 + 1900 per Bezout determinant evaluation",
                    "evals_per_step": ev, "mean_bezout_size": nbar, "sign_ms_per_step": sign_ms,
                    "phase_ms_per_step": ph["k2"]}
    if use_gate:
        gate_tflops = GATE_FLOPS * n_cand / (ph["gate"] * 1e-3) / 1e12
        roof_gate = {"bound": "tensor", "kernel": "gate_kernel (features + BF16 tcgen05 MLP, TMEM accumulator + compaction)",
                     "achieved": gate_tflops, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": gate_tflops / BF16_PEAK_TFLOPS, "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)",
                     "traffic": traffic("gate_kernel", args.workload), "flops_per_candidate": GATE_FLOPS}
        # the dominant phase of the step carries the headline roofline
        if not (batched and roofline.get("pipe") == "fp32"):
            if ph["gate"] >= iso:
                roofline = dict(roof_gate, other={"isolation": roof_iso})
            else:
                roofline = dict(roof_iso, other={"gate": roof_gate})
        else:
            roofline = dict(roofline, other={"gate": roof_gate, "isolation": roof_iso})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("bf16+f32+f64" if use_gate else "f32+f64") if precision == binding.MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": desc, "precision": args.precision, "gate": "learned MLP" if use_gate else "off",
                   "candidates_per_step": pairs,
                   **({"distinct_triangles_per_step": n_cand} if mode == binding.CHAINS_FOOTPRINT_UNIQUE else {}),
                   **({"v1_intervals": args.intervals or 4096} if kind in K2_KINDS + ("mixed",) else {}),
                   "l2": "flushed between steps (512 MiB write)", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "solved_per_s": world * n_solved * args.steps / (total_ms * 1e-3),
        "paths_per_s": world * n_paths * args.steps / (total_ms * 1e-3),
        "solved_per_step": n_solved, "paths_per_step": n_paths, "counters": stats,
        "phase_ms": ph,
        "plain_fp64": plain,
        "render": render,
        "gate": gate_info,
        "autotune": tune,
        "roofline": roofline,
        "gpu_launches": launches_per_step(args.workload, use_gate, stats) * args.steps,
        "clocks": clk,
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        units = 24576 if camera is not None else (64 if kind == "T" else (16 if kind in K2_KINDS + ("mixed",) else 256))
        c, tcpu, _, sample = run_oracle_sample(s, camera, units if kind in K2_KINDS + ("mixed",) else min(units, s.n_queries),
                                               7, kind, args.intervals)
        line["cpu_baseline"] = {"value": c / tcpu, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line))
    pipe.free()
    if mlp is not None:
        ctx.spoly_mlp_free(mlp)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
