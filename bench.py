#!/usr/bin/env python
"""Benchmark of the voxel-grid hot path on GB300.

A step is one measurement of the plain per-frame path: K1 voxelize, K2
inflate, K3 ray-trace, K4 merge (vg_integrate_depth) and the re-centre
(vg_shift: a move of the grid's ring, whose new voxels the next frame's K4
sets to unknown), on the default workload
"seq": 640x480 float32 depth frames
along a seeded trajectory through a 20x20x5 m scene of 200 boxes and
cylinders, depth 5 m, 10% invalid pixels, depth noise sigma 1% of depth,
200x200x100 grid at 0.05 m, vox_inf 2, shift every frame.  Inputs are
synthetic (synth/), all frames resident in HBM before timing.  L2 is
flushed (a 256 MB write) before every timed step, outside its events.

Prints one JSON line.  value = Mvoxel-updates/s (loc voxels merged per
frame x frames / summed per-frame device time); per-frame latency p50/p99
in the same line.  `--impl reference` times the CPU oracle instead (the
reference arm: the paper's method restated in plain C, single core).
Under torchrun each rank runs an independent robot (its own seeded
sequence, no collective on the data path); rank 0 prints.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "per-frame latency p50/p99 and Mvoxel-updates/s, batched/served vs plain, 1 GB300"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="seq")
    ap.add_argument("--frames", type=int, default=100, help="frames in the synthetic sequence")
    ap.add_argument("--lanes", type=int, default=0, help="K3 lanes per ray (0 = library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the library's default schedule (no autotuner)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="oracle sample budget")
    ap.add_argument("--preroll", type=float, default=1.0, help="seconds of untimed frames before timing")
    ap.add_argument("--batch-robots", type=int, default=64,
                    help="robots per step of the batched form, over all ranks (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=200, help="timed steps of the batched form")
    ap.add_argument("--batch-frames", type=int, default=25,
                    help="rendered frames per robot of the batched form (cycled over the steps)")
    ap.add_argument("--serve-cameras", type=int, default=256,
                    help="cameras of the served form, over all ranks (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="seconds of Poisson arrivals (default 60 on one GPU, 20 per run on several, which "
                         "all stay held meanwhile)")
    ap.add_argument("--serve-rate", type=float, default=30.0, help="frames per second per camera")
    ap.add_argument("--serve-rate-high", type=float, default=60.0,
                    help="frames per second per camera of a second, heavier served run (0: skip)")
    ap.add_argument("--serve-seconds-high", type=float, default=2.0, help="seconds of arrivals of that run")
    ap.add_argument("--serve-queue-depth", type=int, default=4, help="launches the server keeps in flight")
    ap.add_argument("--serve-plain-max", type=int, default=0,
                    help="largest served batch run as per-frame kernel chains (0: library default)")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the step benchmark: the paper's Fig. 4 sweeps (step time vs points, "
                         "rays and voxels) on the GPU beside the single-core oracle")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (independent robots per rank)
# ---------------------------------------------------------------------------
class Dist:
    """Ranks of a torchrun launch (RANK / LOCAL_RANK / WORLD_SIZE / MASTER_*
    from the environment).  Only the barrier and the max / sum of the
    timings cross ranks; the data path has no collective.  backend: "nccl"
    on GPUs, "gloo" for the host-only tests of this plumbing."""

    def __init__(self, gpus, backend="nccl"):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        if gpus != self.world:
            raise SystemExit("--gpus %d but WORLD_SIZE %d: launch N>1 with torchrun" % (gpus, self.world))
        self.pg = None
        self.device = "cuda" if backend == "nccl" else "cpu"
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def _reduce(self, v, op):
        if not self.pg:
            return v
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device)
        self.pg.all_reduce(t, op=op)
        return float(t.item())

    def max(self, v):
        return self._reduce(v, self.pg.ReduceOp.MAX if self.pg else None)

    def sum(self, v):
        return self._reduce(v, self.pg.ReduceOp.SUM if self.pg else None)

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the run
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        sel = [p for t, p in self.samples if t0 <= t <= t1]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[0]) for p in sel if num(p[0]) is not None]
        mx = [num(p[1]) for p in sel if num(p[1]) is not None]
        reasons = sorted({self.NAMES[i] for p in sel for i in range(4) if p[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sel)}


def visible_gpu_index(local):
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        ids = [c.strip() for c in cvd.split(",") if c.strip()]
        if local < len(ids):
            return ids[local]
    return str(local)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", FALLBACK_HBM_GBS), "measured", d
    return FALLBACK_HBM_GBS, "fallback", {}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_frames(w, count, budget_s, start=0):
    """Run the oracle over frames start.. of w (integrate + shift, the same
    calls as a step) until count frames or budget_s seconds; returns the
    number of frames and the seconds they took."""
    from oracle import OracleGrid, OracleParams
    g = w.grid
    og = OracleGrid(OracleParams(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf),
                    w.frames[start % len(w.frames)].robot_pos)
    done, spent = 0, 0.0
    while done < count and spent < budget_s:
        f = w.frames[(start + done) % len(w.frames)]
        t = time.perf_counter()
        og.integrate_depth(f.T_wc, f.depth, w.cam.scale)
        og.shift(f.robot_pos)
        spent += time.perf_counter() - t
        done += 1
    return done, spent


def run_reference(args):
    from synth import make
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = make(args.workload, frames=args.frames)
    oracle_frames(w, args.warmup, 1e9)
    n, secs = oracle_frames(w, args.steps, 1e9, start=args.warmup)
    value = w.nvox * n / secs / 1e6
    cores = 1
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mvoxel-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / n * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload_config(w, args),
        "cpu_baseline": {"value": value, "unit": "Mvoxel-updates/s", "cores": cores, "kind": "oracle",
                         "sample": "%d frames of the %s sequence, integrate + shift each" % (n, w.name)},
        "e2e": {"value": value, "unit": "Mvoxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def workload_config(w, args):
    return {"workload": "%s: %dx%d %s depth, %d frames, grid %dx%dx%d at %.2f m, vox_inf %d, depth %.1f m, "
                        "fov %.0fx%.0f, shift every frame" % (
                            w.name, w.cam.W, w.cam.H, w.cam.dtype, len(w.frames), *w.grid.n, w.grid.vox_size,
                            w.grid.vox_inf, w.grid.depth, w.cam.fov_x, w.cam.fov_y),
            "form": "plain (one frame per launch sequence)", "l2": "flushed (256 MB write) before every step",
            "parallelism": "independent robots per GPU" if args.gpus > 1 else "single GPU"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def algorithmic_bytes(kind, w):
    """Bytes one launch of a kernel must move at minimum, as the workload's
    byte model counts them per voxel: its inputs read once and its outputs
    written once, with bit planes of N/8 bytes (N = loc voxels), the
    1-byte-per-voxel loc grid and the depth image.
      K1 voxelize  depth read + occ_raw written        W*H*bpp + N/8
      K2 inflate   occ_raw read + occ_inf written      2N/8
      K3 raytrace  occ_inf read + free, traced written 3N/8
      K4 merge     loc read + written, 3 planes read   2N + 3N/8
      K5 shift     loc read + written                  2N
    (K4 counts the merge with the re-centre's copy of loc, as the workload's
    model does; the ring-addressed grid writes only the voxels a frame marks
    and moves less.)"""
    n = w.nvox
    px = w.cam.W * w.cam.H * (2 if w.cam.dtype == "u16" else 4)
    return {"voxelize": px + n / 8, "inflate": 2 * n / 8, "raytrace": 3 * n / 8,
            "merge": 2 * n + 3 * n / 8, "shift": 2 * n, "loc_occupancy": n + n / 8}[kind]


def frame_bytes(w):
    """Algorithmic bytes of one frame (K1..K4, the re-centre counted in K4)."""
    return sum(algorithmic_bytes(k, w) for k in ("voxelize", "inflate", "raytrace", "merge"))


# One serial Amanatides-Woo step of the paper's ray trace with its
# occupancy test and mark: argmin of three tMax (2 compares, 2 selects),
# loop-end compare, index step, face step, tMax recompute (sub, mul),
# in-grid test (3 compares), linear index step, bit test (shift, and),
# mark (or).  Reported beside the HBM roofline as an issue-rate model.
OPS_PER_VISIT = 16


K3_SOURCES = ["paper_2112_13169_gb300/csrc/k_raytrace.cu", "paper_2112_13169_gb300/csrc/vg_rt.cuh",
              "paper_2112_13169_gb300/csrc/vg_units.cuh", "paper_2112_13169_gb300/csrc/vg_internal.cuh"]


def raytrace_traffic():
    """DRAM bytes per K3 launch from the committed ncu record, or None when
    a source K3 compiles from changed since it was taken."""
    import hashlib
    rec = os.path.join(ROOT, "profiles", "k_raytrace_dram.json")
    try:
        d = json.load(open(rec))
        for rel in K3_SOURCES:
            h = hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()
            if d["sources_sha256"].get(rel) != h:
                return None
        return d["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError, AttributeError):
        return None


def _pcts(ms):
    ms = np.asarray(ms, np.float64)
    return {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)), "mean": float(ms.mean())}


def measure_fused_seq(vg, w, args, flush, stream):
    """The sequence workload through the fused launch, one frame per batch."""
    import torch
    g = w.grid
    F = len(w.frames)
    depth = [torch.from_numpy(f.depth).cuda() for f in w.frames]
    grid = vg.Grid(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
    batch = vg.Batch(1)
    for k in range(max(3, args.warmup)):
        f = w.frames[k % F]
        batch.step([(grid, depth[k % F], f.T_wc, f.robot_pos, w.cam.scale)])
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        f = w.frames[k % F]
        flush.zero_()
        ev[k][0].record(stream)
        batch.step([(grid, depth[k % F], f.T_wc, f.robot_pos, w.cam.scale)])
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    status = batch.status()
    lat = [a.elapsed_time(b) for a, b in ev]
    batch.close()
    grid.close()
    return {"form": "fused: one persistent launch per frame (batch of 1)", "status": vg.strerror(status),
            "value": w.nvox * args.steps / (sum(lat) / 1e3) / 1e6, "unit": "Mvoxel-updates/s",
            "latency_ms": _pcts(lat), "l2": "flushed before every step"}


def shard(ids, rank, world):
    """The units (robots, cameras) rank `rank` of `world` runs: every
    world-th one, so that the ranks partition the units with no overlap and
    no collective on the data path."""
    return [u for u in ids if u % world == rank]


def measure_batched(vg, args, dist, stream):
    """The multi-robot workload: every robot's frame of a step in one fused
    launch (eager, and replayed from a CUDA graph), against the plain path
    on the same frames.  Robots are sharded over the ranks."""
    import torch
    from synth import make
    robots = shard(range(args.batch_robots), dist.rank, dist.world)
    F = args.batch_frames
    ws = [make("robot", robot=i, frames=F) for i in robots]
    depth = [[torch.from_numpy(f.depth).cuda() for f in w.frames] for w in ws]
    nvox = sum(w.nvox for w in ws)

    def grids():
        return [vg.Grid(w.grid.n, w.grid.vox_size, w.cam.fov_x, w.cam.fov_y, w.grid.depth, w.grid.vox_inf,
                        w.frames[0].robot_pos) for w in ws]

    def frames_of(gs, k):
        return [(gs[i], depth[i][k % F], w.frames[k % F].T_wc, w.frames[k % F].robot_pos, w.cam.scale)
                for i, w in enumerate(ws)]

    def agg(vox, secs):
        return dist.sum(vox) / dist.max(secs) / 1e6

    steps = args.batch_steps
    out = {"workload": "%d robots per step (%d on each of %d GPUs), each its own seeded scene and trajectory "
                       "(%d rendered frames per robot, cycled); depth %s f32; voxel {0.05, 0.1, 0.2} m; grids "
                       "80..256 x 80..256 x 40..96; vox_inf 1-3; %.1f M voxels and %.0f MB of depth per step "
                       "per GPU" % (args.batch_robots, len(robots), dist.world, F, "{320x240, 640x480, 848x480}",
                                    nvox / 1e6, sum(w.frames[0].depth.nbytes for w in ws) / 1e6),
           "steps": steps, "l2": "inputs and grids (> 1 GB) exceed L2; no flush"}

    # batched, eager
    gb = grids()
    batch = vg.Batch(len(ws))
    tuned = batch.autotune(frames_of(gb, 0), reps=2, stream=stream)
    for k in range(3):
        batch.step(frames_of(gb, k), stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    dist.barrier()
    t0 = time.perf_counter()
    for k in range(steps):
        ev[k][0].record(stream)
        batch.step(frames_of(gb, k), stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lat = [a.elapsed_time(b) for a, b in ev]
    out["batched"] = {"form": "one persistent fused launch per step", "status": vg.strerror(batch.status()),
                      "value": agg(nvox * steps, sum(lat) / 1e3), "unit": "Mvoxel-updates/s",
                      "step_ms": _pcts(lat), "per_frame_latency_ms": _pcts(lat),
                      "host_wall_Mvoxel_updates_per_s": agg(nvox * steps, wall),
                      "autotuned": dict(tuned, lanes=tuned["lanes"] or "per grid")}

    # batched, replayed from a CUDA graph (prepare on the host, replay)
    batch.prepare(frames_of(gb, 0))
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            batch.enqueue(cap)
    graph.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    dist.barrier()
    t0 = time.perf_counter()
    for k in range(steps):
        batch.prepare(frames_of(gb, k + 1))
        ev[k][0].record(stream)
        graph.replay()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lat = [a.elapsed_time(b) for a, b in ev]
    out["batched_graph"] = {"form": "the fused launch replayed from a CUDA graph",
                            "status": vg.strerror(batch.status()),
                            "value": agg(nvox * steps, sum(lat) / 1e3), "unit": "Mvoxel-updates/s",
                            "step_ms": _pcts(lat), "host_wall_Mvoxel_updates_per_s": agg(nvox * steps, wall)}
    del graph
    batch.close()
    for g in gb:
        g.close()

    # plain, the same frames one robot at a time
    gp = grids()
    for k in range(2):
        for i, w in enumerate(ws):
            f = w.frames[k % F]
            gp[i].integrate_depth(depth[i][k % F], f.T_wc, w.cam.scale)
            gp[i].shift(f.robot_pos)
    torch.cuda.synchronize()
    psteps = max(3, steps // 4)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(psteps)]
    dist.barrier()
    for k in range(psteps):
        ev[k][0].record(stream)
        for i, w in enumerate(ws):
            f = w.frames[k % F]
            gp[i].integrate_depth(depth[i][k % F], f.T_wc, w.cam.scale)
            gp[i].shift(f.robot_pos)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    lat = [a.elapsed_time(b) for a, b in ev]
    out["plain"] = {"form": "plain: one launch per kernel (K1-K4, the re-centre a ring move), robot after robot",
                    "steps": psteps, "value": agg(nvox * psteps, sum(lat) / 1e3), "unit": "Mvoxel-updates/s",
                    "step_ms": _pcts(lat)}
    for g in gp:
        g.close()
    out["speedup_batched_vs_plain"] = out["batched"]["value"] / out["plain"]["value"]
    return out


def _arrivals(n_cams, rate, seconds, seed):
    """Merged Poisson arrivals of n_cams cameras at `rate` Hz each: (time,
    camera) pairs, time in seconds from the start."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    lam = n_cams * rate
    while True:
        t += rng.exponential(1.0 / lam)
        if t > seconds:
            return out
        out.append((t, int(rng.integers(n_cams))))


def _lat_pcts(lat_s):
    ms = np.asarray(lat_s, np.float64) * 1e3
    return {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)), "max": float(ms.max())}


def measure_served(vg, args, dist):
    """Simulated cameras with Poisson arrivals through the continuous-batching
    server, and through a one-frame-at-a-time queue for comparison.  Both
    arms measure a frame's latency from its scheduled arrival time to the
    moment its device work is seen to end, on the host's monotonic clock.
    Cameras are sharded over the ranks (every rank its own server)."""
    import queue
    import threading
    import torch
    from synth import make
    from synth.scenes import CAMERA_KINDS
    nseq = 2 * CAMERA_KINDS
    seqs = [make("camera", robot=i, frames=4) for i in range(nseq)]
    mine = shard(range(args.serve_cameras), dist.rank, dist.world)
    budget = 40 << 30
    out = {"workload": "%d cameras (%d on each of %d GPUs), Poisson arrivals at %.0f Hz each for %.1f s; depth "
                       "from {320x240 f32/u16, 640x480 f32/u16, 1280x720 u16/f32} with grids 80x80x40 at 0.1 m, "
                       "200x200x100 at 0.05 m or 400x400x120 at 0.05 m (each camera draws one of %d rendered "
                       "sequences and cycles its 4 frames); %d GB budget per GPU" % (
                           args.serve_cameras, len(mine), dist.world, args.serve_rate, args.serve_seconds, nseq,
                           budget >> 30),
           "latency": "from each frame's scheduled arrival to the end of its device work (host monotonic clock), "
                      "in both arms"}
    # ---- continuous batching ---------------------------------------------
    server = vg.Server(budget, max_batch=128, max_width=1280, max_height=720, queue_depth=args.serve_queue_depth,
                       pending_frames=1024, plain_max=args.serve_plain_max)
    cams = {}
    for c in mine:
        w = seqs[c % nseq]
        g = w.grid
        try:
            cams[c] = (server.add_camera(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf,
                                         w.frames[0].robot_pos), w)
        except vg.VGError as e:
            if e.status != vg.VG_ENOMEM:
                raise
            break
    warm = [server.submit(cid, w.frames[0].depth, w.frames[0].T_wc, w.frames[0].robot_pos, w.cam.scale)
            for cid, w in cams.values()]
    for t in warm:
        if t is not None:
            server.wait(t)
    server.stats(reset=True)
    arr = [(t, c) for t, c in _arrivals(args.serve_cameras, args.serve_rate, args.serve_seconds, 99) if c in cams]
    nclient = 4
    tickets = [[] for _ in range(nclient)]
    late = [0.0] * nclient
    counter = {c: 1 for c in cams}

    # frames of one camera must be submitted in order: give each camera to one client
    per_client = [[] for _ in range(nclient)]
    for t, c in arr:
        per_client[c % nclient].append((t, c))
    start = [0.0]

    def client_of(k):
        t0 = start[0]
        for t, c in per_client[k]:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            late[k] = max(late[k], time.perf_counter() - t0 - t)
            cid, w = cams[c]
            f = w.frames[counter[c] % len(w.frames)]
            counter[c] += 1
            while True:   # a full pool (VG_EBUSY): retry; the latency still counts from t
                tk = server.submit(cid, f.depth, f.T_wc, f.robot_pos, w.cam.scale)
                if tk is not None:
                    tickets[k].append((tk, t0 + t, w.nvox))
                    break
                time.sleep(0.0002)

    threads = [threading.Thread(target=client_of, args=(k,)) for k in range(nclient)]
    dist.barrier()
    start[0] = time.perf_counter()
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    ok = all(server.wait(tk) == vg.VG_OK for lst in tickets for tk, _, _ in lst)
    elapsed = time.perf_counter() - start[0]
    st = server.stats()
    lat, lat_sub = [], []
    for lst in tickets:
        for tk, t_arr, _ in lst:
            rc, t_sub, t_done = server.ticket_times(tk)
            if rc == vg.VG_OK:
                lat.append(t_done - t_arr)
                lat_sub.append(t_done - t_sub)
    vox = sum(n for lst in tickets for _, _, n in lst)
    frames = sum(len(lst) for lst in tickets)
    out["served"] = {"form": "continuous batching: batches of up to 128 frames, %d in flight; a batch of at most "
                             "%s frames runs as per-frame kernel chains on parallel streams, a larger one as one "
                             "fused launch" % (args.serve_queue_depth,
                                               args.serve_plain_max or "4 (the library default)"),
                     "cameras_admitted": int(dist.sum(len(cams))), "all_ok": ok,
                     "frames": int(dist.sum(frames)), "frames_per_s": dist.sum(frames / elapsed),
                     "value": dist.sum(vox / elapsed / 1e6), "unit": "Mvoxel-updates/s",
                     "latency_ms": {k: dist.max(v) for k, v in _lat_pcts(lat).items()},
                     "latency_from_submit_ms": {k: dist.max(v) for k, v in _lat_pcts(lat_sub).items()},
                     "mean_frames_per_launch": st["mean_batch"], "launches": int(dist.sum(st["batches"])),
                     "device_bytes_in_use": int(st["bytes_in_use"]),
                     "client_max_lateness_ms": dist.max(1e3 * max(late))}
    server.close()

    # ---- a queue alone: one frame at a time through the plain path ---------
    grids = {}
    for c, (cid, w) in cams.items():
        g = w.grid
        grids[c] = vg.Grid(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
    q = queue.Queue()
    lat = []
    done = [0, 0]
    stream = torch.cuda.current_stream()

    def worker():
        while True:
            item = q.get()
            if item is None:
                return
            t_arr, c = item
            cid, w = cams[c]
            f = w.frames[counter[c] % len(w.frames)]
            counter[c] += 1
            grids[c].integrate_depth(f.depth, f.T_wc, w.cam.scale)   # host depth: staged by the library
            grids[c].shift(f.robot_pos)
            stream.synchronize()
            lat.append(time.perf_counter() - t_arr)
            done[0] += 1
            done[1] += w.nvox

    wt = threading.Thread(target=worker)
    wt.start()
    dist.barrier()
    t0 = time.perf_counter()
    for t, c in arr:
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        q.put((t0 + t, c))
    backlog = q.qsize()
    q.put(None)
    wt.join()
    elapsed = time.perf_counter() - t0
    for g in grids.values():
        g.close()
    out["plain_queue"] = {"form": "a queue alone: one frame at a time, plain path, synchronised per frame",
                          "frames": int(dist.sum(done[0])), "frames_per_s": dist.sum(done[0] / elapsed),
                          "value": dist.sum(done[1] / elapsed / 1e6), "unit": "Mvoxel-updates/s",
                          "backlog_when_arrivals_stopped": int(dist.sum(backlog)),
                          "latency_ms": {k: dist.max(v) for k, v in _lat_pcts(lat).items()}}
    for q in ("p50", "p99"):
        out["speedup_served_vs_plain_queue_%s_latency" % q] = (out["plain_queue"]["latency_ms"][q] /
                                                               max(1e-9, out["served"]["latency_ms"][q]))
    return out


def rank_seed(rank):
    """Seed of the robot sequence rank `rank` runs (None: the workload's own
    seed).  Every rank runs an independent robot: weak scaling."""
    return None if rank == 0 else 2000 + 17 * rank


def run_ours(args):
    import torch
    from paper_2112_13169_gb300 import build as vgbuild
    dist = Dist(args.gpus)
    torch.cuda.set_device(dist.local)
    if args.serve_seconds is None:
        args.serve_seconds = 60.0 if dist.world == 1 else 20.0
    vgbuild.build()
    from paper_2112_13169_gb300 import vg
    from synth import make

    w = make(args.workload, frames=args.frames, seed=rank_seed(dist.rank))
    g = w.grid
    F = len(w.frames)
    stream = torch.cuda.current_stream()
    depth_dev = torch.from_numpy(np.stack([f.depth for f in w.frames])).cuda()
    depth_host = torch.from_numpy(np.stack([f.depth for f in w.frames])).pin_memory()
    Ts = [f.T_wc for f in w.frames]
    poss = [f.robot_pos for f in w.frames]
    scale = w.cam.scale
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out_host = torch.empty(w.nvox, dtype=torch.uint8).pin_memory()

    sched = {}   # the schedule the autotuner picks (knob -> value); empty: the library's defaults

    def new_grid(flags=0, tuned=True):
        gr = vg.Grid(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, poss[0], flags=flags)
        if tuned:
            for knob, value in sched.items():
                gr.set(knob, value)
        if args.lanes:
            gr.tune(args.lanes)
        return gr

    def step(gr, k):
        f = k % F
        gr.integrate_depth(depth_dev[f], Ts[f], scale)
        gr.shift(poss[f])

    clocks = ClockSampler(visible_gpu_index(dist.local)) if dist.rank == 0 else None

    # the per-grid autotuner picks the schedule on the sequence's first frame
    # (untimed, on a grid of its own); the timed region runs with it, and the
    # library's default schedule is timed beside it over the same steps
    tune_info = None
    if not args.no_tune:
        grid = new_grid(tuned=False)
        best = grid.autotune(depth_dev[0], Ts[0], scale, reps=15)
        grid.close()
        tiles = {v: k for k, v in vg.TILE_NAMES.items()}
        sched.update({vg.VG_TUNE_INFLATE_TILE: tiles[best["tile"]], vg.VG_TUNE_RT_LANES: best["lanes"],
                      vg.VG_TUNE_RT_CTAS_PER_SM: best["ctas_per_sm"], vg.VG_TUNE_MERGE_WORDS: best["merge_words"],
                      vg.VG_TUNE_INFLATE_TMA: best["inflate_tma"], vg.VG_TUNE_EARLY_INFLATE: best["early_inflate"]})
        tune_info = {"schedule": best,
                     "schedule_is_default": (best["tile"] == "auto" and best["ctas_per_sm"] == 0 and
                                             best["merge_words"] == 256 and best["inflate_tma"] == 1 and
                                             best["early_inflate"] == 1)}

    # warm-up steps, then about a second of pre-roll so clocks settle; the
    # timed steps continue on the same grid (its first frames pay one-time
    # host costs that would otherwise leave the device idle inside a timed
    # step), along the same sequence
    grid = new_grid()
    k0 = 0
    for k0 in range(max(3, args.warmup)):
        step(grid, k0)
    k0 += 1
    torch.cuda.synchronize()
    t_pre = time.time()
    while time.time() - t_pre < args.preroll:
        step(grid, k0)
        k0 += 1
        if k0 % 50 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()

    # ---- timed region: per-frame device time ------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = grid.profile_read()
    dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    # a head start of a few L2 flushes (untimed), so that the host is frames
    # ahead of the device when the first timed frame starts: a host stall
    # right after the synchronize would otherwise leave the device waiting
    # inside that frame's events (one 192 us frame among 20 of 42 us)
    for _ in range(4):
        flush.zero_()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step(grid, k0 + k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    t_wall1 = time.time()
    lat_ms = np.array([a.elapsed_time(b) for a, b in ev])
    launches1 = grid.profile_read()
    gpu_launches = int(sum(launches1[k][2] - launches0[k][2] for k in vg.KERNELS))
    grid.close()

    if tune_info is not None:
        # the tuned and the default schedule over the same steps, frames
        # alternating between a grid of each, in turn first (so drifts and
        # the order hit both alike)
        gt, gd = new_grid(), new_grid(tuned=False)
        for k in range(3):   # untimed first frames of each grid
            step(gt, k)
            step(gd, k)
        ev2 = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
               for _ in range(2)]
        for k in range(args.steps):
            # the tuned grid first in even steps, the default one in odd ones
            for j in ((0, 1) if k % 2 == 0 else (1, 0)):
                flush.zero_()
                ev2[j][k][0].record(stream)
                step((gt, gd)[j], 3 + k)
                ev2[j][k][1].record(stream)
        torch.cuda.synchronize()
        gt.close()
        gd.close()
        for j, name in enumerate(("tuned", "default")):
            l2 = np.array([a.elapsed_time(b) for a, b in ev2[j]])
            tune_info["alternating_%s_latency_ms" % name] = {"p50": float(np.percentile(l2, 50)),
                                                             "p99": float(np.percentile(l2, 99)),
                                                             "mean": float(l2.mean())}
        tune_info["gain_mean"] = (tune_info["alternating_default_latency_ms"]["mean"] /
                                  tune_info["alternating_tuned_latency_ms"]["mean"])

    total_s = float(lat_ms.sum()) / 1e3
    total_s_max = dist.max(total_s)
    vox_all = dist.sum(w.nvox * args.steps)
    value = vox_all / total_s_max / 1e6

    # ---- per-kernel profile over the same steps (roofline) ---------------
    grid = new_grid()
    for k in range(3):   # untimed first frames
        step(grid, k)
    grid.profile(True)
    grid.profile_read(reset=True)
    for k in range(args.steps):
        flush.zero_()
        step(grid, 3 + k)
    torch.cuda.synchronize()
    prof = grid.profile_read(reset=True)
    grid.close()
    # in-grid voxel visits of K3 (stats counters, separate untimed pass)
    grid = new_grid(vg.VG_FLAG_STATS)
    for k in range(args.steps):
        step(grid, k)
    st = grid.stats()
    grid.close()

    # ---- end to end: host buffers through the C ABI -----------------------
    grid = new_grid()
    for k in range(3):   # untimed first frames, through the same host buffers
        grid.integrate_depth(depth_host[k % F], Ts[k % F], scale)
        grid.shift(poss[k % F])
        grid.read(out_host)
    e2e_s = 0.0
    for k in range(3, 3 + args.steps):
        f = k % F
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        grid.integrate_depth(depth_host[f], Ts[f], scale)     # H2D inside the library
        grid.shift(poss[f])
        grid.read(out_host)                                   # D2H of the grid
        stream.synchronize()
        e2e_s += time.perf_counter() - t
    grid.close()
    e2e_value = dist.sum(w.nvox * args.steps) / dist.max(e2e_s) / 1e6

    # ---- other forms (reported beside the headline) ------------------------
    forms = {"fused_seq": measure_fused_seq(vg, w, args, flush, stream)}
    if args.batch_robots > 0:
        forms["multi_robot"] = measure_batched(vg, args, dist, stream)
    if args.serve_cameras > 0:
        forms["served"] = measure_served(vg, args, dist)
        if args.serve_rate_high > 0:
            # twice the stated load: the one-frame-at-a-time queue falls behind
            hi = argparse.Namespace(**vars(args))
            hi.serve_rate, hi.serve_seconds = args.serve_rate_high, args.serve_seconds_high
            forms["served_high_load"] = measure_served(vg, hi, dist)
    t_forms_end = time.time()

    if clocks:
        clocks.stop()

    if dist.rank != 0:
        dist.close()
        return 0

    hbm_peak, peak_kind, peaks = measured_peaks()
    kern = {}
    for name in vg.KERNELS:
        ms, timed, total = prof[name]
        if timed:
            avg_s = ms / timed / 1e3
            alg = algorithmic_bytes(name, w)
            kern[name] = {"avg_us": avg_s * 1e6, "launches": timed, "share": 0.0, "alg_bytes": alg,
                          "gbs": alg / avg_s / 1e9}
    tot = sum(v["avg_us"] * v["launches"] for v in kern.values())
    for v in kern.values():
        v["share"] = v["avg_us"] * v["launches"] / tot
    dom = max(kern, key=lambda k: kern[k]["avg_us"] * kern[k]["launches"])
    d = kern[dom]
    visits_per_frame = st["ray_visits"] / max(1, st["frames"])
    # the dominant kernel against the HBM roofline: its algorithmic bytes per
    # launch over its average event time, against the measured copy peak
    roofline = {"kernel": dom, "bound": "hbm", "achieved": d["gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": d["gbs"] / hbm_peak, "traffic": raytrace_traffic() if dom == "raytrace" else None,
                "peak_source": "%s hbm_gbs" % peak_kind, "alg_bytes_per_launch": d["alg_bytes"],
                "avg_us": d["avg_us"]}
    if dom == "raytrace":
        # K3 is bound by instruction issue, not bytes: the same launch as
        # ray-voxel visits x OPS_PER_VISIT lane operations against every lane
        # of every SM issuing once a cycle at the measured maximum clock
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak_tops = sms * 128 * mhz * 1e6 / 1e12
        achieved = visits_per_frame * OPS_PER_VISIT / (d["avg_us"] * 1e-6) / 1e12
        roofline["alu_model"] = {"achieved": achieved, "peak": peak_tops, "unit": "T lane-ops/s",
                                 "frac": achieved / peak_tops, "ops_per_visit": OPS_PER_VISIT,
                                 "visits_per_launch": visits_per_frame,
                                 "peak_source": "%d SMs x 128 lanes x %.0f MHz (%s sm_max_mhz)" % (
                                     sms, mhz, peak_kind)}
    fb = frame_bytes(w)
    frame_roofline = {"alg_bytes_per_frame": fb, "ms_per_frame": float(lat_ms.mean()),
                      "achieved_GBps": fb / (float(lat_ms.mean()) * 1e-3) / 1e9,
                      "frac": fb / (float(lat_ms.mean()) * 1e-3) / 1e9 / hbm_peak}

    cpu = None
    if not args.no_cpu_baseline:
        n, secs = oracle_frames(w, F, args.cpu_seconds)
        cpu = {"value": w.nvox * n / secs / 1e6, "unit": "Mvoxel-updates/s", "cores": 1, "kind": "oracle",
               "sample": "first %d frames of the %s sequence, integrate + shift each, single thread" % (n, w.name)}

    summ = clocks.summary(t_pre - 0.5, t_wall1 + 0.5) if clocks else {"sm_mhz": None, "sm_max_mhz": None,
                                                                       "reasons": [], "samples": 0}
    line = {
        "metric": METRIC, "value": value, "unit": "Mvoxel-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(lat_ms.mean()),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload_config(w, args),
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                       "mean": float(lat_ms.mean()), "max": float(lat_ms.max())},
        "e2e": {"value": e2e_value, "unit": "Mvoxel-updates/s",
                "h2d_bytes_per_step": int(depth_host[0].numel() * depth_host.element_size()),
                "d2h_bytes_per_step": int(w.nvox),
                "ms_per_step": e2e_s / args.steps * 1e3},
        "gpu_launches": gpu_launches,
        "roofline": roofline,
        "frame_roofline": frame_roofline,
        "kernels": {k: {"avg_us": round(v["avg_us"], 3), "share": round(v["share"], 4),
                        "alg_bytes": int(v["alg_bytes"]), "alg_GBps": round(v["gbs"], 1),
                        "frac_hbm": round(v["gbs"] / hbm_peak, 5)} for k, v in kern.items()},
        "ray_visits_per_frame": visits_per_frame,
        "autotune": tune_info,
        "cpu_baseline": cpu,
        "clocks": {"sm_mhz": summ["sm_mhz"], "sm_max_mhz": summ["sm_max_mhz"], "reasons": summ["reasons"],
                   "samples": summ["samples"]},
        "wall_s_timed_region": t_wall1 - t_wall0,
        "forms": forms,
    }
    print(json.dumps(line))
    dist.close()
    return 0


# ---------------------------------------------------------------------------
# the paper's sweeps (Fig. 4a-c)
# ---------------------------------------------------------------------------
def _kernel_us(vg, grid, feed, frames, flush, kinds):
    """Average event time per frame of the named kernels over `frames` calls
    of feed(grid, k), after three untimed ones; L2 flushed before each."""
    import torch
    for k in range(3):
        feed(grid, k)
    torch.cuda.synchronize()
    grid.profile(True)
    grid.profile_read(reset=True)
    for k in range(frames):
        flush.zero_()
        feed(grid, k)
    torch.cuda.synchronize()
    prof = grid.profile_read(reset=True)
    return sum(prof[kind][0] / max(1, prof[kind][1]) for kind in kinds) * 1e3


def _cpu_us(fn, reps):
    best = None
    for _ in range(reps):
        t = time.perf_counter()
        fn()
        dt = time.perf_counter() - t
        best = dt if best is None else min(best, dt)
    return best * 1e6


def run_sweeps(args):
    """Fig. 4a-c of the paper: the time of step 2 (populate occupied voxels:
    K1 + K2), step 3 (ray-trace: K3) and step 4 (merge: K4) as the number of
    points, rays and voxels grows, for the GPU kernels (CUDA events the
    library records around each launch, L2 flushed before each frame) and
    the oracle's steps on one host core (best of a few runs).  Standard
    set-up of Sec. V unless swept: 320x240, fov 85x101, depth 6.5 m,
    100x100x20 at 0.15 m, vox_inf 2."""
    import torch
    from paper_2112_13169_gb300 import build as vgbuild
    vgbuild.build()
    from paper_2112_13169_gb300 import vg
    from oracle import OracleParams
    from oracle import oracle as O
    from synth import make
    vg.load()
    orc = O.default()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    w = make("paper", frames=1)
    f = w.frames[0]
    pos = f.robot_pos
    std = dict(n=(100, 100, 20), vs=0.15, fx=85.0, fy=101.0, depth=6.5, r=2)
    rng = np.random.default_rng(4)
    out = {}

    def grid(n, vs, fx, fy, depth, r):
        return vg.Grid(n, vs, fx, fy, depth, r, pos)

    def oparams(n, vs, fx, fy, depth, r):
        return OracleParams(tuple(n), vs, fx, fy, depth, r)

    # (a) populate occupied voxels vs obstacle points (a point cloud in the
    # camera frame, uniform in the field of view up to the range)
    rows = []
    for npts in (1000, 5000, 20000, 100000, 300000, 1000000):
        z = rng.uniform(0.3, std["depth"], npts)
        tx, ty = np.tan(np.radians(std["fx"] / 2)), np.tan(np.radians(std["fy"] / 2))
        xyz = np.stack([rng.uniform(-tx, tx, npts) * z, rng.uniform(-ty, ty, npts) * z, z], 1).astype(np.float32)
        dev = torch.from_numpy(xyz).cuda()
        g = grid(**std)
        gpu = _kernel_us(vg, g, lambda gr, k: gr.integrate_points(dev, f.T_wc), 20, flush, ("voxelize", "inflate"))
        g.close()
        p = oparams(**std)
        o = orc.origin(p, pos)
        pose = orc.pose_vc(p, f.T_wc, o)
        cpu = _cpu_us(lambda: orc.inflate(p, orc.voxelize_points(p, pose, xyz)[0]), 3)
        rows.append({"points": npts, "gpu_us": gpu, "cpu_us": cpu, "cpu_over_gpu": cpu / gpu})
    out["populate_vs_points"] = rows

    # (b) ray-trace vs rays: the field of view sets the bundle (the same
    # depth image, back-projected with each field of view's intrinsics)
    rows = []
    dev = torch.from_numpy(f.depth).cuda()
    for fov in (40.0, 60.0, 85.0, 101.0, 120.0, 140.0):
        cfg = dict(std, fx=fov, fy=fov)
        g = grid(**cfg)
        gpu = _kernel_us(vg, g, lambda gr, k: gr.integrate_depth(dev, f.T_wc), 20, flush, ("raytrace",))
        g.close()
        p = oparams(**cfg)
        (vd, hw, hh), nrays = orc.ray_bundle(p)
        o = orc.origin(p, pos)
        pose = orc.pose_vc(p, f.T_wc, o)
        occ_inf = orc.inflate(p, orc.voxelize_depth(p, pose, f.depth)[0])
        cpu = _cpu_us(lambda: orc.raytrace(p, pose, occ_inf), 3)
        rows.append({"fov_deg": fov, "rays": int(nrays), "gpu_us": gpu, "cpu_us": cpu, "cpu_over_gpu": cpu / gpu})
    out["raytrace_vs_rays"] = rows

    # (c) merge vs voxels in the grid (the standard frame, no re-centre)
    rows = []
    for n in ((40, 40, 15), (100, 100, 20), (150, 150, 30), (200, 200, 100), (400, 400, 120)):
        cfg = dict(std, n=n)
        g = grid(**cfg)
        gpu = _kernel_us(vg, g, lambda gr, k: gr.integrate_depth(dev, f.T_wc), 20, flush, ("merge",))
        g.close()
        p = oparams(**cfg)
        o = orc.origin(p, pos)
        pose = orc.pose_vc(p, f.T_wc, o)
        occ_inf = orc.inflate(p, orc.voxelize_depth(p, pose, f.depth)[0])
        fr, tr, _ = orc.raytrace(p, pose, occ_inf)
        loc = np.zeros(p.shape, np.uint8)
        cpu = _cpu_us(lambda: orc.merge(orc.resolve(occ_inf, fr, tr), loc), 3)
        nv = n[0] * n[1] * n[2]
        rows.append({"voxels": nv, "gpu_us": gpu, "cpu_us": cpu, "cpu_over_gpu": cpu / gpu})
    out["merge_vs_voxels"] = rows
    print(json.dumps({"sweeps": out, "gpu": "GB300, one GPU; CUDA events around each launch",
                      "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": "best of 3 runs per point"},
                      "data": "synthetic: the paper workload's first frame, random frustum points"}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweeps(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
