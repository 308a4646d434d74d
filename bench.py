#!/usr/bin/env python
"""Benchmark of BundleFusion's pose-alignment hot path (Sec. 4.2-4.4) on B300.

Workload (the line's value): 256 independent chunk solves of U{3..11} frames at 320x240 (1831
frames, 3.9 GB of FP32 frame planes: larger than L2), all intra-chunk pairs (6559 pairs,
13118 directed dense pairs), 100-400 sparse correspondences per pair (sigma 1 cm, 5 % outliers),
6 Gauss-Newton x 10 PCG iterations each, FP32 arithmetic, FP32 frame storage, solved as one batch
(one launch sequence replayed as a CUDA graph, the dense work decomposition chosen by the
library's autotuner).  One step = the whole hot path once over the batch: frame preprocessing
from device-resident raw depth / luminance, pair-set and table construction, 6 linearisations
(dense + sparse terms, block reduction, assembly), 6 x 10 PCG iterations and pose updates, final
energy and r_max, results read back.

Metric: Gauss-Newton iterations per second (one chunk's iteration = 1; whole job over all ranks),
chunk-solve p50 / p99 latency of the batch and of the plain path (the FP32 one-solve-per-launch
sequence, kernel by kernel), and the dense kernel's algorithmic HBM bandwidth as a fraction of the
measured peak.  Extra legs: the same batch end to end from host buffers, with BF16 storage and as
one persistent launch; the 300-keyframe 80x60 global solve; the 2000-keyframe 160x120 global solve;
serving; the steps around the solver; the FP64 oracle on the host cores.

Under torchrun (N > 1) every rank solves its own replica of the batch (chunks are independent
problems): scaling "weak", no collective on the data path, the step time is the max over ranks.
"""
import argparse
import json
import os

# the FP64 oracle leg runs on one BLAS thread (set before numpy loads its BLAS)
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GN iterations/sec + chunk-solve p50/p99 latency vs plain GPU path; HBM GB/s frac"
UNIT = "GN iterations/s"
DENSE_BYTES_PER_PX = 48  # FP32: source D, n, I (20 B) + target D, n nearest (16 B) + I, grad I bilinear (12 B)
# 16-bit storage: D stays FP32, n, I, grad I take 2 B each: source 4 + 8, target 4 + 6 + 6
DENSE_BYTES_PER_PX_16 = 28
STORAGE_CODES = {"fp32": lambda bf: bf.BF_STORE_FP32, "bf16": lambda bf: bf.BF_STORE_BF16,
                 "fp16": lambda bf: bf.BF_STORE_FP16}


def dense_bytes_per_px(storage):
    return DENSE_BYTES_PER_PX if storage == "fp32" else DENSE_BYTES_PER_PX_16

# FP32 flops of the dense kernel per directed source pixel on this workload: ncu FFMA x 2 + FADD + FMUL
# thread counts of one ACCUM launch divided by its 21.84 M directed source pixels, counted on the
# scalar build (profiles/k_dense_staged_global300_80x60.md); the packed-FMA build performs the
# same operations, two per instruction
DENSE_FLOPS_PER_PX = 122.8
# DRAM bytes (read + write) of one dense ACCUM launch from an ncu capture of the current kernel
# (cold cache); set to None whenever the dense kernel changes until it is captured again.
# 300-keyframe 80x60 workload, k_dense_staged: two launches read 46.44 / 46.43 MB and wrote
# 0.13 / 0.01 MB (ncu, the current kernel): the frames' unique bytes, which stay in L2
DENSE_TRAFFIC_BYTES = 46.50e6
# 256-chunk 320x240 batch, k_dense (tiled, autotuned decomposition): one launch of the 32-chunk batch
# (the same chunk distribution, 1496 directed pairs = 114.9 M directed source pixels) read 523.63 MB and
# wrote 9.80 MB (ncu, one launch, the current kernel: 4 CTAs per SM, register spills included);
# scaled by directed source pixels to the
# 256-chunk launch (1007.5 M): DRAM traffic is the frames' unique bytes, which grow with the batch
DENSE_TRAFFIC_BYTES_CHUNKS = (523.63e6 + 9.80e6) * 1007.5 / 114.9
# untimed warm-up floor after the W warm-up steps (seconds of repeated steps)
WARMUP_MIN_S = 0.5
# B300 FP32 peak: 148 SMs x 128 FP32 lanes x 2 flop x max SM clock
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


def max_over_ranks(x, dist=None):
    """The largest x over all ranks of the process group (x itself without one): the job's time is
    its slowest rank's.  NCCL reduces on the rank's GPU, gloo on the host."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_step, steps, world, total_ms):
    """Whole-job throughput: the units every rank processed in `steps` steps over the (max-over-ranks)
    time; each rank runs its own replica (weak scaling)."""
    return units_per_step * steps * world / (total_ms / 1000.0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["mixed", "fp32"],
                    help="arithmetic of the timed batch (chunk solves meet the accuracy targets in FP32)")
    ap.add_argument("--no-extras", action="store_true", help="skip every leg after the headline (e2e, plain, ...)")
    ap.add_argument("--profile-run", action="store_true", help="short run for ncu: no extras, no clocks")
    ap.add_argument("--no-graph", action="store_true", help="launch kernel by kernel instead of a CUDA graph")
    ap.add_argument("--tile-px", type=int, default=-1,
                    help="dense work item size in source pixels; -1 = the library's autotuner, 0 = staged target")
    ap.add_argument("--global-only", action="store_true",
                    help="run only the 300-keyframe 80x60 global solve leg (one JSON line)")
    ap.add_argument("--serving-only", action="store_true", help="run only the serving leg (one JSON line)")
    ap.add_argument("--serving-seconds", type=float, default=20.0,
                    help="length of the serving session (the full-length stream is 600 s)")
    ap.add_argument("--persistent", action="store_true",
                    help="time the batch as one persistent launch (half-frame tiles) instead of the launch sequence")
    ap.add_argument("--chunks", type=int, default=256,
                    help="chunks in the timed batch (a smaller batch for profiling captures; the line then names it)")
    ap.add_argument("--large-only", action="store_true",
                    help="run only the 2000-keyframe 160x120 BF16 global solve leg (one JSON line)")
    ap.add_argument("--batch-only", action="store_true", help="only the 256-chunk batch legs (FP32 and BF16 storage)")
    ap.add_argument("--next-rows-only", action="store_true",
                    help="run only the pruning / verification / key-point / TSDF legs (one JSON line)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="frame storage of the timed workload (16-bit: normals, I, grad I)")
    ap.add_argument("--dense-tc", type=int, default=0, choices=[0, 1, 3],
                    help="form the dense sums on the tensor cores (1: TF32 operands, 3: three TF32 products)")
    ap.add_argument("--pcg-variant", type=int, default=0, choices=[0, 1, 2, 3],
                    help="PCG kernel: 0 auto, 1 one CTA per problem, 2 grid-cooperative, 3 cluster")
    return ap.parse_args()


def workload(n_chunks=256):
    """The 256-chunk 320x240 batch (its default solve parameters); fewer chunks for profiling."""
    import synth
    prob = synth.cfg3() if n_chunks == 256 else synth.cfg3(n_chunks=n_chunks)
    return prob, prob.solve


def quantile(v, f):
    v = sorted(v)
    return v[min(len(v) - 1, int(f * len(v)))] if v else None


# ------------------------------------------------------------------------------- clocks
class _Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml ships with the driver): the SM clock, its
    maximum and the active clock-event-reason mask of the device torch calls `index`."""
    CLOCK_SM = 1

    def __init__(self, index):
        import ctypes
        self.c = ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.lib = lib
        self.h = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(index).uuid)
        except Exception:
            pass
        ok = uuid and lib.nvmlDeviceGetHandleByUUID(("GPU-" + uuid).encode(), ctypes.byref(self.h)) == 0
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def clock(self, fn):
        v = self.c.c_uint()
        if fn(self.h, self.c.c_int(self.CLOCK_SM), self.c.byref(v)) != 0:
            raise RuntimeError("clock query failed")
        return float(v.value)

    def sm_mhz(self):
        return self.clock(self.lib.nvmlDeviceGetClockInfo)

    def sm_max_mhz(self):
        return self.clock(self.lib.nvmlDeviceGetMaxClockInfo)

    def reasons(self):
        v = self.c.c_ulonglong()
        if self.reasons_fn(self.h, self.c.byref(v)) != 0:
            raise RuntimeError("reason query failed")
        return int(v.value)


class Clocks:
    """SM clock and clock-event-reason sampler running during the timed region.

    NVML (read-only queries) every 5 ms from a thread, so that even a timed region of a few tens of
    milliseconds gets samples; nvidia-smi at its 200 ms minimum period where NVML cannot be loaded."""

    # (name, NVML clock-event-reason bit)
    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_s=0.005):
        self.index = index
        self.period = period_s
        self.rows = []
        self.thread = None
        self.stop_ev = threading.Event()
        self.proc = None
        self.file = None

    def _nvml_loop(self, nv):
        mx = nv.sm_max_mhz()
        while not self.stop_ev.is_set():
            try:
                sm, r = nv.sm_mhz(), nv.reasons()
                self.rows.append((sm, mx, [name for name, bit in self.REASONS if r & bit]))
            except Exception:
                pass
            self.stop_ev.wait(self.period)

    def start(self):
        try:
            nv = _Nvml(self.index)
            self.thread = threading.Thread(target=self._nvml_loop, args=(nv,), daemon=True)
            self.thread.start()
            return
        except Exception:
            self.thread = None
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_ev.set()
            self.thread.join(timeout=5)
            rows, source = self.rows, "nvml, 5 ms"
        elif self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.file.flush()
            rows = []
            with open(self.file.name) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 8 and parts[0].replace(".", "").isdigit():
                        rows.append((float(parts[0]), float(parts[1]) if parts[1].replace(".", "").isdigit() else 0.0,
                                     [name for (name, _), v in zip(self.REASONS, parts[4:8]) if v.lower() == "active"]))
            os.unlink(self.file.name)
            source = "nvidia-smi, 200 ms"
        else:
            return None
        if not rows:
            return None
        sm = [r[0] for r in rows]
        mx = max(r[1] for r in rows)
        load = [x for x in sm if mx and x > 0.5 * mx] or sm
        reasons = sorted({n for r in rows for n in r[2]})
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows),
                "source": source}


# ------------------------------------------------------------------------- CPU baseline
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


class OracleSampler:
    """The FP64 oracle (Sec. 4.4 Gauss-Newton over explicitly assembled normal equations) on the
    host cores, for a bounded sample of the chunk batch: a spawn process pool whose workers build
    the sampled chunks' frames from their raw depth / luminance on first use and evaluate the dense
    pairs; the parent assembles the sparse term, sums the pairs in order, and runs the block-Jacobi
    PCG on the assembled system and the pose update.  One chunk GN iteration = 1 unit, as on the
    GPU."""

    def __init__(self, prob, prm, chunk_ids, processes=None):
        from oracle import frames as ofr, system
        from oracle.system import SolveParams
        self.prob, self.chunk_ids = prob, list(chunk_ids)
        self.P = SolveParams(n_gn=1, n_pcg=prm["n_pcg"], w_sparse=prm["w_sparse"], w_dense=prm["w_dense"],
                             w_photo=prm["w_photo"], w_geo=prm["w_geo"])
        self.cores = processes or host_cores()
        fids = sorted({int(f) for k in self.chunk_ids for f in prob.chunks[k]})
        cache = ofr.FrameCache({f: prob.depth[f] for f in fids}, {f: prob.lum[f] for f in fids}, prob.intr)
        self.pool = system.frame_pool(cache, self.cores)
        self.pool.map(abs, range(4 * self.cores))  # workers started before any timing

    def gn_iterations(self, chunks):
        """One GN iteration of each listed chunk from its initial poses; returns wall seconds."""
        from oracle import solver, system
        prob, P = self.prob, self.P
        pmap = lambda f, tasks: self.pool.map(f, tasks, chunksize=1)  # noqa: E731
        t0 = time.perf_counter()
        for k in chunks:
            ids = [int(f) for f in prob.chunks[k]]
            sp = solver.sparse_pairs_for(prob, ids)
            X0 = prob.init[ids]
            dp = system.dense_pair_set(X0, sp, P.max_angle_deg)
            S = system.assemble([None] * len(ids), prob.intr, X0, sp, dp, P, P.w_dense, pmap=pmap, frame_keys=ids)
            Minv, _ = solver.block_jacobi_inverse(S.A, P.precond)
            delta, _ = solver.pcg(S.A, S.b, Minv, P.n_pcg)
            solver.apply_step(X0, delta)
        return time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_baseline_leg(prob, prm, n_chunks=16):
    """The oracle on a bounded sample: one GN iteration of each of the first n_chunks chunks."""
    chunks = list(range(n_chunks))
    s = OracleSampler(prob, prm, chunks)
    try:
        dt = s.gn_iterations(chunks)
    finally:
        s.close()
    frames = sum(len(prob.chunks[k]) for k in chunks)
    return {"value": len(chunks) / dt, "unit": UNIT, "cores": s.cores, "kind": "oracle",
            "sample": f"one Gauss-Newton iteration ({prm['n_pcg']} PCG) of each of chunks 0..{n_chunks - 1} of this "
                      f"workload ({frames} frames at 320x240, frames preprocessed inside the timing): FP64 numpy, "
                      f"system assembled explicitly, dense pairs spread over {s.cores} spawn processes "
                      f"(1 BLAS thread each), measured, not extrapolated; {dt:.2f} s wall",
            "cpu": cpu_model()}


# ------------------------------------------------------------------------------ reference
def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.  Each step is one GN
    iteration of the next chunk of the batch (in chunk order), measured; the line reports what ran."""
    if rank != 0:
        return
    prob, prm = workload()
    n = args.warmup + args.steps
    chunks = [k % len(prob.chunks) for k in range(n)]
    s = OracleSampler(prob, prm, sorted(set(chunks)))
    try:
        times = [s.gn_iterations([k]) for k in chunks]
    finally:
        s.close()
    timed = times[args.warmup:]
    value = len(timed) / sum(timed)
    frames = sum(len(prob.chunks[k]) for k in chunks[args.warmup:])
    desc = (f"each step: one Gauss-Newton iteration ({prm['n_pcg']} PCG) of one chunk of this workload, chunks "
            f"{chunks[args.warmup]}..{chunks[-1]} in order ({frames} frames at 320x240 in the timed steps), frames "
            f"preprocessed inside the timing; FP64 numpy with explicit normal equations, dense pairs over "
            f"{s.cores} spawn processes; every step measured (ms_per_step x steps is the time that ran)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sum(timed) / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(prob, prm, "fp32", "fp64 (oracle)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": s.cores, "kind": "oracle", "sample": desc,
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(prob, prm, storage, precision, **extra):
    intr = prob.intr
    n = len(prob.chunks)
    cfg = {"workload": f"chunks{n}_320x240: {n} chunk solves of U{{3..11}} frames at 320x240",
           "chunks": len(prob.chunks), "frames": prob.n_frames, "resolution": f"{intr['W']}x{intr['H']}",
           "pairs": int(len(prob.pairs)), "correspondences": prob.n_corr, "n_gn": prm["n_gn"], "n_pcg": prm["n_pcg"],
           "storage": storage, "precision": precision,
           "l2": "inputs larger than L2 (3.9 GB of FP32 frame planes, 126 MB L2): no flush between steps"}
    cfg.update(extra)
    return cfg


# ------------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1604_01093_b300 as bf

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    stream = torch.cuda.Stream(dev)  # the library and the timing events share this stream
    torch.cuda.set_stream(stream)
    only = [(args.large_only, "large_global", lambda: large_global_leg(bf, torch, dev, stream)),
            (args.global_only, "global300", lambda: global300_leg(bf, torch, dev, stream, args)),
            (args.next_rows_only, "next_rows", lambda: next_rows_leg(bf, torch, dev, stream)),
            (args.serving_only, "serving", lambda: serving_leg(bf, torch, dev, seconds=args.serving_seconds)),
            (args.batch_only, "chunk_batch_bf16",
             lambda: chunk_batch_leg(bf, torch, dev, stream, storage="bf16"))]
    for flag, name, fn in only:
        if flag:
            if rank == 0:
                print(json.dumps({name: fn()}), flush=True)
            return

    prob, prm = workload(args.chunks)
    intr = prob.intr
    lists = [c.tolist() for c in prob.chunks]
    cids = list(range(len(lists)))
    all_ids = list(range(prob.n_frames))
    precision = bf.BF_PREC_FP32 if args.precision == "fp32" else bf.BF_PREC_MIXED
    common = {k: prm[k] for k in ("n_gn", "n_pcg", "w_sparse", "w_dense", "w_photo", "w_geo")}
    if args.persistent and args.tile_px == -1:
        args.tile_px = PERSISTENT_TILE_PX
    params = bf.default_params(precision=precision, use_graph=0 if args.no_graph else 1, tile_px=args.tile_px,
                               pcg_variant=args.pcg_variant, persistent=1 if args.persistent else 0,
                               dense_tc=args.dense_tc, **common)
    storage = STORAGE_CODES[args.storage](bf)
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], device=local_rank,
                     stream=stream.cuda_stream, max_frames_hint=prob.n_frames, storage=storage)
    depth_d = torch.from_numpy(prob.depth).to(dev)
    lum_d = torch.from_numpy(prob.lum).to(dev)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, torch.from_numpy(prob.p_i).to(dev),
                                  torch.from_numpy(prob.p_j).to(dev))
    torch.cuda.synchronize(dev)
    gn_per_step = prm["n_gn"] * len(lists)

    def step(p=params):
        ctx.add_frames(0, depth_d, lum_d)
        return ctx.solve_local_batch(cids, lists, p)

    def timed(fn, k, profile=False):
        times = []
        if profile:
            ctx.reset_profile()
            ctx.set_profiling(True)
        out = None
        for _ in range(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        prof = None
        if profile:
            prof = ctx.profile()
            ctx.set_profiling(False)
        return times, out, prof

    t_w = time.perf_counter()
    for _ in range(args.warmup):
        stats = step()
    torch.cuda.synchronize(dev)
    warm_steps = args.warmup
    # then untimed steps until WARMUP_MIN_S has passed (the first runs after an idle period run slow)
    while not args.profile_run and time.perf_counter() - t_w < WARMUP_MIN_S:
        stats = step()
        warm_steps += 1
    torch.cuda.synchronize(dev)
    t_w = time.perf_counter() - t_w
    clocks = None if args.profile_run else Clocks(local_rank)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
    ctx.reset_profile()
    times, stats, _ = timed(step, args.steps)
    launches = ctx.profile()["launches"]
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(sum(times), dist)
    value = job_rate(gn_per_step, args.steps, world, total_ms)
    if args.profile_run:
        if rank == 0:
            print(json.dumps({"profile_run": True, "value": value, "ms_per_step": total_ms / args.steps}))
        return

    # per-kernel device times: a pass kernel by kernel with CUDA events around every launch on the
    # context's stream (the graph replay above carries no events); same decomposition as the graph
    prof_params = bf.default_params(precision=precision, use_graph=0, tile_px=args.tile_px,
                                    pcg_variant=args.pcg_variant, dense_tc=args.dense_tc, **common)
    _, _, prof = timed(lambda: step(prof_params), 2, profile=True)
    tuned = ctx.tuned_tile_px() if args.tile_px == bf.BF_TILE_AUTOTUNE else args.tile_px
    HW = intr["W"] * intr["H"]
    n_dp = 2 * sum(st["n_dense_pairs"] for st in stats)
    dense = prof["kernels"]["dense"]
    dense_ms = dense["ms"] / max(dense["count"], 1)
    units = n_dp * HW
    alg_bytes = dense_bytes_per_px(args.storage) * units
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "of measured (MEASURED_PEAKS.json hbm_gbs: copy bandwidth)"
    if hbm_peak is None:
        hbm_peak, peak_src = 6400.0, "of fallback (6.4 TB/s)"
    achieved = alg_bytes / (dense_ms / 1000.0) / 1e9
    flops = DENSE_FLOPS_PER_PX * units
    achieved_tf = flops / (dense_ms / 1000.0) / 1e12
    traffic = DENSE_TRAFFIC_BYTES_CHUNKS if (args.storage == "fp32" and args.tile_px == bf.BF_TILE_AUTOTUNE and
                                             args.chunks == 256) else None
    tot = sum(v["ms"] for v in prof["kernels"].values())
    kernel_share = {k: round(v["ms"] / max(tot, 1e-9), 4) for k, v in prof["kernels"].items() if v["count"]}
    lat_ms = [t for t in times]  # every chunk of a step completes with its batch: its latency is the step
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(prob, prm, args.storage, args.precision, cuda_graph=not args.no_graph,
                                      directed_dense_pairs=n_dp, tile_px=tuned, warmup_steps_run=warm_steps,
                                      warmup_s=round(t_w, 3), warmup_min_s=WARMUP_MIN_S,
                                      parallelism=f"replicas x{world}"),
            "gpu_launches": launches,
            "chunk_latency": {"batched_p50_ms": quantile(lat_ms, 0.5), "batched_p99_ms": quantile(lat_ms, 0.99),
                              "note": "batched: every chunk of a step completes with its batch (call -> results "
                                      "on the host), so its latency is the step time; quantiles over the steps"},
            "roofline": {"bound": "hbm", "kernel": "k_dense (tiled, accumulate + final energy launches)",
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": traffic, "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "bytes_per_directed_px": dense_bytes_per_px(args.storage), "directed_px_per_launch": units,
                         "avg_launch_ms": dense_ms, "launches_timed": dense["count"],
                         "note": "achieved = algorithmic bytes (source D, n, I; target D, n nearest; I, grad I "
                                 "bilinear) per launch / CUDA-event launch time; traffic = ncu DRAM bytes per launch"},
            "roofline_fp32_view": {"bound": "alu", "achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                   "frac": achieved_tf / FP32_PEAK_TFLOPS, "flops_per_directed_px": DENSE_FLOPS_PER_PX,
                                   "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 flop x 2.032 GHz"},
            "kernel_time_share": kernel_share,
            "energy": {"initial_sum": sum(st["energy"][0] for st in stats),
                       "final_sum": sum(st["energy"][-1] for st in stats)}}
    if clk:
        line["clocks"] = clk

    if not args.no_extras and rank == 0:
        line["e2e"] = chunk_e2e_leg(bf, torch, ctx, prob, stream, cids, lists, params, all_ids, timed,
                                    max(3, args.steps // 2), storage=storage)
        # restore the device-resident correspondences
        ctx.clear_correspondences()
        ctx.add_correspondences_batch(prob.pairs, prob.corr_off, torch.from_numpy(prob.p_i).to(dev),
                                      torch.from_numpy(prob.p_j).to(dev))
        line["plain_fp32"] = chunk_plain_leg(bf, torch, ctx, dev, prob, depth_d, lum_d, cids, lists, common,
                                             gn_per_step, stream)
        line["persistent"] = chunk_persistent_leg(bf, torch, ctx, depth_d, lum_d, cids, lists, common, gn_per_step,
                                                  stats, stream)
        line["compensated_sums"] = chunk_compensated_leg(bf, torch, ctx, depth_d, lum_d, cids, lists, common,
                                                         gn_per_step, stats, stream, tuned)
        line["tensor_core_sums"] = {
            f"dense_tc{tc}": chunk_compensated_leg(bf, torch, ctx, depth_d, lum_d, cids, lists, common, gn_per_step,
                                                   stats, stream, tuned, dense_tc=tc) for tc in (3, 1)}
        ctx.close()
        line["bf16_storage"] = chunk_batch_leg(bf, torch, dev, stream, prob=prob, storage="bf16")
        line["global300"] = global300_leg(bf, torch, dev, stream, args)
        line["large_global"] = large_global_leg(bf, torch, dev, stream)
        line["serving"] = serving_leg(bf, torch, dev, chunk_prob=prob, seconds=args.serving_seconds)
        line["next_rows"] = next_rows_leg(bf, torch, dev, stream)
        line["chunk11_latency"] = chunk_latency(bf, torch, dev)
        line["cpu_baseline"] = cpu_baseline_leg(prob, prm)
    else:
        ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def chunk_e2e_leg(bf, torch, ctx, prob, stream, cids, lists, params, all_ids, timed, steps, storage=None):
    """The batch end to end through the C ABI from pinned host buffers: every step uploads the raw
    frames and the correspondences, solves, and reads every frame's pose back (one context, step
    after step, CUDA events around each step).  two_contexts: the same steps on two contexts and
    streams driven by two host threads, so that one step's uploads overlap the other's solve (host
    clock around all steps of both); the upload's 1.16 GB through L2 slows the concurrent solve
    about as much as the overlap saves."""
    import threading
    depth_h = torch.from_numpy(prob.depth).pin_memory()
    lum_h = torch.from_numpy(prob.lum).pin_memory()
    pi_h = torch.from_numpy(prob.p_i).pin_memory()
    pj_h = torch.from_numpy(prob.p_j).pin_memory()

    def step_e2e(c=ctx):
        c.add_frames(0, depth_h, lum_h)
        c.clear_correspondences()
        c.add_correspondences_batch(prob.pairs, prob.corr_off, pi_h, pj_h)
        s = c.solve_local_batch(cids, lists, params)
        c.get_poses(all_ids)
        return s

    for _ in range(2):
        step_e2e()
    te, _, _ = timed(step_e2e, steps)
    h2d = prob.depth.nbytes + prob.lum.nbytes + prob.p_i.nbytes + prob.p_j.nbytes + prob.pairs.nbytes + \
        prob.corr_off.nbytes
    d2h = prob.n_frames * 16 * 8
    gn = params.n_gn * len(lists)
    serial = {"value": gn / (statistics.mean(te) / 1000.0), "ms_per_step": statistics.mean(te)}
    # two contexts, two streams, two host threads
    intr = prob.intr
    stream2 = torch.cuda.Stream(stream.device)
    ctx2 = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], device=stream.device.index,
                      stream=stream2.cuda_stream, max_frames_hint=prob.n_frames,
                      storage=storage if storage is not None else bf.BF_STORE_FP32)
    for _ in range(2):
        step_e2e(ctx2)
    errors = []

    def run(c, k):
        try:
            for _ in range(k):
                step_e2e(c)
        except Exception as e:  # reported below
            errors.append(e)

    torch.cuda.synchronize(stream.device)
    t0 = time.perf_counter()
    threads = [threading.Thread(target=run, args=(c, steps)) for c in (ctx, ctx2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    torch.cuda.synchronize(stream.device)
    wall = time.perf_counter() - t0
    ctx2.close()
    if errors:
        raise errors[0]
    return {"value": serial["value"], "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": serial["ms_per_step"],
            "two_contexts": {"value": 2 * steps * gn / wall, "ms_per_step": 1000.0 * wall / (2 * steps)},
            "note": "pinned host depth, luminance and correspondences uploaded, poses of all frames read back, "
                    "every step; per-chunk statistics also come back each step.  two_contexts: two contexts on "
                    "two streams, one host thread each, whole steps in parallel, host clock around all 2 x steps"}


def chunk_plain_leg(bf, torch, ctx, dev, prob, depth_d, lum_d, cids, lists, common, gn_per_step, stream, steps=2):
    """The plain path: one FP32 solve per chunk, kernel by kernel (no batching, no graph); chunk-solve
    latency = call -> poses on the host."""
    pp = bf.default_params(precision=bf.BF_PREC_FP32, use_graph=0, **common)
    lat, tot, done = [], [], []
    for rep in range(steps + 1):
        ctx.add_frames(0, depth_d, lum_d)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for cid, lst in zip(cids, lists):
            t1 = time.perf_counter()
            ctx.solve_local(cid, lst, pp)
            ctx.get_poses(lst)
            if rep:
                lat.append(1000.0 * (time.perf_counter() - t1))
                done.append(1000.0 * (time.perf_counter() - t0))
        if rep:
            tot.append(time.perf_counter() - t0)
    return {"value": gn_per_step / statistics.mean(tot), "unit": UNIT, "ms_per_step": 1000.0 * statistics.mean(tot),
            "solves_per_s": len(lists) / statistics.mean(tot), "chunk_latency_p50_ms": quantile(lat, 0.5),
            "chunk_latency_p99_ms": quantile(lat, 0.99),
            "all_at_once": {"p50_ms": quantile(done, 0.5), "p99_ms": quantile(done, 0.99),
                            "note": "the step's chunks all requested at its start and served one call after "
                                    "another: each chunk's completion time from the start (compare with "
                                    "chunk_latency.batched_*)"},
            "precision": "fp32", "cuda_graph": False,
            "note": "same chunks, one bf_solve_local per chunk (host clock around each call)"}


# tiles of half a 320x240 frame for the persistent launch (the fastest of 19200 / 38400 / 76800 there)
PERSISTENT_TILE_PX = 38400


def chunk_persistent_leg(bf, torch, ctx, depth_d, lum_d, cids, lists, common, gn_per_step, ref_stats, stream,
                         steps=3):
    """The same batch as ONE persistent cooperative launch over a device work queue."""
    pk = bf.default_params(precision=bf.BF_PREC_FP32, use_graph=1, tile_px=PERSISTENT_TILE_PX, persistent=1, **common)

    def run():
        ctx.add_frames(0, depth_d, lum_d)
        return ctx.solve_local_batch(cids, lists, pk)

    run()
    ts = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sk = run()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return {"value": gn_per_step / (statistics.mean(ts) / 1000.0), "unit": UNIT, "ms_per_step": statistics.mean(ts),
            "launches_per_solve": 1, "tile_px": PERSISTENT_TILE_PX, "cuda_graph": True,
            "final_energy_max_rel_diff_vs_launch_sequence": max(
                abs(a["energy"][-1] - b["energy"][-1]) / abs(b["energy"][-1]) for a, b in zip(sk, ref_stats))}


def chunk_compensated_leg(bf, torch, ctx, depth_d, lum_d, cids, lists, common, gn_per_step, ref_stats, stream, tile,
                          steps=3, **variant):
    """The same batch with another form of the dense sums (same tiles): compensated (Kahan)
    per-thread sums by default, or the variant given (dense_tc = 1 or 3: tensor-core sums)."""
    variant = variant or {"compensated": 1}
    pc = bf.default_params(precision=bf.BF_PREC_FP32, use_graph=1, tile_px=tile, **variant, **common)

    def run(p):
        ctx.add_frames(0, depth_d, lum_d)
        return ctx.solve_local_batch(cids, lists, p)

    run(pc)
    ts = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sc = run(pc)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ctx.reset_profile()
    ctx.set_profiling(True)
    run(bf.default_params(precision=bf.BF_PREC_FP32, use_graph=0, tile_px=tile, **variant, **common))
    dense = ctx.profile()["kernels"]["dense"]
    ctx.set_profiling(False)
    return {"value": gn_per_step / (statistics.mean(ts) / 1000.0), "unit": UNIT, "ms_per_step": statistics.mean(ts),
            "tile_px": tile, "dense_avg_launch_ms": dense["ms"] / max(dense["count"], 1),
            "final_energy_max_rel_diff_vs_fp32_fma_sums": max(
                abs(a["energy"][-1] - b["energy"][-1]) / abs(b["energy"][-1]) for a, b in zip(sc, ref_stats))}


def global300_leg(bf, torch, dev, stream, args, steps=10, warmup=3):
    """The 300-keyframe 80x60 global solve (8 GN x 20 PCG, mixed precision, CUDA graph; its frames
    fit in L2): GN iterations/s, end to end from host buffers, the plain FP32 path, BF16 storage,
    the dense kernel's FP32 and algorithmic-byte rates, the matrix-free sparse term."""
    import synth
    prob = synth.cfg2()
    prm = prob.solve
    intr = prob.intr
    n = prob.n_frames
    ids = list(range(n))
    common = {k: prm[k] for k in ("n_gn", "n_pcg", "w_sparse", "w_dense", "w_photo", "w_geo")}
    params = bf.default_params(precision=bf.BF_PREC_MIXED, use_graph=1, tile_px=0, **common)
    prof_params = bf.default_params(precision=bf.BF_PREC_MIXED, use_graph=0, tile_px=0, **common)
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], stream=stream.cuda_stream,
                     max_frames_hint=n)
    depth_d = torch.from_numpy(prob.depth).to(dev)
    lum_d = torch.from_numpy(prob.lum).to(dev)
    pi_d = torch.from_numpy(prob.p_i).to(dev)
    pj_d = torch.from_numpy(prob.p_j).to(dev)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, pi_d, pj_d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2

    def step(p=params):
        ctx.add_frames(0, depth_d, lum_d, init_pose=prob.init)
        return ctx.solve_global(ids, p)

    def timed(fn, k, profile=False):
        times = []
        if profile:
            ctx.reset_profile()
            ctx.set_profiling(True)
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        prof = None
        if profile:
            prof = ctx.profile()
            ctx.set_profiling(False)
        return times, out, prof

    t_w = time.perf_counter()
    for _ in range(warmup):
        step()
    while time.perf_counter() - t_w < WARMUP_MIN_S:
        step()
    torch.cuda.synchronize(dev)
    clocks = Clocks(dev.index if dev.index is not None else 0)
    clocks.start()
    times, st, _ = timed(step, steps)
    clk = clocks.stop()
    _, _, prof = timed(lambda: step(prof_params), 3, profile=True)
    n_gn = prm["n_gn"]
    n_dp = 2 * st["n_dense_pairs"]
    HW = intr["W"] * intr["H"]
    dense = prof["kernels"]["dense"]
    dense_ms = dense["ms"] / max(dense["count"], 1)
    units = n_dp * HW
    out = {"workload": prob.name, "keyframes": n, "resolution": f"{intr['W']}x{intr['H']}",
           "pairs": int(len(prob.pairs)), "dense_pairs": st["n_dense_pairs"], "correspondences": prob.n_corr,
           "n_gn": n_gn, "n_pcg": prm["n_pcg"], "precision": "mixed", "cuda_graph": True,
           "value": n_gn / (statistics.mean(times) / 1000.0), "unit": UNIT, "ms_per_step": statistics.mean(times),
           "l2": "256 MB buffer written between timed steps (inputs < L2)", "clocks": clk,
           "initial_energy": st["energy"][0], "final_energy": st["energy"][-1],
           "dense_kernel": {"kernel": "k_dense_staged", "avg_launch_ms": dense_ms, "directed_px_per_launch": units,
                            "fp32_TFLOPs": DENSE_FLOPS_PER_PX * units / (dense_ms / 1000.0) / 1e12,
                            "fp32_frac": DENSE_FLOPS_PER_PX * units / (dense_ms / 1000.0) / 1e12 / FP32_PEAK_TFLOPS,
                            "algorithmic_GBps": DENSE_BYTES_PER_PX * units / (dense_ms / 1000.0) / 1e9,
                            "traffic": DENSE_TRAFFIC_BYTES,
                            "note": "frames L2-resident: DRAM traffic is the unique frame bytes"},
           "kernel_time_share": {k: round(v["ms"] / max(sum(x["ms"] for x in prof["kernels"].values()), 1e-9), 4)
                                 for k, v in prof["kernels"].items() if v["count"]}}
    # end to end from pinned host buffers
    depth_h = torch.from_numpy(prob.depth).pin_memory()
    lum_h = torch.from_numpy(prob.lum).pin_memory()
    pi_h = torch.from_numpy(prob.p_i).pin_memory()
    pj_h = torch.from_numpy(prob.p_j).pin_memory()

    def step_e2e():
        ctx.add_frames(0, depth_h, lum_h, init_pose=prob.init)
        ctx.clear_correspondences()
        ctx.add_correspondences_batch(prob.pairs, prob.corr_off, pi_h, pj_h)
        s = ctx.solve_global(ids, params)
        ctx.get_poses(ids)
        return s

    for _ in range(2):
        step_e2e()
    te, _, _ = timed(step_e2e, 5)
    out["e2e"] = {"value": n_gn / (statistics.mean(te) / 1000.0), "unit": UNIT, "ms_per_step": statistics.mean(te),
                  "h2d_bytes_per_step": int(prob.depth.nbytes + prob.lum.nbytes + 2 * 16 * prob.n_corr +
                                            prob.init.nbytes), "d2h_bytes_per_step": n * 16 * 8 + n * 12 * 8}
    ctx.clear_correspondences()
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, pi_d, pj_d)
    plain = bf.default_params(precision=bf.BF_PREC_FP32, **common)
    for _ in range(2):
        step(plain)
    tp, stp, _ = timed(lambda: step(plain), 5)
    out["plain_fp32"] = {"value": n_gn / (statistics.mean(tp) / 1000.0), "unit": UNIT,
                         "ms_per_step": statistics.mean(tp), "final_energy": stp["energy"][-1]}
    out["sparse_term"] = sparse_term_leg(bf, step, timed, prm, bf.BF_PREC_MIXED, 5)
    ctx.close()
    out["bf16_storage"] = storage_leg(bf, torch, dev, stream, prob, params, prof_params, "bf16")
    return out


def sparse_term_leg(bf, step, timed, prm, precision, steps):
    """Global solve with the sparse term as assembled blocks vs matrix-free, grid-cooperative PCG."""
    out = {"pcg_kernel": "k_pcg_coop (grid-cooperative)", "n_pcg": prm["n_pcg"]}
    for name, mode in (("blocks", bf.BF_SPARSE_BLOCKS), ("matfree", bf.BF_SPARSE_MATFREE)):
        kw = dict(n_gn=prm["n_gn"], n_pcg=prm["n_pcg"], w_sparse=prm["w_sparse"], w_dense=prm["w_dense"],
                  w_photo=prm["w_photo"], w_geo=prm["w_geo"], precision=precision, pcg_variant=bf.BF_PCG_GRID,
                  sparse_mode=mode)
        pg = bf.default_params(use_graph=1, **kw)
        pp = bf.default_params(use_graph=0, **kw)
        for _ in range(2):
            step(pg)
        tt, st, _ = timed(lambda: step(pg), steps)
        _, _, prof = timed(lambda: step(pp), 2, profile=True)
        k = prof["kernels"]
        per_solve = {n: round(v["ms"] / 2, 4) for n, v in k.items() if v["count"]}
        out[name] = {"value": prm["n_gn"] / (statistics.mean(tt) / 1000.0), "unit": UNIT,
                     "ms_per_step": statistics.mean(tt), "final_energy": st["energy"][-1],
                     "pcg_ms_per_launch": k["pcg"]["ms"] / max(k["pcg"]["count"], 1),
                     "kernel_ms_per_solve": per_solve}
    out["pcg_iteration_us"] = {n: 1000.0 * out[n]["pcg_ms_per_launch"] / prm["n_pcg"] for n in ("blocks", "matfree")}
    return out


def storage_leg(bf, torch, dev, stream, prob, params, prof_params, kind, steps=5):
    """The timed global solve with frames held in 16-bit storage (same poses, pairs, parameters)."""
    intr = prob.intr
    n = prob.n_frames
    ids = list(range(n))
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], stream=stream.cuda_stream,
                     max_frames_hint=n, storage=STORAGE_CODES[kind](bf))
    depth_d = torch.from_numpy(prob.depth).to(dev)
    lum_d = torch.from_numpy(prob.lum).to(dev)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, torch.from_numpy(prob.p_i).to(dev),
                                  torch.from_numpy(prob.p_j).to(dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(p):
        ctx.add_frames(0, depth_d, lum_d, init_pose=prob.init)
        return ctx.solve_global(ids, p)

    for _ in range(3):
        step(params)
    ts = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step(params)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ctx.reset_profile()
    ctx.set_profiling(True)
    step(prof_params)
    dense = ctx.profile()["kernels"]["dense"]
    ctx.set_profiling(False)
    ctx.close()
    n_gn = params.n_gn
    dense_ms = dense["ms"] / max(dense["count"], 1)
    units = 2 * st["n_dense_pairs"] * intr["W"] * intr["H"]
    return {"storage": kind, "value": n_gn / (statistics.mean(ts) / 1000.0), "unit": UNIT,
            "ms_per_step": statistics.mean(ts), "final_energy": st["energy"][-1],
            "dense_avg_launch_ms": dense_ms,
            "dense_algorithmic_GBps": dense_bytes_per_px(kind) * units / (dense_ms / 1000.0) / 1e9,
            "frame_bytes": int(n * intr["W"] * intr["H"] * 16)}



def next_rows_leg(bf, torch, dev, stream):
    """The steps around the solver on the 300-keyframe workload (Sec. 4.1.1, 4.4.1, 5).

    verify: every pair, both directions, at the ground-truth relative poses (one launch);
    keypoints: every pair's matches through the key-point and surface-area filters (one launch);
    pruning: the global solve with r_max pruning at 0.05 m (the workload has 5 % random outliers,
    so pairs are pruned until the round cap); tsdf: the 300 frames integrated then de-integrated
    (1 cm voxels)."""
    import numpy as np
    import synth
    prob = synth.cfg2()
    prm = prob.solve
    intr = prob.intr
    n = prob.n_frames
    ids = list(range(n))
    out = {}

    def ctx_new():
        c = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], stream=stream.cuda_stream,
                       max_frames_hint=n)
        c.add_frames(0, torch.from_numpy(prob.depth).to(dev), torch.from_numpy(prob.lum).to(dev),
                     init_pose=prob.gt)
        return c

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            r = fn()
        torch.cuda.synchronize(dev)
        return (time.perf_counter() - t0) / reps, r

    ctx = ctx_new()
    pairs = np.asarray(prob.pairs, dtype=np.int32)
    rel = np.stack([np.linalg.inv(prob.gt[j]) @ prob.gt[i] for i, j in pairs])
    HW = intr["W"] * intr["H"]
    t, res = timed(lambda: ctx.verify_pairs(pairs, rel), 5)
    out["verify"] = {"pairs": len(pairs), "ms_per_call": 1e3 * t, "pairs_per_s": len(pairs) / t,
                     "valid_pairs": int(sum(r["valid"] for r in res)),
                     "algorithmic_GBps": 2 * len(pairs) * HW * 36 / t / 1e9,
                     "note": "host call incl. record upload and result read-back; 36 B per directed pixel"}
    t, (keep, T, status) = timed(lambda: ctx.filter_keypoints(prob.corr_off.astype(np.int32), prob.p_i, prob.p_j),
                                 3)
    out["keypoints"] = {"pairs": len(pairs), "matches": int(prob.corr_off[-1]), "ms_per_call": 1e3 * t,
                        "pairs_per_s": len(pairs) / t, "kept_pairs": int((status == 0).sum()),
                        "kept_matches": int(keep.sum()), "arithmetic": "FP64, one warp per pair"}
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, prob.p_i, prob.p_j)
    ctx.add_frames(0, torch.from_numpy(prob.depth).to(dev), torch.from_numpy(prob.lum).to(dev), init_pose=prob.init)
    pp = bf.default_params(n_gn=prm["n_gn"], n_pcg=prm["n_pcg"], w_sparse=prm["w_sparse"], w_dense=prm["w_dense"],
                           w_photo=prm["w_photo"], w_geo=prm["w_geo"], prune_rmax=0.05, prune_rounds=8)
    t0 = time.perf_counter()
    st = ctx.solve_global(ids, pp)
    t = time.perf_counter() - t0
    out["pruning"] = {"solves": st["solves"], "pruned_pairs": st["n_pruned"], "invalid_frames": st["n_invalid"],
                      "ms_total": 1e3 * t, "final_r_max": st["r_max"], "gn_iterations_per_s": st["solves"] * prm["n_gn"] / t}
    ctx.close()
    ctx = ctx_new()
    ctx.tsdf_init(voxel_size=0.01, table_log2=21, max_blocks=1 << 17)

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(n):
        ctx.tsdf_integrate(k)  # at the frame's world pose
    t_in = time.perf_counter() - t0
    t0 = time.perf_counter()
    for k in range(n):
        ctx.tsdf_deintegrate(k)
    t_de = time.perf_counter() - t0
    blocks = len(ctx.tsdf_export())
    out["tsdf"] = {"frames": n, "voxel_m": 0.01, "blocks": blocks, "integrate_ms_per_frame": 1e3 * t_in / n,
                   "deintegrate_ms_per_frame": 1e3 * t_de / n, "frames_per_s": n / t_in,
                   "note": "synchronous calls (status read back per frame)"}
    ctx.close()
    return out


def large_global_leg(bf, torch, dev, stream, steps=3, warmup=1):
    """Large global mixed-precision solve: 2000 keyframes at 160x120 in BF16 frame storage, 25k
    pairs, 2.5M correspondences (10 % outliers), 10 GN x 30 PCG, CUDA graph.  The frames
    (2000 x 19200 px x 18 B = 0.69 GB) exceed L2, so the dense kernel streams them from HBM."""
    import synth
    t_gen = time.perf_counter()
    prob = synth.cfg5()
    t_gen = time.perf_counter() - t_gen
    intr = prob.intr
    n = prob.n_frames
    ids = list(range(n))
    prm = prob.solve
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], stream=stream.cuda_stream,
                     max_frames_hint=n, storage=bf.BF_STORE_BF16)
    depth_d = torch.from_numpy(prob.depth).to(dev)
    lum_d = torch.from_numpy(prob.lum).to(dev)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, torch.from_numpy(prob.p_i).to(dev),
                                  torch.from_numpy(prob.p_j).to(dev))
    common = {k: prm[k] for k in ("n_gn", "n_pcg", "w_sparse", "w_dense", "w_photo", "w_geo")}
    # the dense work decomposition from the library's autotuner (timed once, in the warm-up)
    p = bf.default_params(precision=bf.BF_PREC_MIXED, use_graph=1, tile_px=bf.BF_TILE_AUTOTUNE, **common)

    def step(pp=p):
        ctx.add_frames(0, depth_d, lum_d, init_pose=prob.init)
        return ctx.solve_global(ids, pp)

    for _ in range(warmup):
        step()
    ts = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ctx.reset_profile()
    ctx.set_profiling(True)
    step(bf.default_params(precision=bf.BF_PREC_MIXED, use_graph=0, tile_px=bf.BF_TILE_AUTOTUNE, **common))
    prof = ctx.profile()
    tuned = ctx.tuned_tile_px()
    ctx.set_profiling(False)
    ctx.close()
    dense = prof["kernels"]["dense"]
    dense_ms = dense["ms"] / max(dense["count"], 1)
    HW = intr["W"] * intr["H"]
    units = 2 * st["n_dense_pairs"] * HW
    tot = sum(v["ms"] for v in prof["kernels"].values())
    return {"workload": prob.name, "keyframes": n, "resolution": f"{intr['W']}x{intr['H']}", "storage": "bf16",
            "pairs": int(len(prob.pairs)), "dense_pairs": st["n_dense_pairs"], "correspondences": prob.n_corr,
            "n_gn": prm["n_gn"], "n_pcg": prm["n_pcg"], "precision": "mixed", "generation_s": t_gen,
            "value": prm["n_gn"] / (statistics.mean(ts) / 1000.0), "unit": UNIT, "ms_per_step": statistics.mean(ts),
            "initial_energy": st["energy"][0], "final_energy": st["energy"][-1], "tile_px_autotuned": tuned,
            "dense_kernel": {"avg_launch_ms": dense_ms, "directed_px_per_launch": units,
                             "algorithmic_GBps": DENSE_BYTES_PER_PX_16 * units / (dense_ms / 1000.0) / 1e9,
                             "frame_bytes": n * HW * 18},
            "kernel_time_share": {k: round(v["ms"] / max(tot, 1e-9), 4) for k, v in prof["kernels"].items()
                                  if v["count"]}}

def chunk_batch_leg(bf, torch, dev, stream, steps=3, warmup=1, n_chunks=256, prob=None, storage="fp32"):
    """Batched chunk solves: 256 chunks of U{3..11} frames at 320x240, 6 GN x 10 PCG.

    batched: all chunks in one launch sequence (one problem per chunk), replayed as a CUDA graph;
    plain: one solve per chunk, kernel by kernel, no graph (FP32 storage only); FP32 arithmetic
    with pairwise sums in both.  Each step re-runs frame preprocessing from device-resident raw frames.  Chunk-solve
    latency: call -> poses on the host; in the batched mode every chunk completes with its batch."""
    import synth
    prob = prob or synth.cfg3(n_chunks=n_chunks)
    intr = prob.intr
    prm = prob.solve
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], stream=stream.cuda_stream,
                     max_frames_hint=prob.n_frames, storage=STORAGE_CODES[storage](bf))
    depth_d = torch.from_numpy(prob.depth).to(dev)
    lum_d = torch.from_numpy(prob.lum).to(dev)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, torch.from_numpy(prob.p_i).to(dev),
                                  torch.from_numpy(prob.p_j).to(dev))
    ids = list(range(len(prob.chunks)))
    lists = [c.tolist() for c in prob.chunks]
    common = {k: prm[k] for k in ("n_gn", "n_pcg", "w_sparse", "w_dense", "w_photo", "w_geo")}
    # chunk solves in FP32 arithmetic with pairwise (tree) sums in both modes: on these problems it
    # meets the oracle tolerances as well as the FP64-merged mode, so the comparison is at equal
    # accuracy and isolates batching + graph replay
    pb = bf.default_params(precision=bf.BF_PREC_FP32, use_graph=1, tile_px=bf._lib.BF_TILE_AUTOTUNE, **common)
    pp = bf.default_params(precision=bf.BF_PREC_FP32, use_graph=0, **common)
    gn_per_step = prm["n_gn"] * len(lists)

    def run(fn, k):
        ts = []
        for _ in range(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts, out

    def batched():
        ctx.add_frames(0, depth_d, lum_d)
        return ctx.solve_local_batch(ids, lists, pb)

    lat = []

    def plain():
        ctx.add_frames(0, depth_d, lum_d)
        torch.cuda.synchronize(dev)
        out = []
        for cid, lst in zip(ids, lists):
            t0 = time.perf_counter()
            out.append(ctx.solve_local(cid, lst, pp))
            ctx.get_poses(lst)
            lat.append(1000.0 * (time.perf_counter() - t0))
        return out

    run(batched, warmup)
    tb, sb = run(batched, steps)

    # the same batch as ONE persistent launch (device work queue over tiles, segments and solves)
    pk = bf.default_params(precision=bf.BF_PREC_FP32, use_graph=1, tile_px=PERSISTENT_TILE_PX, persistent=1, **common)

    def persistent():
        ctx.add_frames(0, depth_d, lum_d)
        return ctx.solve_local_batch(ids, lists, pk)

    run(persistent, warmup)
    tk, sk = run(persistent, steps)
    ctx.reset_profile()
    ctx.set_profiling(True)
    persistent_kernel = None
    ctx.add_frames(0, depth_d, lum_d)
    ctx.solve_local_batch(ids, lists, bf.default_params(precision=bf.BF_PREC_FP32, use_graph=0, persistent=1,
                                                        tile_px=PERSISTENT_TILE_PX, **common))
    kp = ctx.profile()["kernels"]
    if kp["batch"]["count"]:
        persistent_kernel = {"launches": kp["batch"]["count"], "ms": kp["batch"]["ms"] / kp["batch"]["count"]}
    ctx.set_profiling(False)
    # dense kernel time in this workload (kernel by kernel, CUDA events around each launch)
    ctx.reset_profile()
    ctx.set_profiling(True)
    ctx.add_frames(0, depth_d, lum_d)
    ctx.solve_local_batch(ids, lists, bf.default_params(precision=bf.BF_PREC_FP32, use_graph=0,
                                                        tile_px=bf._lib.BF_TILE_AUTOTUNE, **common))
    tuned = ctx.tuned_tile_px()
    prof = ctx.profile()
    ctx.set_profiling(False)
    tp = None
    if storage == "fp32":
        run(plain, 1)
        lat.clear()
        tp, _ = run(plain, max(1, steps - 1))
        lat.sort()
    HW = intr["W"] * intr["H"]
    n_dp = 2 * sum(s["n_dense_pairs"] for s in sb)
    dense = prof["kernels"]["dense"]
    dense_ms = dense["ms"] / max(dense["count"], 1)
    alg_bytes = dense_bytes_per_px(storage) * n_dp * HW
    out = {"workload": prob.name, "storage": storage, "chunks": len(lists), "frames": prob.n_frames,
           "pairs": int(len(prob.pairs)),
           "directed_dense_pairs": n_dp, "correspondences": prob.n_corr, "n_gn": prm["n_gn"], "n_pcg": prm["n_pcg"],
           "batched": {"value": gn_per_step / (statistics.mean(tb) / 1000.0), "unit": UNIT,
                       "ms_per_step": statistics.mean(tb),
                       "solves_per_s": len(lists) / (statistics.mean(tb) / 1000.0),
                       "chunk_latency_p50_ms": statistics.mean(tb), "chunk_latency_p99_ms": max(tb),
                       "precision": "fp32", "cuda_graph": True,
                       "tile_px": {"autotuned": tuned, "meaning": "0 = target frame staged in shared memory"}},
           "persistent": {"value": gn_per_step / (statistics.mean(tk) / 1000.0), "unit": UNIT,
                          "ms_per_step": statistics.mean(tk), "solves_per_s": len(lists) / (statistics.mean(tk) / 1000.0),
                          "launches_per_solve": 1, "kernel": persistent_kernel, "cuda_graph": True,
                          "tile_px": PERSISTENT_TILE_PX,
                          "final_energy_max_rel_diff_vs_launch_sequence": max(
                              abs(a["energy"][-1] - b["energy"][-1]) / abs(b["energy"][-1]) for a, b in zip(sk, sb)),
                          "note": "tiles of tile_px pixels here, the autotuned size in the launch sequence; at equal "
                                  "tiles the two are bitwise equal (tests/test_gpu_persistent.py)"},
           "dense_kernel": {"avg_launch_ms": dense_ms, "launches": dense["count"],
                            "algorithmic_bytes_per_launch": alg_bytes,
                            "algorithmic_GBps": alg_bytes / (dense_ms / 1000.0) / 1e9,
                            "unique_frame_bytes": int(prob.n_frames * HW * (32 if storage == "fp32" else 16))}}
    if tp:
        out["plain_fp32"] = {"value": gn_per_step / (statistics.mean(tp) / 1000.0), "unit": UNIT,
                             "ms_per_step": statistics.mean(tp),
                             "solves_per_s": len(lists) / (statistics.mean(tp) / 1000.0),
                             "chunk_latency_p50_ms": lat[len(lat) // 2],
                             "chunk_latency_p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))]}
    ctx.close()
    return out


SERVING_HBM_BUDGET = 40 * 1024 ** 3


def _serve_session(cctx, gctx, arrivals, cparams, gparams, lib):
    """Submit every request at its arrival time to the serving loops; latency = submit ->
    completion, as the library measures it; the session ends at the last completion (submit time
    + latency), not when this thread has collected every result."""
    ct, gt = [], []
    t0 = time.perf_counter()
    for ta, kind, ids, cid in arrivals:
        while time.perf_counter() - t0 < ta:
            time.sleep(0.0002)
        if kind == "chunk":
            ct.append((time.perf_counter(), cctx.submit(ids, chunk_id=cid, params=cparams)))
        else:
            gt.append((time.perf_counter(), gctx.submit(ids, kind=lib.BF_REQ_GLOBAL, params=gparams)))
    cres = [(ts, cctx.wait(t)[1]["ms"]) for ts, t in ct]
    gres = [(ts, gctx.wait(t)[1]["ms"]) for ts, t in gt]
    end = max(ts + 1e-3 * ms for ts, ms in cres + gres)
    return [ms for _, ms in cres], [ms for _, ms in gres], end - t0


def _plain_session(cctx, gctx, arrivals, cparams, gparams):
    """The plain path: one host loop takes the requests in arrival order and calls
    bf_solve_local / bf_solve_global for each (synchronous: results on the host when the call
    returns); latency = arrival -> return, so a request that arrives while another is being
    solved waits for it."""
    clat, glat = [], []
    t0 = time.perf_counter()
    for ta, kind, ids, cid in arrivals:
        while time.perf_counter() - t0 < ta:
            time.sleep(0.0002)
        if kind == "chunk":
            cctx.solve_local(cid, ids, params=cparams)
            clat.append(1000.0 * (time.perf_counter() - t0 - ta))
        else:
            gctx.solve_global(ids, params=gparams)
            glat.append(1000.0 * (time.perf_counter() - t0 - ta))
    return clat, glat, time.perf_counter() - t0


def serving_leg(bf, torch, dev, chunk_prob=None, seconds=20.0, rate=30.0, seed=1604):
    """The serving stream: Poisson arrivals of chunk requests (320x240, 3-11 frames, 6 GN x 10 PCG)
    at `rate` per second for `seconds`, and with every 10th chunk a global request over the first k
    keyframes of a 2000-keyframe 80x60 loop (8 GN x 20 PCG), k growing linearly from 100 to 2000
    over the session (over 10 minutes at full length; a shorter session compresses the growth).
    served: the library's serving loops on two persistent contexts (chunks: 2 slots, continuous
    batching up to 16, high-priority streams, FP32 arithmetic; globals: 1 slot, low-priority
    stream, FP64-merged mixed precision, cluster PCG), admission by a 40 GB HBM budget per context, frames,
    correspondences and solve workspaces resident.  plain: the same arrivals served one request at
    a time, in arrival order, by synchronous calls of the plain FP32 path.  Then a chunk-only
    stream at 600 requests/s, both ways.  p50 / p99 per request kind and over all requests."""
    import synth
    chunk_prob = chunk_prob or synth.cfg3()
    t_gen = time.perf_counter()
    global_prob = synth.cfg4_global()
    t_gen = time.perf_counter() - t_gen
    rng = np.random.default_rng(seed)
    n_req = int(seconds * rate)
    t_arr = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    lists = [c.tolist() for c in chunk_prob.chunks]
    arrivals, ks = [], []
    for r in range(n_req):
        arrivals.append((float(t_arr[r]), "chunk", lists[r % len(lists)], r))
        if r % 10 == 9:
            k = int(round(100 + 1900 * r / max(1, n_req - 1)))
            ks.append(k)
            arrivals.append((float(t_arr[r]), "global", list(range(k)), 0))
    hi_rate, hi_n = 600.0, 1200
    h_arr = np.cumsum(rng.exponential(1.0 / hi_rate, size=hi_n))
    burst = [(float(h_arr[r]), "chunk", lists[r % len(lists)], 300000 + r) for r in range(hi_n)]
    ci, gi = chunk_prob.intr, global_prob.intr
    pc = {k: chunk_prob.solve[k] for k in ("n_gn", "n_pcg", "w_sparse", "w_dense", "w_photo", "w_geo")}
    pg = {k: global_prob.solve[k] for k in ("n_gn", "n_pcg", "w_sparse", "w_dense", "w_photo", "w_geo")}
    q = lambda v, f: float(v[min(len(v) - 1, int(f * len(v)))]) if v else None  # noqa: E731
    out = {"arrival_rate_per_s": rate, "seconds": seconds, "chunk_requests": n_req, "global_requests": len(ks),
           "global_keyframes": [ks[0], ks[-1]] if ks else None, "chunk_workload": chunk_prob.name,
           "global_workload": f"{global_prob.name}: {global_prob.n_frames} keyframes, {len(global_prob.pairs)} pairs, "
                              f"{global_prob.n_corr} correspondences (prefixes of k keyframes)",
           "global_generation_s": round(t_gen, 1), "hbm_budget_bytes_per_context": SERVING_HBM_BUDGET}
    for name in ("served", "plain_fp32"):
        served = name == "served"
        cctx = bf.Context(ci["W"], ci["H"], ci["fx"], ci["fy"], ci["cx"], ci["cy"], max_frames_hint=chunk_prob.n_frames,
                          hbm_budget_bytes=SERVING_HBM_BUDGET)
        cctx.add_frames(0, torch.from_numpy(chunk_prob.depth).to(dev), torch.from_numpy(chunk_prob.lum).to(dev))
        cctx.add_correspondences_batch(chunk_prob.pairs, chunk_prob.corr_off, torch.from_numpy(chunk_prob.p_i).to(dev),
                                       torch.from_numpy(chunk_prob.p_j).to(dev))
        gctx = bf.Context(gi["W"], gi["H"], gi["fx"], gi["fy"], gi["cx"], gi["cy"], max_frames_hint=global_prob.n_frames,
                          hbm_budget_bytes=SERVING_HBM_BUDGET)
        gctx.add_frames(0, global_prob.depth, global_prob.lum, init_pose=global_prob.init)
        gctx.add_correspondences_batch(global_prob.pairs, global_prob.corr_off, global_prob.p_i, global_prob.p_j)
        torch.cuda.synchronize(dev)
        cparams = bf.default_params(precision=bf.BF_PREC_FP32, **pc)
        # served globals run the 16-CTA cluster PCG, which leaves the other SMs to the chunk solves
        # running beside them (the grid-cooperative kernel AUTO picks for >= 1000 keyframes is faster
        # alone but holds every SM); the plain path, one request at a time, keeps AUTO
        gparams = (bf.default_params(precision=bf.BF_PREC_MIXED, pcg_variant=bf.BF_PCG_CLUSTER, **pg) if served
                   else bf.default_params(precision=bf.BF_PREC_FP32, **pg))
        if served:
            cctx.serve_start(n_slots=2, max_batch=16, max_queue=100000)
            gctx.serve_start(n_slots=1, max_batch=1, max_queue=100000)
            # warm-up (not timed): every slot allocates its workspace and pinned staging on first use
            warm = [cctx.submit(lists[k % len(lists)], chunk_id=100000 + k, params=cparams) for k in range(8)]
            for k in (100, 2000):
                gctx.wait(gctx.submit(list(range(k)), kind=bf._lib.BF_REQ_GLOBAL, params=gparams))
            for t in warm:
                cctx.wait(t)
            clat, glat, wall = _serve_session(cctx, gctx, arrivals, cparams, gparams, bf._lib)
            for t in [cctx.submit(lists[k % len(lists)], chunk_id=200000 + k, params=cparams) for k in range(8)]:
                cctx.wait(t)
            hlat, _, hwall = _serve_session(cctx, None, burst, cparams, None, bf._lib)
            cctx.serve_stop()
            gctx.serve_stop()
        else:
            for k in range(8):
                cctx.solve_local(100000 + k, lists[k % len(lists)], params=cparams)
            for k in (100, 2000):
                gctx.solve_global(list(range(k)), params=gparams)
            clat, glat, wall = _plain_session(cctx, gctx, arrivals, cparams, gparams)
            hlat, _, hwall = _plain_session(cctx, None, burst, cparams, None)
        gctx.close()
        cctx.close()
        allat = sorted(clat + glat)
        clat.sort()
        glat.sort()
        hlat.sort()
        out[name] = {"chunk_p50_ms": q(clat, 0.5), "chunk_p99_ms": q(clat, 0.99), "global_p50_ms": q(glat, 0.5),
                     "global_p99_ms": q(glat, 0.99), "all_p50_ms": q(allat, 0.5), "all_p99_ms": q(allat, 0.99),
                     "global_max_ms": glat[-1] if glat else None, "solves_per_s": len(allat) / wall, "wall_s": wall,
                     "chunk_only_600_per_s": {"p50_ms": q(hlat, 0.5), "p99_ms": q(hlat, 0.99),
                                              "solves_per_s": len(hlat) / hwall, "requests": len(hlat)},
                     "precision": {"chunk": "fp32", "global": "mixed" if served else "fp32"},
                     "global_pcg": "cluster" if served else "auto",
                     "form": ("serving loops: chunks 2 slots x batches of up to 16 on high-priority streams, globals "
                              "1 slot on a low-priority stream" if served else
                              "one host loop, requests in arrival order, synchronous bf_solve_local / bf_solve_global")}
    return out


def chunk_latency(bf, torch, dev, reps=40):
    """Chunk-solve latency (call -> poses on the host) for single 11-frame 80x60 chunks."""
    import synth
    prob = synth.cfg1()
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                     stream=torch.cuda.current_stream(dev).cuda_stream or None)
    ctx.add_frames(0, prob.depth, prob.lum)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, prob.p_i, prob.p_j)
    ids = list(range(prob.n_frames))
    out = {"workload": prob.name, "n_gn": prob.solve["n_gn"], "n_pcg": prob.solve["n_pcg"], "reps": reps}
    # optimised: FP32 arithmetic (equal accuracy to the oracle on chunks) with the Gauss-Newton loop
    # replayed as a CUDA graph and the autotuned dense decomposition; plain: FP32, kernel by kernel
    for name, kw in (("optimised_fp32_graph", dict(precision=bf.BF_PREC_FP32, use_graph=1,
                                                   tile_px=bf._lib.BF_TILE_AUTOTUNE)),
                     ("mixed", dict(precision=bf.BF_PREC_MIXED)),
                     ("plain_fp32", dict(precision=bf.BF_PREC_FP32))):
        p = bf.default_params(**kw, **{k: v for k, v in prob.solve.items()})
        for _ in range(5):
            ctx.solve_local(0, ids, p)
        lat = []
        for _ in range(reps):
            t0 = time.perf_counter()
            ctx.solve_local(0, ids, p)
            ctx.get_poses(ids)
            lat.append(1000.0 * (time.perf_counter() - t0))
        lat.sort()
        out[name] = {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                     "solves_per_s": 1000.0 / statistics.mean(lat)}
    ctx.close()
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
