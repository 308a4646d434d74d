#!/usr/bin/env python
"""Benchmark of the global pose alignment solve (BundleFusion Sec. 4.2-4.4) on B300.

Workload (default): the global solve over 300 keyframes at 80x60 along a ~60 m loop of a
synthetic ring corridor, pairs with ground-truth overlap > 30 %, 64-256 correspondences
per pair (sigma 1 cm, 5 % outliers), dense weight 0.5, 8 Gauss-Newton x 20 PCG
iterations.  One step = the whole hot path once: frame preprocessing from device-resident
raw depth/luminance, pair-set construction, 8 linearisations (dense + sparse terms,
block reduction, assembly), 8 x 20 PCG iterations and pose updates, final energy and r_max.

Metric: Gauss-Newton iterations per second (whole job over all ranks).  Extra fields:
the plain FP32 one-solve-per-launch path on the same workload, chunk-solve latency
p50/p99 (single 11-frame 80x60 chunks, optimised vs plain path), the roofline of the
dominant kernel (dense term) and the FP64 oracle timed on the host cores.

Under torchrun (N > 1) every rank solves its own replica (the global solve does not
shard; chunk solves would): scaling "weak", no collective on the data path, the step
time is the max over ranks.
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
# (cold cache); set to None whenever the dense kernel changes until it is captured again
DENSE_TRAFFIC_BYTES = 46.43e6 + 0.314e6
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
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32"])
    ap.add_argument("--no-extras", action="store_true", help="skip plain-path, latency and CPU-baseline legs")
    ap.add_argument("--profile-run", action="store_true", help="short run for ncu: no extras, no clocks")
    ap.add_argument("--no-graph", action="store_true", help="launch kernel by kernel instead of a CUDA graph")
    ap.add_argument("--tile-px", type=int, default=0,
                    help="dense work item size in source pixels; 0 = automatic (target frame staged in shared memory)")
    ap.add_argument("--large-only", action="store_true",
                    help="run only the 2000-keyframe 160x120 BF16 global solve leg (one JSON line)")
    ap.add_argument("--batch-only", action="store_true", help="only the 256-chunk batch legs (FP32 and BF16 storage)")
    ap.add_argument("--next-rows-only", action="store_true",
                    help="run only the pruning / verification / key-point / TSDF legs (one JSON line)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="frame storage of the timed workload (16-bit: normals, I, grad I)")
    ap.add_argument("--pcg-variant", type=int, default=0, choices=[0, 1, 2, 3],
                    help="PCG kernel: 0 auto, 1 one CTA per problem, 2 grid-cooperative, 3 cluster")
    return ap.parse_args()


def workload():
    import synth
    prob = synth.cfg2()
    prm = prob.solve
    return prob, prm


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
def oracle_gn_iteration_rate(prob, prm, budget_s=15.0, max_pairs=None):
    """Time the FP64 oracle's Gauss-Newton iteration on a bounded sample of pairs and scale.

    The sample is the first k pairs (in pair order) with all their frames; assemble time is
    scaled by n_pairs / k, the PCG over the full explicit system is timed as is.  Single
    BLAS thread.  Returns (GN iterations/s, description, cores)."""
    from oracle import frames as ofr, solver, system
    from oracle.system import SolveParams

    P = SolveParams(n_gn=prm["n_gn"], n_pcg=prm["n_pcg"], w_sparse=prm["w_sparse"], w_dense=prm["w_dense"],
                    w_photo=prm["w_photo"], w_geo=prm["w_geo"])
    n = prob.n_frames
    sp_all = solver.sparse_pairs_for(prob, range(n))
    cache = {}
    t0 = time.perf_counter()
    done = 0
    t_assemble = 0.0
    for sp in sp_all:
        if max_pairs is not None and done >= max_pairs:
            break
        if time.perf_counter() - t0 > budget_s:
            break
        ts = time.perf_counter()
        for f in (sp.a, sp.b):
            if f not in cache:
                cache[f] = ofr.Frame(prob.depth[f], prob.lum[f], prob.intr)
        fr = [cache.get(k) for k in range(n)]
        dp = system.dense_pair_set(prob.init, [sp], P.max_angle_deg)
        system.assemble(fr, prob.intr, prob.init, [sp], dp, P, P.w_dense)
        t_assemble += time.perf_counter() - ts
        done += 1
    m = 6 * (n - 1)
    rng = np.random.default_rng(0)
    B = rng.normal(size=(m, m))
    A = B @ B.T + m * np.eye(m)
    b = rng.normal(size=m)
    ts = time.perf_counter()
    Minv, _ = solver.block_jacobi_inverse(A, "block")
    solver.pcg(A, b, Minv, P.n_pcg)
    t_pcg = time.perf_counter() - ts
    per_iter = t_assemble * (len(sp_all) / max(done, 1)) + t_pcg
    desc = (f"oracle GN iteration: system assembly over {done} of {len(sp_all)} pairs (dense both directions "
            f"+ sparse) timed and scaled to all pairs, plus block-Jacobi PCG ({P.n_pcg} it.) over the full "
            f"{m}x{m} system; numpy, 1 BLAS thread")
    return 1.0 / per_iter, desc, 1


# ------------------------------------------------------------------------------ reference
def run_reference(args, rank, world):
    if rank != 0:
        return
    prob, prm = workload()
    vals = []
    desc = ""
    for k in range(args.warmup + args.steps):
        v, desc, cores = oracle_gn_iteration_rate(prob, prm, budget_s=4.0)
        if k >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * prm["n_gn"] / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": prob.name, "keyframes": prob.n_frames,
                                            "pairs": int(len(prob.pairs)), "n_gn": prm["n_gn"],
                                            "n_pcg": prm["n_pcg"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1604_01093_b300 as bf

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    prob, prm = workload()
    intr = prob.intr
    n = prob.n_frames
    ids = list(range(n))
    if args.large_only:
        stream = torch.cuda.Stream(dev)
        torch.cuda.set_stream(stream)
        if rank == 0:
            print(json.dumps({"large_global": large_global_leg(bf, torch, dev, stream)}), flush=True)
        return
    if args.batch_only:
        stream = torch.cuda.Stream(dev)
        torch.cuda.set_stream(stream)
        if rank == 0:
            import synth
            cprob = synth.cfg3()
            print(json.dumps({"chunk_batch": chunk_batch_leg(bf, torch, dev, stream, prob=cprob),
                              "chunk_batch_bf16": chunk_batch_leg(bf, torch, dev, stream, prob=cprob,
                                                                  storage="bf16")}), flush=True)
        return
    if args.next_rows_only:
        stream = torch.cuda.Stream(dev)
        torch.cuda.set_stream(stream)
        if rank == 0:
            print(json.dumps({"next_rows": next_rows_leg(bf, torch, dev, stream, prob, prm)}), flush=True)
        return
    precision = bf.BF_PREC_MIXED if args.precision == "mixed" else bf.BF_PREC_FP32
    params = bf.default_params(n_gn=prm["n_gn"], n_pcg=prm["n_pcg"], w_sparse=prm["w_sparse"],
                               w_dense=prm["w_dense"], w_photo=prm["w_photo"], w_geo=prm["w_geo"],
                               precision=precision, pcg_variant=args.pcg_variant, use_graph=0 if args.no_graph else 1,
                               tile_px=args.tile_px)
    prof_params = bf.default_params(n_gn=prm["n_gn"], n_pcg=prm["n_pcg"], w_sparse=prm["w_sparse"],
                                    w_dense=prm["w_dense"], w_photo=prm["w_photo"], w_geo=prm["w_geo"],
                                    precision=precision, pcg_variant=args.pcg_variant, use_graph=0,
                                    tile_px=args.tile_px)
    stream = torch.cuda.Stream(dev)  # the library and the timing events share this stream
    torch.cuda.set_stream(stream)
    storage = STORAGE_CODES[args.storage](bf)
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], device=local_rank,
                     stream=stream.cuda_stream, max_frames_hint=n, storage=storage)
    depth_d = torch.from_numpy(prob.depth).to(dev)
    lum_d = torch.from_numpy(prob.lum).to(dev)
    pi_d = torch.from_numpy(prob.p_i).to(dev)
    pj_d = torch.from_numpy(prob.p_j).to(dev)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, pi_d, pj_d)
    torch.cuda.synchronize(dev)
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

    for _ in range(args.warmup):
        st = step()
    torch.cuda.synchronize(dev)
    # then more untimed steps until WARMUP_MIN_S has passed: W steps of this solve take ~10 ms,
    # too short for the GPU and host to settle after an idle period
    t_w = time.perf_counter()
    while not args.profile_run and time.perf_counter() - t_w < WARMUP_MIN_S:
        st = step()
        torch.cuda.synchronize(dev)
    clocks = None if args.profile_run else Clocks(local_rank)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
    t_wall = time.perf_counter()
    ctx.reset_profile()
    times, st, _ = timed(step, args.steps)
    launches = ctx.profile()["launches"]
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(sum(times), dist)
    n_gn = prm["n_gn"]
    value = job_rate(n_gn, args.steps, world, total_ms)
    if args.profile_run:
        if rank == 0:
            print(json.dumps({"profile_run": True, "value": value, "ms_per_step": total_ms / args.steps}))
        return

    # per-kernel device times: a second pass, kernel by kernel, CUDA events around every launch on
    # the context's stream (the graph replay above carries no events)
    _, _, prof = timed(lambda: step(prof_params), max(3, args.steps // 2), profile=True)
    # roofline of the dominant kernel (dense term, ACCUM launches): FP32 flops per launch / event time
    n_dp = 2 * st["n_dense_pairs"]
    HW = intr["W"] * intr["H"]
    dense = prof["kernels"]["dense"]
    dense_ms = dense["ms"] / max(dense["count"], 1)
    units = n_dp * HW
    flops = DENSE_FLOPS_PER_PX * units
    alg_bytes = dense_bytes_per_px(args.storage) * units
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    achieved_tf = flops / (dense_ms / 1000.0) / 1e12
    achieved_gbs = alg_bytes / (dense_ms / 1000.0) / 1e9
    gpu_launches = launches
    # the captured DRAM traffic belongs to the default configuration's dense kernel only
    traffic = DENSE_TRAFFIC_BYTES if (args.storage == "fp32" and args.tile_px == 0) else None
    kernel_share = {k: round(v["ms"] / max(sum(x["ms"] for x in prof["kernels"].values()), 1e-9), 4)
                    for k, v in prof["kernels"].items() if v["count"]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": prob.name, "keyframes": n, "resolution": f"{intr['W']}x{intr['H']}",
                       "cuda_graph": not args.no_graph, "tile_px": args.tile_px,
                       "pairs": int(len(prob.pairs)), "dense_pairs": st["n_dense_pairs"],
                       "directed_dense_pairs": n_dp, "correspondences": prob.n_corr, "n_gn": n_gn,
                       "n_pcg": prm["n_pcg"], "precision": args.precision, "storage": args.storage,
                       "l2": "256 MB buffer written between timed steps (inputs < L2)",
                       "warmup_min_s": WARMUP_MIN_S,
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": gpu_launches,
            "roofline": {"bound": "alu", "kernel": "k_dense", "achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved_tf / FP32_PEAK_TFLOPS,
                         "traffic": traffic, "avg_launch_ms": dense_ms,
                         "flops_per_launch": flops, "flops_per_directed_px": DENSE_FLOPS_PER_PX,
                         "directed_px_per_launch": units,
                         "peak_source": "derived FP32 peak: 148 SMs x 128 lanes x 2 flop x 2.032 GHz"},
            "roofline_hbm_view": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                                  "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                                  "algorithmic_bytes_per_launch": alg_bytes,
                                  "note": f"{dense_bytes_per_px(args.storage)} B per directed source pixel; "
                                          "the frames stay in L2, so DRAM traffic is the unique frame bytes "
                                          "(of measured)"},
            "kernel_time_share": kernel_share,
            "final_energy": st["energy"][-1], "initial_energy": st["energy"][0]}
    if clk:
        line["clocks"] = clk

    if not args.no_extras and rank == 0:
        # e2e through the public API with host (pinned) buffers
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
        te, _, _ = timed(step_e2e, max(3, args.steps // 2))
        h2d = prob.depth.nbytes + prob.lum.nbytes + 2 * 16 * prob.n_corr + prob.init.nbytes
        d2h = n * 16 * 8 + n * 12 * 8
        line["e2e"] = {"value": n_gn / (statistics.mean(te) / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": statistics.mean(te)}
        # restore device-resident correspondences
        ctx.clear_correspondences()
        ctx.add_correspondences_batch(prob.pairs, prob.corr_off, pi_d, pj_d)

        # plain FP32 one-solve-per-launch path on the same workload
        plain = bf.default_params(n_gn=prm["n_gn"], n_pcg=prm["n_pcg"], w_sparse=prm["w_sparse"],
                                  w_dense=prm["w_dense"], w_photo=prm["w_photo"], w_geo=prm["w_geo"],
                                  precision=bf.BF_PREC_FP32)
        for _ in range(2):
            step(plain)
        tp, stp, _ = timed(lambda: step(plain), max(3, args.steps // 2))
        line["plain_fp32"] = {"value": n_gn / (statistics.mean(tp) / 1000.0), "unit": UNIT,
                              "ms_per_step": statistics.mean(tp), "final_energy": stp["energy"][-1]}

        # Sec. 4.4's matrix-free sparse term (J p, then J^T (J p) every PCG iteration) against the
        # sparse 6x6 blocks assembled once per GN iteration, both on the grid-cooperative PCG kernel
        line["sparse_term"] = sparse_term_leg(bf, step, timed, prm, precision, max(3, args.steps // 2))

        # the same global solve on 16-bit frame storage
        if args.storage == "fp32":
            line["bf16_storage"] = storage_leg(bf, torch, dev, stream, prob, params, prof_params, "bf16")

        line["chunk_latency"] = chunk_latency(bf, torch, dev)
        import synth
        cprob = synth.cfg3()
        line["chunk_batch"] = chunk_batch_leg(bf, torch, dev, stream, prob=cprob)
        line["chunk_batch_bf16"] = chunk_batch_leg(bf, torch, dev, stream, prob=cprob, storage="bf16")
        line["serving"] = serving_leg(bf, torch, dev, cprob, prob)

        line["next_rows"] = next_rows_leg(bf, torch, dev, stream, prob, prm)
        line["large_global"] = large_global_leg(bf, torch, dev, stream)

        v, desc, cores = oracle_gn_iteration_rate(prob, prm, budget_s=15.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


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



def next_rows_leg(bf, torch, dev, stream, prob, prm):
    """The steps around the solver on the 300-keyframe workload (Sec. 4.1.1, 4.4.1, 5).

    verify: every pair, both directions, at the ground-truth relative poses (one launch);
    keypoints: every pair's matches through the key-point and surface-area filters (one launch);
    pruning: the global solve with r_max pruning at 0.05 m (the workload has 5 % random outliers,
    so pairs are pruned until the round cap); tsdf: the 300 frames integrated then de-integrated
    (1 cm voxels)."""
    import numpy as np
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

# tiles of half a 320x240 frame for the persistent launch (the fastest of 19200 / 38400 / 76800 there)
PERSISTENT_TILE_PX = 38400


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


def serving_leg(bf, torch, dev, chunk_prob, global_prob, seconds=8.0, rate=30.0, seed=1604):
    """Serving: Poisson arrivals of chunk requests (320x240, 3-11 frames, 6 GN x 10 PCG) at `rate`
    per second for `seconds`, and after every 10th chunk a global request over the first k
    keyframes of the 300-keyframe 80x60 corridor (k grows from 100 to 300; 8 GN x 20 PCG).
    served: continuous batching (2 slots, batches of up to 16, chunk solves on high-priority
    streams, FP32 chunk arithmetic, FP64-merged global solves); plain: the same arrivals served one
    request at a time by the plain FP32 path (1 slot, batch 1).  Latency = submit -> completion;
    p50 / p99 per request kind."""
    rng = np.random.default_rng(seed)
    n_req = int(seconds * rate)
    gaps = rng.exponential(1.0 / rate, size=n_req)
    ci, gi = chunk_prob.intr, global_prob.intr
    lists = [c.tolist() for c in chunk_prob.chunks]
    pc = {k: chunk_prob.solve[k] for k in ("n_gn", "n_pcg", "w_sparse", "w_dense", "w_photo", "w_geo")}
    pg = {k: global_prob.solve[k] for k in ("n_gn", "n_pcg", "w_sparse", "w_dense", "w_photo", "w_geo")}
    out = {"arrival_rate_per_s": rate, "seconds": seconds, "chunk_requests": n_req,
           "global_requests": n_req // 10, "chunk_workload": chunk_prob.name, "global_workload": global_prob.name,
           "hbm_budget_bytes_per_context": SERVING_HBM_BUDGET}
    for name, slots, batch, cprec, gprec in (("served", 2, 16, bf.BF_PREC_FP32, bf.BF_PREC_MIXED),
                                             ("plain_fp32", 1, 1, bf.BF_PREC_FP32, bf.BF_PREC_FP32)):
        # admission by a 40 GB HBM budget (each context; batches that would exceed it are split)
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
        cctx.serve_start(n_slots=slots, max_batch=batch, max_queue=4096)
        gctx.serve_start(n_slots=1, max_batch=1, max_queue=4096)
        cparams = bf.default_params(precision=cprec, **pc)
        gparams = bf.default_params(precision=gprec, **pg)
        # warm-up (not timed): every slot allocates its workspace and pinned staging on first use
        warm = [cctx.submit(lists[k % len(lists)], chunk_id=100000 + k, params=cparams) for k in range(4 * slots)]
        warm.append(gctx.submit(list(range(100)), kind=bf._lib.BF_REQ_GLOBAL, params=gparams))
        for t in warm[:-1]:
            cctx.wait(t)
        gctx.wait(warm[-1])
        ct, gt = [], []
        t0 = time.perf_counter()
        t_next = t0
        for r in range(n_req):
            t_next += gaps[r]
            while time.perf_counter() < t_next:
                time.sleep(0.0002)
            ct.append(cctx.submit(lists[r % len(lists)], chunk_id=r, params=cparams))
            if r % 10 == 9:
                k = int(100 + 200 * r / max(1, n_req - 1))
                gt.append(gctx.submit(list(range(k)), kind=bf._lib.BF_REQ_GLOBAL, params=gparams))
        clat = [cctx.wait(t)[1]["ms"] for t in ct]
        glat = [gctx.wait(t)[1]["ms"] for t in gt]
        wall = time.perf_counter() - t0
        cctx.serve_stop()
        gctx.serve_stop()
        gctx.close()
        # a heavier chunk-only stream, where requests overlap and batching pays
        hi_rate, hi_n = 600.0, 1200
        hgaps = rng.exponential(1.0 / hi_rate, size=hi_n)
        cctx.serve_start(n_slots=slots, max_batch=batch, max_queue=100000)
        for t in [cctx.submit(lists[k % len(lists)], chunk_id=200000 + k, params=cparams) for k in range(4 * slots)]:
            cctx.wait(t)
        ht = []
        th0 = time.perf_counter()
        t_next = th0
        for r in range(hi_n):
            t_next += hgaps[r]
            while time.perf_counter() < t_next:
                time.sleep(0.0001)
            ht.append(cctx.submit(lists[r % len(lists)], chunk_id=300000 + r, params=cparams))
        hlat = sorted(cctx.wait(t)[1]["ms"] for t in ht)
        hwall = time.perf_counter() - th0
        cctx.serve_stop()
        cctx.close()
        clat.sort()
        glat.sort()
        q = lambda v, f: v[min(len(v) - 1, int(f * len(v)))] if v else None  # noqa: E731
        out[name] = {"chunk_p50_ms": q(clat, 0.5), "chunk_p99_ms": q(clat, 0.99), "global_p50_ms": q(glat, 0.5),
                     "global_p99_ms": q(glat, 0.99), "solves_per_s": (len(clat) + len(glat)) / wall,
                     "wall_s": wall, "slots": slots, "max_batch": batch,
                     "chunk_only_600_per_s": {"p50_ms": q(hlat, 0.5), "p99_ms": q(hlat, 0.99),
                                              "solves_per_s": len(hlat) / hwall, "requests": len(hlat)},
                     "precision": {"chunk": "fp32", "global": "mixed" if gprec == bf.BF_PREC_MIXED else "fp32"}}
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
