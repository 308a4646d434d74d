"""Full-size parity in the launch configurations bench.py times, against the FP64 oracle.

* The 300-keyframe global solve (mixed precision, target frames staged in shared memory, cluster
  PCG, the Gauss-Newton loop replayed as a CUDA graph), 8 Gauss-Newton x 20 PCG:
  - single steps: from the oracle's own iterates X_0, X_3 and X_7 (stored in
    tests/golden/global300_oracle.json), the library's Gauss-Newton step against the oracle's step
    from the same poses, run here on the library's checked association decisions (tests/replay.py):
    1e-4 rad, 1e-5 m, 1e-5 relative energy;
  - the whole solve (graph captured and replayed: bitwise the solve recorded kernel by kernel)
    against the oracle's whole solve on the recorded decisions and against the stored oracle solve
    on its own decisions: all nine energies within 1e-5 relative.  The poses after eight steps are
    not fixed to 1e-5 m: the loop's weakly constrained directions amplify any perturbation of a
    step (two oracle runs that decide a few tie pixels differently end 9.6e-4 rad and 2.8e-4 m
    apart with energies equal to 1.4e-7), so the final poses are held only to 2e-2 rad and 2e-2 m
    and the deviations are printed.
* The whole 256-chunk 320x240 batch (FP32 arithmetic, graph; launch sequence and persistent
  launch; FP32 and BF16 frame storage): 18 chunks, two of every length 3..11, each bitwise its solve
  alone, whose association is recorded at every iteration; the oracle's solve on those decisions
  (checked against its own) on the same planes: 1e-4 rad, 1e-5 m, 1e-5;
  against the stored solves of the oracle on its own decisions (tests/golden/chunks256_oracle.json)
  the error is printed and held to 1e-4 rad, 1e-4 m, 1e-4 (a single tie decided the other way
  moves a chunk's energy by up to ~1e-5: a residual at the 0.15 m distance gate).
* The 2000-keyframe 160x120 solve (BF16 frame storage, tiled dense kernel, its PCG): its first
  Gauss-Newton step against the stored step of the oracle on its own decisions, on the same
  BF16-rounded planes: energies 1e-5; the poses of all 2000 keyframes, the 99th percentile within
  1e-4 m and every keyframe within 1e-3 rad and 1e-3 m (the ties decided the other way, 7.6e-6
  of the valid pixels, move a weakly connected stretch of the loop, keyframes 1130-1142 with 14-18
  pairs each, by up to 3.1e-4 m; elsewhere the steps agree to a few 1e-5 m).  With
  BF_SLOW_TESTS=1 the oracle's step on the library's own (checked) decisions is computed here
  (about four minutes on the host cores) and every keyframe is held to 1e-4 rad and 1e-5 m
  (measured 2.3e-6 rad, 8.6e-6 m).  The step's error against the oracle on the unrounded frames
  is printed.

The stored results are written by the make_*_oracle.py scripts beside them from the oracle and
the seeded scene generator alone.
"""
import json
import os

import numpy as np
import pytest

import replay
import synth
from oracle import frames as ofr, lie, solver, system
from oracle.system import SolveParams

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROT_TOL, TRANS_TOL, ENERGY_RTOL = 1e-4, 1e-5, 1e-5
# whole 8-step loop solve: see the module docstring
LOOP_ROT_TOL, LOOP_TRANS_TOL = 2e-2, 2e-2
# the whole loop solve against the oracle on the recorded decisions: only arithmetic differs (a few
# 1e-6 per step), which the loop's weakly constrained directions amplify over the eight steps
LOOP_REC_TOL = 2e-2
# a single step compared with the oracle on its own decisions (no replay): see the module docstring
STEP_TRANS_TOL_OWN = 1e-4
STEP2000_OWN_TOL, STEP2000_OWN_P99_TRANS = 1e-3, 1e-4


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


@pytest.fixture(scope="module")
def global300():
    return synth.cfg2()


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "global300_oracle.json")) as f:
        return json.load(f)


def make_ctx(bf, prob):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                     max_frames_hint=prob.n_frames)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, prob.p_i, prob.p_j)
    return ctx


def params(prob, n_gn):
    d = prob.solve
    return dict(n_gn=n_gn, n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
                w_geo=d["w_geo"], use_graph=1)


def poses44(rows):
    out = np.tile(np.eye(4), (len(rows), 1, 1))
    out[:, :3, :] = np.array(rows).reshape(-1, 3, 4)
    return out


def worst_pose_error(P, Q):
    e = [lie.pose_error(P[k], Q[k]) for k in range(len(P))]
    return max(x[0] for x in e), max(x[1] for x in e)


def test_golden_matches_the_workload(global300, golden):
    assert golden["workload"] == global300.name and golden["n_frames"] == global300.n_frames
    assert golden["pairs"] == len(global300.pairs) and golden["n_pcg"] == global300.solve["n_pcg"]
    assert golden["n_gn"] == global300.solve["n_gn"] and len(golden["energy"]) == golden["n_gn"] + 1


def test_global300_single_steps_match_oracle(bf, global300, golden):
    """Gauss-Newton steps k = 0, 3, 7 of the 8-step solve, each from the oracle's iterate X_k."""
    prob = global300
    n = prob.n_frames
    ids = list(range(n))
    frames = [ofr.Frame(prob.depth[k], prob.lum[k], prob.intr) for k in ids]
    sp = solver.sparse_pairs_for(prob, ids)
    d = prob.solve
    prm = SolveParams(n_gn=1, n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
                      w_geo=d["w_geo"])
    ctx = make_ctx(bf, prob)
    rep = replay.from_ctx(ctx, ids, prob.intr["W"], prob.intr["H"])
    hist = golden["iterates"]
    with system.frame_pool(frames, min(16, os.cpu_count() or 1)) as pool:
        pmap = lambda f, tasks: pool.map(f, tasks, chunksize=16)  # noqa: E731
        for k in (0, 3, 7):
            Xk = prob.init if k == 0 else poses44(hist[str(k)])
            # the dense pair set is fixed at the solve's initial poses (Sec. 4.3): here X_k, on both sides
            dp = system.dense_pair_set(Xk, sp, prm.max_angle_deg)
            S = system.assemble(frames, prob.intr, Xk, sp, dp, prm, prm.w_dense, assoc=rep, pmap=pmap)
            Minv, _ = solver.block_jacobi_inverse(S.A, prm.precond)
            delta, _ = solver.pcg(S.A, S.b, Minv, prm.n_pcg)
            Xn = solver.apply_step(Xk, delta)
            ctx.add_frames(0, prob.depth, prob.lum, init_pose=Xk)
            st = ctx.solve_global(ids, **params(prob, 1))
            assert st["flags"] == 0
            assert abs(st["energy"][0] - S.energy) <= ENERGY_RTOL * S.energy, (k, st["energy"][0], S.energy)
            assert abs(st["energy"][0] - golden["energy"][k]) <= ENERGY_RTOL * golden["energy"][k]
            rot, tr = worst_pose_error(ctx.get_poses(ids), Xn)
            print(f"step {k}: energy rel {abs(st['energy'][0] - S.energy) / S.energy:.2e}, pose {rot:.2e} rad "
                  f"{tr:.2e} m, association flips {rep.n_flips} of {rep.n_valid}")
            assert rot <= ROT_TOL and tr <= TRANS_TOL, (k, rot, tr)
    assert rep.n_flips <= 1e-4 * rep.n_valid


def test_global300_whole_bench_solve_matches_oracle(bf, global300, golden):
    """The bench's own solve (8 GN x 20 PCG): captured as a graph, then replayed, bitwise the solve
    launched kernel by kernel with its association recorded; the oracle's whole solve on the
    recorded decisions; and the stored solve of the oracle on its own decisions (all nine energies
    within 1e-5; the final poses, which the loop's weakly constrained directions leave undetermined
    to a few 1e-3 m by a handful of ties, printed and held to LOOP_*_TOL)."""
    prob = global300
    ctx = make_ctx(bf, prob)
    ids = list(range(prob.n_frames))
    runs = []
    for _ in range(2):  # capture, then replay the graph
        ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
        st = ctx.solve_global(ids, **params(prob, prob.solve["n_gn"]))
        assert st["flags"] == 0 and st["n_gn"] == prob.solve["n_gn"]
        runs.append((st, ctx.get_poses(ids)))
    gold = np.array(golden["energy"])
    rel = np.abs(np.array(runs[0][0]["energy"]) - gold) / gold
    rot, tr = worst_pose_error(runs[0][1], poses44(golden["poses"]))
    print(f"whole solve vs the oracle on its own decisions: energy {rel.max():.2e}, final poses {rot:.2e} rad "
          f"{tr:.2e} m")
    assert rel.max() <= ENERGY_RTOL, rel
    assert rot <= LOOP_ROT_TOL and tr <= LOOP_TRANS_TOL, (rot, tr)
    # the same solve kernel by kernel, recorded; the oracle on its decisions
    d = prob.solve
    prm = SolveParams(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"],
                      w_photo=d["w_photo"], w_geo=d["w_geo"])
    frames = ofr.FrameCache(prob.depth, prob.lum, prob.intr)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    with system.frame_pool(frames, min(16, os.cpu_count() or 1)) as pool:
        st, P, ref = replay.recorded_solve(ctx, ids, lambda: ctx.solve_global(ids, **dict(params(prob, d["n_gn"]),
                                                                                         use_graph=0)),
                                           [None] * len(ids), prob.intr, prob.init, solver.sparse_pairs_for(prob, ids),
                                           prm, pmap=lambda f, tasks: pool.map(f, tasks, chunksize=16),
                                           frame_keys=ids)
    assert st["energy"] == runs[0][0]["energy"] and st["energy"] == runs[1][0]["energy"]
    np.testing.assert_array_equal(P, runs[0][1])
    np.testing.assert_array_equal(P, runs[1][1])
    rel = np.abs(np.array(st["energy"]) - np.array(ref.energy)) / np.array(ref.energy)
    rot, tr = worst_pose_error(P, ref.poses)
    print(f"whole solve vs the oracle on the recorded decisions: energy {rel.max():.2e}, final poses {rot:.2e} rad "
          f"{tr:.2e} m, flips {ref.replay.n_flips} of {ref.replay.n_valid}")
    assert rel.max() <= ENERGY_RTOL, rel
    assert rot <= LOOP_REC_TOL and tr <= LOOP_REC_TOL, (rot, tr)
    assert ref.replay.n_flips <= 1e-4 * ref.replay.n_valid


@pytest.fixture(scope="module")
def chunks256():
    return synth.cfg3()


@pytest.fixture(scope="module")
def golden_chunks():
    with open(os.path.join(HERE, "golden", "chunks256_oracle.json")) as f:
        return json.load(f)


def sampled_chunks(prob):
    """Two chunks of every length 3..11 (the first two of that length)."""
    out = []
    for n in range(3, 12):
        out += [k for k, c in enumerate(prob.chunks) if len(c) == n][:2]
    return out


def chunk_context(bf, prob, storage):
    import torch
    intr = prob.intr
    dev = torch.device("cuda", 0)
    code = {"fp32": bf.BF_STORE_FP32, "bf16": bf.BF_STORE_BF16}[storage]
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                     max_frames_hint=prob.n_frames, storage=code)
    ctx.add_frames(0, torch.from_numpy(prob.depth).to(dev), torch.from_numpy(prob.lum).to(dev))
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, torch.from_numpy(prob.p_i).to(dev),
                                  torch.from_numpy(prob.p_j).to(dev))
    return ctx


@pytest.fixture(scope="module")
def chunk_oracle(bf, chunks256):
    """Per frame storage: the batch's autotuned decomposition, and for each sampled chunk its solve
    alone with that decomposition (association recorded; alone = inside the batch, bitwise) and the
    oracle's solve (6 GN x 10 PCG from the identity) on the recorded decisions, the dense pairs of
    each assembly spread over a spawn pool of the host's cores."""
    prob = chunks256
    d = prob.solve
    prm = SolveParams(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"],
                      w_photo=d["w_photo"], w_geo=d["w_geo"])
    kw = dict(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
              w_geo=d["w_geo"], precision=bf.BF_PREC_FP32)
    cache = {}

    def get(storage):
        if storage in cache:
            return cache[storage]
        chunks = sampled_chunks(prob)
        fids = sorted({int(f) for k in chunks for f in prob.chunks[k]})
        frames = ofr.FrameCache({f: prob.depth[f] for f in fids}, {f: prob.lum[f] for f in fids}, prob.intr,
                                storage=None if storage == "fp32" else storage)
        ctx = chunk_context(bf, prob, storage)
        ctx.solve_local(0, prob.chunks[0].tolist(), tile_px=bf.BF_TILE_AUTOTUNE, **kw)  # the autotuner's choice
        tile = ctx.tuned_tile_px()
        out = {"tile": tile, "alone": {}, "oracle": {}}
        with system.frame_pool(frames, min(16, os.cpu_count() or 1)) as pool:
            pmap = lambda f, tasks: pool.map(f, tasks, chunksize=1)  # noqa: E731
            for k in chunks:
                ids = [int(f) for f in prob.chunks[k]]
                st, P, ref = replay.recorded_solve(
                    ctx, ids, lambda: ctx.solve_local(5000 + k, ids, tile_px=tile, **kw), [None] * len(ids),
                    prob.intr, prob.init[ids], solver.sparse_pairs_for(prob, ids), prm, storage=storage, pmap=pmap,
                    frame_keys=ids)
                out["alone"][k] = (st, P)
                out["oracle"][k] = ref
        ctx.close()
        cache[storage] = out
        return out

    return get


@pytest.mark.parametrize("storage,persistent", [("fp32", 0), ("fp32", 1), ("bf16", 0)])
def test_chunks256_batch_matches_oracle_on_sampled_chunks(bf, chunks256, chunk_oracle, golden_chunks, storage,
                                                         persistent):
    """The whole 256-chunk 320x240 batch in bench.py's configuration (FP32 arithmetic, CUDA graph,
    the autotuned decomposition; the launch sequence and the persistent launch): two chunks of every
    length 3..11 are bitwise their solve alone, which matches the oracle's solve on the decisions it
    recorded (the accuracy targets); against the stored solves of the oracle on its own decisions
    the error is printed (it includes the ties decided the other way)."""
    prob = chunks256
    assert golden_chunks["workload"] == prob.name and golden_chunks["chunks"] == len(prob.chunks)
    ref = chunk_oracle(storage)
    ctx = chunk_context(bf, prob, storage)
    d = prob.solve
    lists = [c.tolist() for c in prob.chunks]
    stats = ctx.solve_local_batch(list(range(len(lists))), lists, n_gn=d["n_gn"], n_pcg=d["n_pcg"],
                                  w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
                                  w_geo=d["w_geo"], precision=bf.BF_PREC_FP32, use_graph=1, tile_px=ref["tile"],
                                  persistent=persistent)
    assert sorted({len(lists[k]) for k in ref["oracle"]}) == list(range(3, 12)) and len(ref["oracle"]) >= 16
    worst = [0.0, 0.0, 0.0]
    flips = valid = 0
    for k, res in ref["oracle"].items():
        st, P = ref["alone"][k]
        assert stats[k]["energy"] == st["energy"], k
        np.testing.assert_array_equal(ctx.get_poses(lists[k]), P)
        rel = np.abs(np.array(st["energy"]) - np.array(res.energy)) / np.array(res.energy)
        rot, tr = worst_pose_error(P, res.poses)
        worst = [max(worst[0], rot), max(worst[1], tr), max(worst[2], rel.max())]
        assert rel.max() <= ENERGY_RTOL, (k, rel)
        assert rot <= ROT_TOL and tr <= TRANS_TOL, (k, rot, tr)
        flips, valid = flips + res.replay.n_flips, valid + res.replay.n_valid
    assert flips <= 1e-4 * valid
    own = [0.0, 0.0, 0.0]
    for s in golden_chunks["samples"]:
        if s["storage"] != storage:
            continue
        k = s["chunk"]
        assert lists[k] == s["frames"]
        rel = np.abs(np.array(stats[k]["energy"]) - np.array(s["energy"])) / np.array(s["energy"])
        rot, tr = worst_pose_error(ctx.get_poses(lists[k]), poses44(s["poses"]))
        own = [max(own[0], rot), max(own[1], tr), max(own[2], rel.max())]
    print(f"{storage} persistent={persistent} tile={ref['tile']}: {len(ref['oracle'])} chunks, replayed oracle: "
          f"{worst[0]:.2e} rad {worst[1]:.2e} m energy {worst[2]:.2e} (flips {flips} of {valid}); oracle on its "
          f"own decisions: {own[0]:.2e} rad {own[1]:.2e} m energy {own[2]:.2e}")
    assert own[0] <= ROT_TOL and own[1] <= 1e-4 and own[2] <= 1e-4
    ctx.close()


@pytest.fixture(scope="module")
def global2000():
    return synth.cfg5()


@pytest.fixture(scope="module")
def golden2000():
    with open(os.path.join(HERE, "golden", "global2000_oracle.json")) as f:
        return json.load(f)


def test_global2000_first_step_matches_oracle(bf, global2000, golden2000):
    """The 2000-keyframe 160x120 solve in bench.py's configuration (BF16 frame storage, mixed
    precision, tiled dense kernel with the autotuned decomposition, its PCG, CUDA graph): its first
    Gauss-Newton step against the oracle's on the same BF16-rounded planes (energies, and the poses
    of all 2000 keyframes); the bench's own 10-step solve starts at the same two energies.  The
    step's error against the oracle on the unrounded frames (the cost of BF16 storage, every 32nd
    keyframe) is printed."""
    import torch
    prob = global2000
    assert golden2000["workload"] == prob.name and golden2000["n_frames"] == prob.n_frames
    intr = prob.intr
    dev = torch.device("cuda", 0)
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                     max_frames_hint=prob.n_frames, storage=bf.BF_STORE_BF16)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, torch.from_numpy(prob.p_i).to(dev),
                                  torch.from_numpy(prob.p_j).to(dev))
    depth, lum = torch.from_numpy(prob.depth).to(dev), torch.from_numpy(prob.lum).to(dev)
    d = prob.solve
    common = dict(n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
                  w_geo=d["w_geo"], use_graph=1, tile_px=bf.BF_TILE_AUTOTUNE)
    ids = list(range(prob.n_frames))
    ctx.add_frames(0, depth, lum, init_pose=prob.init)
    st = ctx.solve_global(ids, n_gn=1, **common)
    assert st["flags"] == 0
    for ref_name in ("fp32", "bf16"):
        g = golden2000[ref_name]
        gold_e = np.array(g["energy"])
        rel = np.abs(np.array(st["energy"]) - gold_e) / gold_e
        P = ctx.get_poses(g["frames_kept"])
        rot, tr = worst_pose_error(P, poses44(g["poses"]))
        trs = [lie.pose_error(a, b)[1] for a, b in zip(P, poses44(g["poses"]))]
        p99 = float(np.quantile(trs, 0.99))
        print(f"2000 keyframes, BF16 storage vs oracle on {ref_name} planes: energy {rel.max():.2e}, "
              f"poses {rot:.2e} rad {tr:.2e} m (99th percentile {p99:.2e} m)")
        if ref_name == "bf16":
            assert rel.max() <= ENERGY_RTOL, rel
            # the oracle decided on its own here (no replay): see the module docstring
            assert rot <= STEP2000_OWN_TOL and tr <= STEP2000_OWN_TOL, (rot, tr)
            assert p99 <= STEP2000_OWN_P99_TRANS, p99
    gold_e = np.array(golden2000["bf16"]["energy"])
    ctx.add_frames(0, depth, lum, init_pose=prob.init)
    full = ctx.solve_global(ids, n_gn=d["n_gn"], **common)
    assert abs(full["energy"][0] - gold_e[0]) <= ENERGY_RTOL * gold_e[0]
    assert abs(full["energy"][1] - gold_e[1]) <= ENERGY_RTOL * gold_e[1]
    assert full["energy"][-1] < full["energy"][0]


@pytest.mark.skipif(os.environ.get("BF_SLOW_TESTS") != "1", reason="slow (about four minutes): BF_SLOW_TESTS=1")
def test_global2000_first_step_on_library_decisions(bf, global2000):
    """The 2000-keyframe first Gauss-Newton step against the oracle's step on the library's own
    association decisions (fetched at the oracle's poses and checked: ties only), every keyframe."""
    import torch
    prob = global2000
    d = prob.solve
    ids = list(range(prob.n_frames))
    frames = [ofr.Frame(prob.depth[k], prob.lum[k], prob.intr, storage="bf16") for k in ids]
    intr = prob.intr
    dev = torch.device("cuda", 0)
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                     max_frames_hint=prob.n_frames, storage=bf.BF_STORE_BF16)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, torch.from_numpy(prob.p_i).to(dev),
                                  torch.from_numpy(prob.p_j).to(dev))
    ctx.add_frames(0, torch.from_numpy(prob.depth).to(dev), torch.from_numpy(prob.lum).to(dev), init_pose=prob.init)
    kw = dict(n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"], w_geo=d["w_geo"])
    st = ctx.solve_global(ids, n_gn=1, use_graph=1, tile_px=bf.BF_TILE_AUTOTUNE, **kw)
    P = ctx.get_poses(ids)
    rep = replay.from_ctx(ctx, ids, intr["W"], intr["H"], storage="bf16")
    with system.frame_pool(frames, None) as pool:
        ref = solver.gauss_newton(frames, intr, prob.init, solver.sparse_pairs_for(prob, ids),
                                  SolveParams(n_gn=1, **kw), assoc=rep,
                                  pmap=lambda f, tasks: pool.map(f, tasks, chunksize=64))
    rel = np.abs(np.array(st["energy"]) - np.array(ref.energy)) / np.array(ref.energy)
    rot, tr = worst_pose_error(P, ref.poses)
    print(f"2000 keyframes on the library's decisions: energy {rel.max():.2e}, poses {rot:.2e} rad {tr:.2e} m, "
          f"flips {rep.n_flips} of {rep.n_valid}")
    assert rel.max() <= ENERGY_RTOL and rot <= ROT_TOL and tr <= TRANS_TOL, (rel.max(), rot, tr)
    assert rep.n_flips <= 1e-4 * rep.n_valid
    ctx.close()
