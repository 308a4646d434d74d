"""Error of GPU solves against the FP64 oracle, for the precision / storage options.

The accuracy targets are 1e-4 rad in rotation, 1e-5 m in translation and 1e-5 relative in the
per-iteration energy.  Two problems are solved:

* the 11-frame 80x60 chunk, in mixed precision, in plain FP32 and with BF16 frame storage;
* one 5-frame chunk of the 256-chunk 320x240 batch, in the batch's FP32 arithmetic, with FP32 and
  with BF16 storage (a chunk solved alone gives the same bits as inside its batch).

The oracle sees the unrounded frames in every case.  FP32 storage must meet the targets.  BF16
storage is a memory-traffic option: its error against unrounded frames is printed, not asserted.
Against the oracle on the same rounded planes it is parity-green; tests/test_gpu_storage16.py
checks that.  Run with -s to print the table.
"""
import json

import numpy as np
import pytest

import synth
from oracle import frames as ofr, lie, solver
from oracle.system import SolveParams

pytestmark = pytest.mark.gpu

TOL = {"rotation_rad": 1e-4, "translation_m": 1e-5, "energy_rel": 1e-5}


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


def errors(st, poses, ref):
    rot = max(lie.pose_error(poses[k], ref.poses[k])[0] for k in range(len(poses)))
    tr = max(lie.pose_error(poses[k], ref.poses[k])[1] for k in range(len(poses)))
    en = max(abs(a - b) / abs(b) for a, b in zip(st["energy"], ref.energy))
    return {"rotation_rad": rot, "translation_m": tr, "energy_rel": en}


def case(bf, prob, ids, runs):
    d = prob.solve
    intr = prob.intr
    fr = [ofr.Frame(prob.depth[f], prob.lum[f], intr) for f in ids]
    ref = solver.gauss_newton(fr, intr, prob.init[ids], solver.sparse_pairs_for(prob, ids),
                              SolveParams(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"],
                                          w_dense=d["w_dense"], w_photo=d["w_photo"], w_geo=d["w_geo"]))
    out = {}
    for name, storage, kw in runs:
        ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], storage=storage,
                         max_frames_hint=len(ids))
        ctx.add_frames(0, prob.depth[ids], prob.lum[ids])
        loc = {f: k for k, f in enumerate(ids)}
        for k, (i, j) in enumerate(prob.pairs):
            if int(i) in loc and int(j) in loc:
                p, q = prob.pair_corr(k)
                ctx.add_correspondences(loc[int(i)], loc[int(j)], p, q)
        st = ctx.solve_local(0, list(range(len(ids))),
                             **{k: d[k] for k in ("n_gn", "n_pcg", "w_sparse", "w_dense", "w_photo", "w_geo")}, **kw)
        out[name] = errors(st, ctx.get_poses(list(range(len(ids)))), ref)
        ctx.close()
    return out


def check(table, fp32_names):
    print(json.dumps(table, indent=1))
    for name in fp32_names:
        for k, tol in TOL.items():
            assert table[name][k] <= tol, (name, k, table[name][k])


def test_chunk11_80x60(bf):
    c1 = synth.cfg1()
    table = case(bf, c1, list(range(c1.n_frames)),
                 [("mixed", bf.BF_STORE_FP32, {}), ("plain_fp32", bf.BF_STORE_FP32, {"precision": bf.BF_PREC_FP32}),
                  ("mixed_bf16_storage", bf.BF_STORE_BF16, {})])
    check(table, ["mixed", "plain_fp32"])


def test_batch_chunk_320x240(bf):
    prob = synth.cfg3()
    k = min(range(len(prob.chunks)), key=lambda c: (len(prob.chunks[c]) != 5, c))
    ids = [int(f) for f in prob.chunks[k]]
    table = case(bf, prob, ids, [("fp32_arith_fp32_storage", bf.BF_STORE_FP32, {"precision": bf.BF_PREC_FP32}),
                                 ("fp32_arith_bf16_storage", bf.BF_STORE_BF16, {"precision": bf.BF_PREC_FP32})])
    check(table, ["fp32_arith_fp32_storage"])
    assert np.isfinite(table["fp32_arith_bf16_storage"]["translation_m"])


def test_compensated_sums_320x240(bf):
    """Normal equations of a 5-frame 320x240 chunk at perturbed poses (mixed precision: tile sums
    merged in FP64, so the FP32 per-thread runs are the main rounding source), with tiles of a
    whole frame (runs of 300 pixels per thread), of half a frame and of 4800 pixels (runs of 19),
    each with plain and with compensated per-thread sums, against the oracle on the same (checked)
    decisions.  Printed with -s; every variant within the parity tolerance, and compensation does
    not make the long runs less accurate."""
    import replay
    from oracle import solver, system
    prob = synth.chunk_batch(57, n_chunks=6, W=320, H=240, length=(5, 5), n_corr=(100, 200), name="batch320")
    ids = [int(f) for f in prob.chunks[0]]
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], max_frames_hint=prob.n_frames)
    ctx.add_frames(0, prob.depth, prob.lum)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, prob.p_i, prob.p_j)
    rng = np.random.default_rng(4)
    poses = prob.gt[ids].copy()
    for k in range(1, len(ids)):
        R, t = lie.apply_update(poses[k][:3, :3], poses[k][:3, 3], np.r_[rng.normal(0, 0.005, 3), rng.normal(0, 0.01, 3)])
        poses[k] = lie.to44(R, t)
    fr = [ofr.Frame(prob.depth[f], prob.lum[f], intr) for f in ids]
    prm = SolveParams(w_sparse=0.0, w_dense=1.0, w_photo=0.1, w_geo=1.0)
    sp = solver.sparse_pairs_for(prob, ids)
    S = system.assemble(fr, intr, poses, sp, system.dense_pair_set(poses, sp, prm.max_angle_deg), prm, 1.0,
                        assoc=replay.from_ctx(ctx, ids, intr["W"], intr["H"]))
    table = {}
    for tile in (76800, 38400, 4800):
        for comp in (0, 1):
            g = ctx.build_system(ids, poses, w_sparse=0.0, w_dense=1.0, w_photo=0.1, w_geo=1.0, tile_px=tile,
                                 compensated=comp, precision=bf.BF_PREC_MIXED)
            assert g["n_dense"] == S.n_dense
            table[f"tile{tile}_{'compensated' if comp else 'plain'}"] = {
                "A": float(np.abs(g["A"] - S.A).max() / np.abs(S.A).max()),
                "b": float(np.abs(g["b"] - S.b).max() / np.abs(S.b).max()),
                "energy": abs(g["energy"] - S.energy) / S.energy}
    print(json.dumps(table, indent=1))
    for v in table.values():
        assert v["A"] <= 2e-5 and v["b"] <= 2e-5 and v["energy"] <= TOL["energy_rel"]
    long_plain, long_comp = table["tile76800_plain"], table["tile76800_compensated"]
    assert long_comp["A"] <= 1.5 * long_plain["A"] and long_comp["energy"] <= 1.5 * long_plain["energy"] + 1e-9
