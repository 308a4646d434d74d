"""GPU parity with 16-bit frame storage: normals, I and grad I held as BF16 or FP16 (depth FP32).

The oracle rounds its own FP64 planes to the same format (round to nearest, ties to even), so
both sides evaluate the energy on the same stored images except for the rare value whose FP32
(device) and FP64 (oracle) results straddle a 16-bit rounding boundary; those differ by one
16-bit ulp.  Association decisions are compared as with FP32 storage (identical except on ties,
tests/replay.py), with the normal gate's tie window widened to the 16-bit normals' rounding, and
everything that compares arithmetic runs the oracle on the library's checked decisions.
Everything downstream keeps the FP32-storage tolerances.
"""
import numpy as np
import pytest

import replay
import synth
from oracle import association, frames as ofr, lie, solver, system
from oracle.system import SolveParams

pytestmark = pytest.mark.gpu

BITS = {"bf16": 8, "fp16": 11}


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


@pytest.fixture(scope="module")
def cfg1():
    return synth.cfg1()


def code(bf, kind):
    return {"fp32": bf.BF_STORE_FP32, "bf16": bf.BF_STORE_BF16, "fp16": bf.BF_STORE_FP16}[kind]


def make_ctx(bf, prob, kind):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], storage=code(bf, kind))
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    for k, (i, j) in enumerate(prob.pairs):
        p, q = prob.pair_corr(k)
        ctx.add_correspondences(int(i), int(j), p, q)
    return ctx


def perturb(poses, seed, rot=0.01, trans=0.02):
    rng = np.random.default_rng(seed)
    out = poses.copy()
    for k in range(1, len(poses)):
        out[k] = poses[k].copy()
        out[k][:3, :3] = lie.exp_so3(rng.normal(scale=rot, size=3)) @ poses[k][:3, :3]
        out[k][:3, 3] += rng.normal(scale=trans, size=3)
    return out


@pytest.mark.parametrize("kind", ["bf16", "fp16"])
def test_stored_planes_are_the_rounded_oracle_planes(bf, cfg1, kind):
    ctx = make_ctx(bf, cfg1, kind)
    ulp = 2.0 ** (1 - BITS[kind])
    for k in (0, 6):
        P = ctx.frame_planes(k)
        f = ofr.Frame(cfg1.depth[k], cfg1.lum[k], cfg1.intr, storage=kind)
        np.testing.assert_array_equal(P[0] > 0, f.valid)
        np.testing.assert_array_equal(P[0][f.valid], cfg1.depth[k][f.valid])
        np.testing.assert_array_equal(np.any(P[1:4] != 0, axis=0), f.nvalid)
        dev = np.concatenate([np.moveaxis(P[1:4], 0, -1).reshape(-1), P[4:7].reshape(-1)]).astype(np.float64)
        ora = np.concatenate([f.N.reshape(-1), f.I.reshape(-1), f.Ix.reshape(-1), f.Iy.reshape(-1)])
        # the FP32-storage tolerances of the unrounded values (normals 2e-5, I planes 2e-6)
        atol = np.concatenate([np.full(f.N.size, 2e-5), np.full(3 * f.I.size, 2e-6)])
        np.testing.assert_array_equal(ofr.round_to_storage(dev, kind), dev)  # representable
        diff = dev != ora
        # only values whose FP32 and FP64 results straddle a rounding boundary differ: a share
        # of about (FP32 error / 16-bit ulp), larger for FP16's finer grid and for small
        # differences of I (cancellation)
        assert diff.mean() < 1e-2, diff.mean()
        # ... by one 16-bit ulp, plus the FP32 error of the value before rounding
        np.testing.assert_array_less(np.abs(dev - ora)[diff], (ulp * np.abs(ora) + atol)[diff])


@pytest.mark.parametrize("kind", ["bf16", "fp16"])
def test_association_agrees_with_the_oracle_on_16bit_frames(bf, cfg1, kind):
    ctx = make_ctx(bf, cfg1, kind)
    fr = [ofr.Frame(cfg1.depth[k], cfg1.lum[k], cfg1.intr, storage=kind) for k in range(cfg1.n_frames)]
    rep = replay.from_ctx(ctx, range(cfg1.n_frames), cfg1.intr["W"], cfg1.intr["H"], storage=kind)
    for poses in (cfg1.gt, perturb(cfg1.gt, 3)):
        for (a, b) in cfg1.pairs:
            for (i, j) in ((int(a), int(b)), (int(b), int(a))):
                M = association.relative_transform(poses[i][:3, :3], poses[i][:3, 3], poses[j][:3, :3],
                                                   poses[j][:3, 3])
                rep(i, j, poses, association.associate(fr[i], fr[j], M, cfg1.intr))
    assert rep.n_valid > 100_000
    # 16-bit normals put more pixels next to the normal gate within rounding: report, bound loosely
    print(f"{kind}: {rep.n_flips} flips of {rep.n_valid} valid")
    assert rep.n_flips <= 1e-3 * rep.n_valid


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", ["bf16", "fp16"])
def test_build_system_matches_oracle_16bit(bf, cfg1, kind, precision):
    ctx = make_ctx(bf, cfg1, kind)
    fr = [ofr.Frame(cfg1.depth[k], cfg1.lum[k], cfg1.intr, storage=kind) for k in range(cfg1.n_frames)]
    poses = perturb(cfg1.gt, 11)
    ids = list(range(cfg1.n_frames))
    w = dict(w_sparse=1.0, w_dense=0.5, w_photo=0.1, w_geo=1.0)
    g = ctx.build_system(ids, poses, precision=precision, **w)
    op = SolveParams(**w)
    sp = solver.sparse_pairs_for(cfg1, ids)
    rep = replay.from_ctx(ctx, ids, cfg1.intr["W"], cfg1.intr["H"], storage=kind)
    S = system.assemble(fr, cfg1.intr, poses, sp, system.dense_pair_set(poses, sp, op.max_angle_deg), op, op.w_dense,
                        assoc=rep)
    tol = 2e-5 if precision == 0 else 2e-4
    assert g["n_dense"] == S.n_dense
    np.testing.assert_allclose(g["A"], S.A, rtol=0, atol=tol * np.abs(S.A).max())
    np.testing.assert_allclose(g["b"], S.b, rtol=0, atol=tol * np.abs(S.b).max())
    assert abs(g["energy"] - S.energy) <= (1e-5 if precision == 0 else 1e-4) * S.energy


@pytest.mark.parametrize("tile_px", [0, 1100])
def test_local_solve_bf16_matches_oracle(bf, cfg1, tile_px):
    """Staged (whole target frame in shared memory) and tiled dense kernels on BF16 frames."""
    fr = [ofr.Frame(cfg1.depth[k], cfg1.lum[k], cfg1.intr, storage="bf16") for k in range(cfg1.n_frames)]
    d = cfg1.solve
    prm = SolveParams(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"],
                      w_photo=d["w_photo"], w_geo=d["w_geo"])
    ctx = make_ctx(bf, cfg1, "bf16")
    ids = list(range(11))
    st, poses, ref = replay.recorded_solve(ctx, ids, lambda: ctx.solve_local(0, ids, tile_px=tile_px, **dict(d)), fr,
                                           cfg1.intr, cfg1.init, solver.sparse_pairs_for(cfg1, ids), prm,
                                           storage="bf16")
    rel = np.abs(np.array(st["energy"]) - ref.energy) / np.abs(ref.energy)
    assert rel.max() <= 1e-5, rel
    for k in range(11):
        rot, tr = lie.pose_error(poses[k], ref.poses[k])
        assert rot <= 1e-4 and tr <= 1e-5, (k, rot, tr)


def test_16bit_store_halves_frame_memory(bf, cfg1):
    """FP32 storage holds two 16-byte planes per pixel (the intensity rides in the second), 16-bit
    storage one 16-byte record plane plus a 2-byte intensity plane."""
    ctxs = {kind: make_ctx(bf, cfg1, kind) for kind in ("fp32", "bf16", "fp16")}
    intr = cfg1.intr
    px = 64 * intr["W"] * intr["H"]  # default capacity: 64 frames
    for kind in ("bf16", "fp16"):
        assert ctxs["fp32"].device_bytes() - ctxs[kind].device_bytes() == px * (16 - 2)
