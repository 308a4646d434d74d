"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerances (the accuracy targets, and ones derived from the FP32 evaluation):
* final poses: rotation <= 1e-4 rad, translation <= 1e-5 m;
* per-iteration energy: relative error <= 1e-5;
* association: the library decides in FP32, the oracle in FP64 (Sec. 4.3 as written); they
  must agree on every pixel except ties (a decision within FP32 rounding of its threshold),
  and the ties that do flip stay below 1e-4 of the valid residuals;
* everything that compares arithmetic runs the oracle on the library's checked decisions
  (tests/replay.py): the normal equations at given poses on the decisions bf_debug_association
  returns there, the solves on the decisions the library recorded at every Gauss-Newton iteration
  (bf_debug_record_association), so both sides sum the same pixels at every step;
* assembled normal equations: FP32 per-pixel evaluation with FP64 merging, so entries
  agree to ~1e-6 of the block's scale; tested at 2e-5 of the largest entry of A (b: of
  the largest entry of b).
"""
import numpy as np
import pytest

import replay
import synth
from oracle import association, frames as ofr, hierarchy, lie, solver, system
from oracle.system import SolveParams

pytestmark = pytest.mark.gpu

ROT_TOL = 1e-4
TRANS_TOL = 1e-5
ENERGY_RTOL = 1e-5
FLIP_BUDGET = 1e-4  # association flips (ties decided the other way) per valid residual


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


@pytest.fixture(scope="module")
def cfg1():
    return synth.cfg1()


@pytest.fixture(scope="module")
def cfg1_frames(cfg1):
    return [ofr.Frame(cfg1.depth[k], cfg1.lum[k], cfg1.intr) for k in range(cfg1.n_frames)]


def make_ctx(bf, prob, **kw):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], **kw)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    for k, (i, j) in enumerate(prob.pairs):
        p, q = prob.pair_corr(k)
        ctx.add_correspondences(int(i), int(j), p, q)
    return ctx


def oracle_params(d):
    return SolveParams(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"],
                       w_photo=d["w_photo"], w_geo=d["w_geo"])


def perturb(poses, seed, rot=0.01, trans=0.02):
    rng = np.random.default_rng(seed)
    out = poses.copy()
    for k in range(1, len(out)):
        R, t = lie.apply_update(out[k][:3, :3], out[k][:3, 3], np.r_[rng.normal(0, rot, 3), rng.normal(0, trans, 3)])
        out[k] = lie.to44(R, t)
    return out


# ----------------------------------------------------------------------------- preprocessing

def test_preprocess_matches_oracle(bf, cfg1, cfg1_frames):
    ctx = make_ctx(bf, cfg1)
    for k in (0, 5, 10):
        P = ctx.frame_planes(k)
        f = cfg1_frames[k]
        np.testing.assert_array_equal(P[0] > 0, f.valid)
        np.testing.assert_array_equal(P[0][f.valid], cfg1.depth[k][f.valid])
        nvalid = np.any(P[1:4] != 0, axis=0)
        np.testing.assert_array_equal(nvalid, f.nvalid)
        np.testing.assert_allclose(np.moveaxis(P[1:4], 0, -1)[f.nvalid], f.N[f.nvalid], atol=2e-5)
        np.testing.assert_allclose(P[4], f.I, atol=2e-6)
        np.testing.assert_allclose(P[5], f.Ix, atol=2e-6)
        np.testing.assert_allclose(P[6], f.Iy, atol=2e-6)


def test_malformed_depth_is_invalid_and_the_solve_stays_finite(bf, cfg1):
    """Host-side fault injection: NaN, +-inf, negative and out-of-range depths in the input frames
    are invalid pixels exactly as the oracle marks them (and so are their normals' neighbours), and
    a solve over the corrupted frames stays finite."""
    depth = cfg1.depth.copy()
    rng = np.random.default_rng(3)
    for k in range(cfg1.n_frames):
        idx = rng.choice(depth[k].size, 60, replace=False)
        flat = depth[k].reshape(-1)
        flat[idx[:15]] = np.nan
        flat[idx[15:30]] = np.inf
        flat[idx[30:45]] = -np.inf
        flat[idx[45:52]] = -1.0
        flat[idx[52:]] = 1e6
    intr = cfg1.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"])
    ctx.add_frames(0, depth, cfg1.lum)
    for k, (i, j) in enumerate(cfg1.pairs):
        p, q = cfg1.pair_corr(k)
        ctx.add_correspondences(int(i), int(j), p, q)
    for k in (0, 7):
        P = ctx.frame_planes(k)
        f = ofr.Frame(depth[k], cfg1.lum[k], intr)
        np.testing.assert_array_equal(P[0] > 0, f.valid)
        np.testing.assert_array_equal(np.any(P[1:4] != 0, axis=0), f.nvalid)
        assert np.isfinite(P).all()
    st = ctx.solve_local(0, list(range(cfg1.n_frames)), **dict(cfg1.solve))
    assert np.isfinite(st["energy"]).all() and np.isfinite(ctx.get_poses(list(range(cfg1.n_frames)))).all()


# ------------------------------------------------------------------------------- association

@pytest.mark.parametrize("seed", [None, 3, 4])
def test_association_agrees_with_the_fp64_oracle(bf, cfg1, cfg1_frames, seed):
    """Every directed pair of the 11-frame chunk at ground truth and at perturbed poses (general
    position): the library's FP32 decisions equal the oracle's FP64 ones except on ties, and the
    flipped ties are at most 1e-4 of the valid residuals."""
    ctx = make_ctx(bf, cfg1)
    poses = cfg1.gt if seed is None else perturb(cfg1.gt, seed, 0.02, 0.04)
    W, H = cfg1.intr["W"], cfg1.intr["H"]
    rep = replay.from_ctx(ctx, range(cfg1.n_frames), W, H)
    for (a, b) in cfg1.pairs:
        for (i, j) in ((int(a), int(b)), (int(b), int(a))):
            M = association.relative_transform(poses[i][:3, :3], poses[i][:3, 3], poses[j][:3, :3], poses[j][:3, 3])
            rep(i, j, poses, association.associate(cfg1_frames[i], cfg1_frames[j], M, cfg1.intr))
    assert rep.n_valid > 100_000
    assert rep.n_flips <= FLIP_BUDGET * rep.n_valid, (rep.n_flips, rep.n_valid)


def test_association_agrees_with_the_fp64_oracle_at_320x240(bf, batch320):
    """The same at 320x240 (focal length 262.5 px: four times the projection's rounding in pixels)."""
    prob = batch320
    ctx = make_ctx(bf, prob, max_frames_hint=prob.n_frames)
    W, H = prob.intr["W"], prob.intr["H"]
    fr = {}
    poses = perturb(prob.gt, 8, 0.01, 0.02)
    rep = replay.from_ctx(ctx, range(prob.n_frames), W, H)
    for (a, b) in prob.pairs[:24]:
        for (i, j) in ((int(a), int(b)), (int(b), int(a))):
            for k in (i, j):
                if k not in fr:
                    fr[k] = ofr.Frame(prob.depth[k], prob.lum[k], prob.intr)
            M = association.relative_transform(poses[i][:3, :3], poses[i][:3, 3], poses[j][:3, :3], poses[j][:3, 3])
            rep(i, j, poses, association.associate(fr[i], fr[j], M, prob.intr))
    assert rep.n_valid > 1_000_000
    assert rep.n_flips <= FLIP_BUDGET * rep.n_valid, (rep.n_flips, rep.n_valid)


# ----------------------------------------------------------------------- normal equations

WEIGHTS = {
    "sparse_only": dict(w_sparse=1.0, w_dense=0.0, dense_on=0),
    "geo_only": dict(w_sparse=0.0, w_dense=1.0, w_photo=0.0, w_geo=1.0),
    "photo_only": dict(w_sparse=0.0, w_dense=1.0, w_photo=1.0, w_geo=0.0),
    "full": dict(w_sparse=1.0, w_dense=0.5, w_photo=0.1, w_geo=1.0),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("wname", list(WEIGHTS))
def test_build_system_matches_oracle(bf, cfg1, cfg1_frames, wname, precision):
    w = WEIGHTS[wname]
    ctx = make_ctx(bf, cfg1)
    poses = perturb(cfg1.gt, 11)
    ids = list(range(cfg1.n_frames))
    g = ctx.build_system(ids, poses, precision=precision, **w)
    op = SolveParams(w_sparse=w["w_sparse"], w_dense=w["w_dense"], w_photo=w.get("w_photo", 0.1),
                     w_geo=w.get("w_geo", 1.0), dense_on=bool(w.get("dense_on", 1)))
    sp = solver.sparse_pairs_for(cfg1, ids)
    dp = system.dense_pair_set(poses, sp, op.max_angle_deg) if op.dense_on else []
    rep = replay.from_ctx(ctx, ids, cfg1.intr["W"], cfg1.intr["H"])
    S = system.assemble(cfg1_frames, cfg1.intr, poses, sp, dp, op, op.w_dense, assoc=rep)
    # both paths at the same tolerance (the plain path's FP32 merges included)
    tol = 2e-5
    assert g["n_dense"] == S.n_dense
    np.testing.assert_allclose(g["A"], S.A, rtol=0, atol=tol * np.abs(S.A).max())
    np.testing.assert_allclose(g["b"], S.b, rtol=0, atol=tol * np.abs(S.b).max())
    assert abs(g["energy"] - S.energy) <= ENERGY_RTOL * S.energy


def test_ragged_tiles_give_the_same_system(bf, cfg1, cfg1_frames):
    """Tiles of 1100 px split 4800-px frames into 4 full tiles and a ragged 400-px tail."""
    ctx = make_ctx(bf, cfg1)
    poses = perturb(cfg1.gt, 12)
    ids = list(range(cfg1.n_frames))
    a = ctx.build_system(ids, poses, tile_px=1100)
    b = ctx.build_system(ids, poses, tile_px=4800)
    c = ctx.build_system(ids, poses, tile_px=97)
    for x in (a, c):
        np.testing.assert_allclose(x["A"], b["A"], rtol=0, atol=1e-5 * np.abs(b["A"]).max())
        assert x["n_dense"] == b["n_dense"]


# ------------------------------------------------------------------------------ full solves

def compare_solve(res_gpu, poses_gpu, res_or, label):
    e_g = np.array(res_gpu["energy"])
    e_o = np.array(res_or.energy)
    rel = np.abs(e_g - e_o) / np.abs(e_o)
    assert rel.max() <= ENERGY_RTOL, (label, rel)
    for k in range(len(poses_gpu)):
        rot, tr = lie.pose_error(poses_gpu[k], res_or.poses[k])
        assert rot <= ROT_TOL and tr <= TRANS_TOL, (label, k, rot, tr)


def recorded(bf, prob, ids, solve_kw, prm, local=True, ctx=None, frames=None, chunk_id=0, **ctx_kw):
    """The library's solve of frames ids (recorded) and the oracle's solve on its decisions."""
    ctx = ctx or make_ctx(bf, prob, **ctx_kw)
    ids = [int(f) for f in ids]
    if frames is None:
        frames = [ofr.Frame(prob.depth[f], prob.lum[f], prob.intr) for f in ids]
    if local:
        solve = lambda: ctx.solve_local(chunk_id, ids, **solve_kw)  # noqa: E731
    else:
        solve = lambda: ctx.solve_global(ids, **solve_kw)  # noqa: E731
    return replay.recorded_solve(ctx, ids, solve, frames, prob.intr, prob.init[ids],
                                 solver.sparse_pairs_for(prob, ids), prm)


def test_local_solve_matches_oracle(bf, cfg1, cfg1_frames):
    st, poses, ref = recorded(bf, cfg1, range(11), dict(cfg1.solve), oracle_params(cfg1.solve), frames=cfg1_frames)
    compare_solve(st, poses, ref, "cfg1 mixed")
    assert st["r_max_pair"] == tuple(ref.r_max_pair) or abs(st["r_max"] - ref.r_max) < 1e-6
    assert abs(st["r_max"] - ref.r_max) <= 1e-5 * ref.r_max
    assert st["n_dense"] == ref.n_dense
    assert ref.replay.n_flips <= FLIP_BUDGET * ref.replay.n_valid


def test_local_solve_fp32_path_matches_oracle(bf, cfg1, cfg1_frames):
    """The plain FP32 path (FP32 merges and PCG scalars): the same accuracy targets as the mixed
    path, so the two are compared at equal accuracy."""
    st, poses, ref = recorded(bf, cfg1, range(11), dict(cfg1.solve, precision=1), oracle_params(cfg1.solve),
                              frames=cfg1_frames)
    compare_solve(st, poses, ref, "cfg1 plain FP32")


@pytest.mark.parametrize("seed,n", [(5, 3), (6, 7)])
def test_short_chunks_match_oracle(bf, seed, n):
    prob = synth.chunk_problem(seed, n, 80, 60, (50, 120), name=f"chunk{n}")
    st, poses, ref = recorded(bf, prob, range(n), dict(n_gn=3, n_pcg=8, w_dense=0.5),
                              SolveParams(n_gn=3, n_pcg=8, w_dense=0.5))
    compare_solve(st, poses, ref, f"chunk{n}")


def test_batched_equals_alone(bf):
    """Each chunk's result is identical alone and inside a batch (deterministic reductions)."""
    prob = synth.chunk_batch(31, n_chunks=5, W=80, H=60, length=(3, 8), n_corr=(40, 80))
    ctx = make_ctx(bf, prob)
    ids = [c.tolist() for c in prob.chunks]
    batch = ctx.solve_local_batch(list(range(100, 105)), ids, n_gn=3, n_pcg=6)
    pb = [ctx.get_poses(c) for c in ids]
    for k, c in enumerate(ids):
        st = ctx.solve_local(200 + k, c, n_gn=3, n_pcg=6)
        np.testing.assert_array_equal(ctx.get_poses(c), pb[k])
        assert st["energy"] == batch[k]["energy"]


@pytest.fixture(scope="module")
def small_global():
    return synth.global_problem(77, n_kf=48, outer=(12.0, 2.8, 9.0), inner=(6.0, 3.0), n_corr=(40, 100),
                                name="global48")


def test_global_solve_matches_oracle(bf, small_global):
    prob = small_global
    n = prob.n_frames
    st, poses, ref = recorded(bf, prob, range(n), dict(n_gn=4, n_pcg=20, w_dense=0.5),
                              SolveParams(n_gn=4, n_pcg=20, w_dense=0.5), local=False)
    compare_solve(st, poses, ref, "global48")
    assert st["n_pairs"] == len(prob.pairs)


# ------------------------------------------------------------------------- hierarchy, edges

def test_keyframe_composition(bf):
    """Sec. 4.2: chunk members' world poses are the keyframe's global pose composed with the local pose."""
    prob = synth.chunk_batch(41, n_chunks=2, W=80, H=60, length=(4, 4), n_corr=(60, 60))
    ctx = make_ctx(bf, prob)
    c0, c1 = prob.chunks
    ctx.solve_local(0, c0.tolist(), n_gn=2, n_pcg=6)
    loc = ctx.get_poses(c0.tolist())
    np.testing.assert_allclose(loc[0], np.eye(4), atol=0)
    G = np.eye(4)
    G[:3, 3] = [1.0, 2.0, 3.0]
    ctx.add_frames(int(c0[0]), prob.depth[c0[:1]], prob.lum[c0[:1]], init_pose=G[None])
    world = ctx.get_poses(c0.tolist())
    for k in range(len(c0)):
        np.testing.assert_allclose(world[k], hierarchy.compose(G, loc[k]), atol=1e-12)


def test_frame_without_constraints_stays_fixed(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    ctx.add_frames(50, cfg1.depth[:1], cfg1.lum[:1])
    st = ctx.solve_local(1, [0, 1, 2, 50], n_gn=2, n_pcg=5, dense_on=0)
    assert st["flags"] & bf.BF_FLAG_EMPTY_FRAME
    np.testing.assert_allclose(ctx.get_poses([50])[0], np.eye(4), atol=0)


def test_invalid_arguments(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    with pytest.raises(bf.BFError) as e:
        ctx.solve_local(0, [0, 999], n_gn=1)
    assert e.value.status == 4
    with pytest.raises(bf.BFError) as e:
        ctx.add_correspondences(3, 3, np.zeros((2, 3)), np.zeros((2, 3)))
    assert e.value.status == 1
    with pytest.raises(bf.BFError) as e:
        ctx.solve_local(0, [0, 1, 1], n_gn=1)
    assert e.value.status == 1
    with pytest.raises(bf.BFError) as e:
        ctx.solve_local(0, [0, 1], n_gn=bf._lib.BF_MAX_GN + 1)
    assert e.value.status == 1
    # a pair with fewer than 3 correspondences cannot take part in a solve
    n = cfg1.n_frames
    ctx.add_frames(n, cfg1.depth[:2], cfg1.lum[:2])
    ctx.add_correspondences(n, n + 1, np.ones((2, 3), np.float32), np.ones((2, 3), np.float32))
    with pytest.raises(bf.BFError) as e:
        ctx.solve_local(1, [n, n + 1], n_gn=1)
    assert e.value.status == 1
    ctx.add_correspondences(n, n + 1, np.ones((1, 3), np.float32), np.ones((1, 3), np.float32))
    ctx.solve_local(1, [n, n + 1], n_gn=1)  # three now


def test_single_frame_and_empty_solves(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    st = ctx.solve_local(0, [3], n_gn=2)
    assert st["n_pairs"] == 0 and st["energy"] == [0.0, 0.0, 0.0]
    np.testing.assert_allclose(ctx.get_poses([3])[0], np.eye(4))
    st = ctx.solve_local(0, [0, 1], n_gn=0)
    assert len(st["energy"]) == 1


def test_hbm_budget_refuses(bf, cfg1):
    intr = cfg1.intr
    ctx = bf.Context(intr["W"], intr["H"], hbm_budget_bytes=200_000, max_frames_hint=4)
    with pytest.raises(bf.BFError) as e:
        ctx.add_frames(0, cfg1.depth, cfg1.lum)
    assert e.value.status == 2


def test_batch_correspondence_upload_equals_per_pair(bf, cfg1):
    """bf_add_correspondences_batch (host and device inputs) == one bf_add_correspondences per pair."""
    import torch
    ref = make_ctx(bf, cfg1)
    poses = perturb(cfg1.gt, 21)
    ids = list(range(cfg1.n_frames))
    a = ref.build_system(ids, poses)
    pairs = cfg1.pairs.copy()
    pairs[::2] = pairs[::2, ::-1]  # reversed order for half of the pairs: exercises the swap
    pi, pj = cfg1.p_i.copy(), cfg1.p_j.copy()
    for k in range(0, len(pairs), 2):
        s = slice(cfg1.corr_off[k], cfg1.corr_off[k + 1])
        pi[s], pj[s] = cfg1.p_j[s], cfg1.p_i[s]
    for device in (False, True):
        intr = cfg1.intr
        ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"])
        ctx.add_frames(0, cfg1.depth, cfg1.lum)
        if device:
            ctx.add_correspondences_batch(pairs, cfg1.corr_off, torch.from_numpy(pi).cuda(),
                                          torch.from_numpy(pj).cuda())
        else:
            ctx.add_correspondences_batch(pairs, cfg1.corr_off, pi, pj)
        b = ctx.build_system(ids, poses)
        np.testing.assert_array_equal(a["A"], b["A"])
        np.testing.assert_array_equal(a["b"], b["b"])


def test_profiling_counts_launches(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    ctx.reset_profile()
    ctx.set_profiling(True)
    ctx.solve_local(0, list(range(11)), n_gn=2, n_pcg=4)
    p = ctx.profile()
    k = p["kernels"]
    # one pair-transform launch, then per GN iteration dense, sparse, merge, assemble and PCG (which
    # also records the energy, updates the poses and refreshes the transforms); a final energy pass
    assert k["dense"]["count"] == 3 and k["pcg"]["count"] == 2 and k["energy"]["count"] == 1
    assert k["xform"]["count"] == 1 and k["update"]["count"] == 0
    assert p["launches"] == sum(v["count"] for v in k.values())
    assert k["dense"]["ms"] > 0


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_pcg_variants_agree(bf, small_global, variant):
    """Per-problem CTA, grid-cooperative and cluster PCG kernels solve the same system to rounding.

    The variants group the FP32 products of each dot product into warps differently, so alpha and
    beta differ in their last FP32 bits; over 2 x 15 PCG iterations on this loop the poses move by up
    to about 6e-6; the variants must agree within the oracle tolerance (1e-5), which each meets."""
    prob = small_global
    n = prob.n_frames
    ctx = make_ctx(bf, prob)
    ref = ctx.solve_global(list(range(n)), n_gn=2, n_pcg=15, pcg_variant=1)
    P_ref = ctx.get_poses(list(range(n)))
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    st = ctx.solve_global(list(range(n)), n_gn=2, n_pcg=15, pcg_variant=variant)
    P = ctx.get_poses(list(range(n)))
    for k in range(n):
        rot, tr = lie.pose_error(P[k], P_ref[k])
        assert rot < TRANS_TOL and tr < TRANS_TOL, (k, rot, tr)
    np.testing.assert_allclose(st["energy"], ref["energy"], rtol=1e-6)


def test_graph_replay_equals_direct_launches(bf, small_global):
    """The captured Gauss-Newton graph gives bitwise the same result as kernel-by-kernel launches,
    on capture and on replay with new initial poses (the graph reads them from the workspace)."""
    prob = small_global
    n = prob.n_frames
    ids = list(range(n))
    ctx = make_ctx(bf, prob)
    init2 = perturb(prob.init, 5, 0.002, 0.005)
    for init in (prob.init, init2, prob.init):
        ctx.add_frames(0, prob.depth, prob.lum, init_pose=init)
        a = ctx.solve_global(ids, n_gn=3, n_pcg=10, use_graph=0)
        Pa = ctx.get_poses(ids)
        ctx.add_frames(0, prob.depth, prob.lum, init_pose=init)
        b = ctx.solve_global(ids, n_gn=3, n_pcg=10, use_graph=1)
        Pb = ctx.get_poses(ids)
        np.testing.assert_array_equal(Pa, Pb)
        assert a["energy"] == b["energy"]


def test_staged_and_tiled_dense_kernels_agree(bf, cfg1):
    """Automatic decomposition (target frame staged in shared memory by TMA bulk copies) and the
    tiled kernel build the same normal equations up to FP32 summation order."""
    ctx = make_ctx(bf, cfg1)
    poses = perturb(cfg1.gt, 23)
    ids = list(range(cfg1.n_frames))
    staged = ctx.build_system(ids, poses, tile_px=0)
    tiled = ctx.build_system(ids, poses, tile_px=4800)
    assert staged["n_dense"] == tiled["n_dense"]
    np.testing.assert_allclose(staged["A"], tiled["A"], rtol=0, atol=1e-5 * np.abs(tiled["A"]).max())
    np.testing.assert_allclose(staged["b"], tiled["b"], rtol=0, atol=1e-5 * np.abs(tiled["b"]).max())
    assert abs(staged["energy"] - tiled["energy"]) <= 1e-6 * tiled["energy"]


@pytest.fixture(scope="module")
def batch320():
    return synth.chunk_batch(57, n_chunks=6, W=320, H=240, length=(3, 5), n_corr=(100, 200), name="batch320")


def test_batched_chunks_320x240_match_oracle(bf, batch320):
    """Full-resolution chunks (320x240, tiled dense kernel) solved in one batch (CUDA graph); the two
    smallest chunks are solved again alone with the association recorded (bitwise the batch's
    result) and checked against the oracle's solve on those decisions."""
    prob = batch320
    ctx = make_ctx(bf, prob, max_frames_hint=prob.n_frames)
    lists = [c.tolist() for c in prob.chunks]
    kw = dict(n_gn=3, n_pcg=8)
    stats = ctx.solve_local_batch(list(range(len(lists))), lists, use_graph=1, **kw)
    P_batch = [ctx.get_poses(lst) for lst in lists]
    order = sorted(range(len(lists)), key=lambda k: len(lists[k]))[:2]
    for k in order:
        st, poses, ref = recorded(bf, prob, lists[k], kw, SolveParams(**kw), ctx=ctx, chunk_id=1000 + k)
        np.testing.assert_array_equal(poses, P_batch[k])
        assert st["energy"] == stats[k]["energy"]
        compare_solve(st, poses, ref, f"chunk {k} at 320x240")
        assert ref.replay.n_flips <= FLIP_BUDGET * ref.replay.n_valid


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_waits_give_up_and_the_context_survives(bf, cfg1, which):
    """Failure detection without a fault: a wait on a flag nothing sets (0), an mbarrier nothing
    arrives on (1) or a work-queue slot nothing publishes (2) ends after its poll limit with
    BF_ERR_TIMEOUT; the same context then solves."""
    ctx = make_ctx(bf, cfg1)
    status, gave_up = ctx.selftest_wait_timeout(which, 1 << 14)
    assert status == 6 and gave_up == 1  # BF_ERR_TIMEOUT
    st = ctx.solve_local(0, list(range(11)), n_gn=1, n_pcg=4)
    assert st["n_gn"] == 1 and np.isfinite(st["energy"]).all()


def test_workspace_growth_reuploads_tables(bf):
    """A solve that needs a larger workspace than the previous one (here: the grid-cooperative PCG
    after the cluster PCG) gets its tables uploaded again even if the new allocation lands at the
    old address; its result equals the same solve on a fresh context."""
    prob = synth.cfg2()
    n = prob.n_frames

    def ctx_for():
        intr = prob.intr
        c = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], max_frames_hint=n)
        c.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
        c.add_correspondences_batch(prob.pairs, prob.corr_off, prob.p_i, prob.p_j)
        return c

    kw = dict(n_gn=2, n_pcg=5, w_dense=0.5)
    ref = ctx_for().solve_global(list(range(n)), pcg_variant=2, **kw)
    ctx = ctx_for()
    ctx.reset_profile()
    ctx.set_profiling(True)
    ctx.solve_global(list(range(n)), pcg_variant=3, **kw)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    st = ctx.solve_global(list(range(n)), pcg_variant=2, **kw)
    assert st["energy"] == ref["energy"] and st["flags"] == 0


def test_autotuned_decomposition(bf, cfg1, cfg1_frames):
    """tile_px = BF_TILE_AUTOTUNE times the candidate decompositions once, keeps the fastest, and
    then gives the same result as asking for that decomposition explicitly; the solve matches the
    oracle like any other."""
    ctx = make_ctx(bf, cfg1)
    assert ctx.tuned_tile_px() is None
    st, poses, ref = recorded(bf, cfg1, range(11), dict(cfg1.solve, tile_px=bf._lib.BF_TILE_AUTOTUNE),
                              oracle_params(cfg1.solve), ctx=ctx, frames=cfg1_frames)
    chosen = ctx.tuned_tile_px()
    assert chosen == 0 or 256 <= chosen <= 4800
    compare_solve(st, poses, ref, "autotuned")
    again = make_ctx(bf, cfg1).solve_local(0, list(range(11)), tile_px=chosen, **dict(cfg1.solve))
    assert again["energy"] == st["energy"]
