"""GPU parity of the matrix-free sparse term (Sec. 4.4: J p, then J^T (J p) every PCG iteration).

The matrix-free product and the assembled 6x6 sparse blocks are the same linear operator, so the
two modes must give the same Gauss-Newton steps up to FP32 rounding (compared like the PCG kernel
variants: 1e-5 in the poses, 1e-6 relative in the energies), and both must meet the accuracy
targets against the FP64 oracle, which assembles the normal equations explicitly (on the library's
association decisions, checked against its own: tests/replay.py).
"""
import numpy as np
import pytest

import replay
import synth
from oracle import frames as ofr, lie, solver
from oracle.system import SolveParams

pytestmark = pytest.mark.gpu

MATFREE = 1
ROT_TOL, TRANS_TOL, ENERGY_RTOL = 1e-4, 1e-5, 1e-5


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
def small_global():
    return synth.global_problem(77, n_kf=48, outer=(12.0, 2.8, 9.0), inner=(6.0, 3.0), n_corr=(40, 100),
                                name="global48")


def make_ctx(bf, prob):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"])
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    for k, (i, j) in enumerate(prob.pairs):
        p, q = prob.pair_corr(k)
        ctx.add_correspondences(int(i), int(j), p, q)
    return ctx


def solve_both(bf, prob, solve, ids, **kw):
    """The same problem solved with assembled sparse blocks and matrix-free, from the same start."""
    ctx = make_ctx(bf, prob)
    ref = solve(ctx, ids, **kw)
    P_ref = ctx.get_poses(ids)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    st = solve(ctx, ids, sparse_mode=MATFREE, **kw)
    return ref, P_ref, st, ctx.get_poses(ids)


def assert_same_steps(ref, P_ref, st, P):
    for k in range(len(P)):
        rot, tr = lie.pose_error(P[k], P_ref[k])
        assert rot < 1e-5 and tr < 1e-5, (k, rot, tr)
    np.testing.assert_allclose(st["energy"], ref["energy"], rtol=1e-6)


def compare_oracle(st, P, ref, label):
    rel = np.abs(np.array(st["energy"]) - ref.energy) / np.abs(ref.energy)
    assert rel.max() <= ENERGY_RTOL, (label, rel)
    for k in range(len(P)):
        rot, tr = lie.pose_error(P[k], ref.poses[k])
        assert rot <= ROT_TOL and tr <= TRANS_TOL, (label, k, rot, tr)


def glob(ctx, ids, **kw):
    return ctx.solve_global(ids, **kw)


def loc(ctx, ids, **kw):
    return ctx.solve_local(0, ids, **kw)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_matfree_equals_blocks_global(bf, small_global, variant):
    """47 free keyframes: AUTO and GRID run the grid-cooperative kernel, CTA the per-problem one;
    the assembled-blocks reference runs on the same kernel."""
    ids = list(range(small_global.n_frames))
    ref_variant = 2 if variant == 0 else variant
    ctx = make_ctx(bf, small_global)
    ref = ctx.solve_global(ids, n_gn=2, n_pcg=15, pcg_variant=ref_variant)
    P_ref = ctx.get_poses(ids)
    ctx.add_frames(0, small_global.depth, small_global.lum, init_pose=small_global.init)
    st = ctx.solve_global(ids, n_gn=2, n_pcg=15, pcg_variant=variant, sparse_mode=MATFREE)
    assert_same_steps(ref, P_ref, st, ctx.get_poses(ids))


def test_matfree_sparse_only_equals_blocks(bf, small_global):
    """Without the dense term the whole operator is matrix-free (the assembled blocks are zero)."""
    ids = list(range(small_global.n_frames))
    ref, P_ref, st, P = solve_both(bf, small_global, glob, ids, n_gn=3, n_pcg=20, dense_on=0, pcg_variant=2)
    assert_same_steps(ref, P_ref, st, P)


def test_matfree_chunk_equals_blocks(bf, cfg1):
    """Chunk (10 free frames): blocks take the shared-memory dense path, matrix-free the general one."""
    ids = list(range(cfg1.n_frames))
    ref, P_ref, st, P = solve_both(bf, cfg1, loc, ids, **cfg1.solve)
    assert_same_steps(ref, P_ref, st, P)


def test_matfree_global_matches_oracle(bf, small_global):
    prob = small_global
    n = prob.n_frames
    fr = [ofr.Frame(prob.depth[k], prob.lum[k], prob.intr) for k in range(n)]
    ctx = make_ctx(bf, prob)
    ids = list(range(n))
    st, P, ref = replay.recorded_solve(
        ctx, ids, lambda: ctx.solve_global(ids, n_gn=4, n_pcg=20, w_dense=0.5, sparse_mode=MATFREE), fr, prob.intr,
        prob.init, solver.sparse_pairs_for(prob, ids), SolveParams(n_gn=4, n_pcg=20, w_dense=0.5))
    compare_oracle(st, P, ref, "global48 matrix-free")


def test_matfree_chunk_matches_oracle(bf, cfg1):
    n = cfg1.n_frames
    fr = [ofr.Frame(cfg1.depth[k], cfg1.lum[k], cfg1.intr) for k in range(n)]
    d = cfg1.solve
    prm = SolveParams(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"],
                      w_photo=d["w_photo"], w_geo=d["w_geo"])
    ctx = make_ctx(bf, cfg1)
    ids = list(range(n))
    st, P, ref = replay.recorded_solve(ctx, ids, lambda: ctx.solve_local(0, ids, sparse_mode=MATFREE, **d), fr,
                                       cfg1.intr, cfg1.init, solver.sparse_pairs_for(cfg1, ids), prm)
    compare_oracle(st, P, ref, "cfg1 matrix-free")


def test_matfree_rejects_cluster_kernel_and_unknown_modes(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    for kw in ({"sparse_mode": MATFREE, "pcg_variant": 3}, {"sparse_mode": 7}):
        with pytest.raises(bf.BFError) as e:
            ctx.solve_local(0, list(range(cfg1.n_frames)), n_gn=1, **kw)
        assert e.value.status == 1
