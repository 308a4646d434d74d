"""GPU parity of the persistent batched solve (one launch for the whole Gauss-Newton loop of a
batch of chunks, its CTAs fed by a device work queue).

Every work item runs the same device code as the launch sequence, and every partial sum is
written to a fixed slot and merged in a fixed order, so the persistent launch must reproduce the
launch sequence bit for bit, whatever order the queue hands the items out in; against the FP64
oracle it then meets the accuracy targets (1e-4 rad, 1e-5 m, 1e-5 relative energy) like the
launch sequence does.
"""
import numpy as np
import pytest

import replay
import synth
from oracle import frames as ofr, lie, solver
from oracle.system import SolveParams

pytestmark = pytest.mark.gpu

ROT_TOL, TRANS_TOL, ENERGY_RTOL = 1e-4, 1e-5, 1e-5


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


@pytest.fixture(scope="module")
def batch80():
    return synth.chunk_batch(31, n_chunks=7, W=80, H=60, length=(3, 9), n_corr=(40, 120), name="batch80")


@pytest.fixture(scope="module")
def batch320():
    return synth.chunk_batch(57, n_chunks=6, W=320, H=240, length=(3, 5), n_corr=(100, 200), name="batch320")


def make_ctx(bf, prob, **kw):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                     max_frames_hint=prob.n_frames, **kw)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    for k, (i, j) in enumerate(prob.pairs):
        p, q = prob.pair_corr(k)
        ctx.add_correspondences(int(i), int(j), p, q)
    return ctx


def solve_batch(ctx, prob, **kw):
    lists = [c.tolist() for c in prob.chunks]
    stats = ctx.solve_local_batch(list(range(len(lists))), lists, **kw)
    return stats, [ctx.get_poses(c) for c in lists]


def assert_bitwise(a, b):
    (sa, pa), (sb, pb) = a, b
    for k in range(len(sa)):
        assert sa[k]["energy"] == sb[k]["energy"], k
        assert sa[k]["n_dense"] == sb[k]["n_dense"], k
        assert sa[k]["r_max"] == sb[k]["r_max"], k
        assert sa[k]["flags"] == sb[k]["flags"], k
        np.testing.assert_array_equal(pa[k], pb[k])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("graph", [0, 1])
def test_persistent_equals_launch_sequence_80x60(bf, batch80, precision, graph):
    kw = dict(n_gn=3, n_pcg=8, w_dense=0.5, tile_px=1200, precision=precision, use_graph=graph)
    ctx = make_ctx(bf, batch80)
    ref = solve_batch(ctx, batch80, **kw)
    ctx.reset_profile()
    ctx.set_profiling(graph == 0)
    got = solve_batch(ctx, batch80, persistent=1, **kw)
    assert_bitwise(got, ref)
    if graph == 0:
        k = ctx.profile()["kernels"]
        assert k["batch"]["count"] == 1
        assert k["dense"]["count"] == 0 and k["pcg"]["count"] == 0 and k["merge"]["count"] == 0


@pytest.mark.parametrize("storage", [0, 1])
def test_persistent_equals_launch_sequence_320x240(bf, batch320, storage):
    kw = dict(n_gn=3, n_pcg=8, tile_px=19200)
    ctx = make_ctx(bf, batch320, storage=storage)
    ref = solve_batch(ctx, batch320, **kw)
    got = solve_batch(ctx, batch320, persistent=1, **kw)
    assert_bitwise(got, ref)


def test_persistent_repeatable(bf, batch80):
    """The queue hands items out in a different order on every run; the results must not change."""
    ctx = make_ctx(bf, batch80)
    first = solve_batch(ctx, batch80, n_gn=2, n_pcg=6, tile_px=600, persistent=1)
    for _ in range(4):
        assert_bitwise(solve_batch(ctx, batch80, n_gn=2, n_pcg=6, tile_px=600, persistent=1), first)


def test_persistent_matches_oracle(bf, batch320):
    """The persistent launch on 320x240 chunks; the two smallest chunks are solved again alone with
    the association recorded (bitwise the persistent result, same tiles) and checked against the
    oracle's solve on those decisions."""
    prob = batch320
    ctx = make_ctx(bf, prob)
    kw = dict(n_gn=3, n_pcg=8, tile_px=19200)
    stats, poses = solve_batch(ctx, prob, persistent=1, use_graph=1, **kw)
    lists = [c.tolist() for c in prob.chunks]
    prm = SolveParams(n_gn=3, n_pcg=8)
    for k in sorted(range(len(lists)), key=lambda k: len(lists[k]))[:2]:
        ids = lists[k]
        fr = [ofr.Frame(prob.depth[f], prob.lum[f], prob.intr) for f in ids]
        st, P, ref = replay.recorded_solve(ctx, ids, lambda: ctx.solve_local(2000 + k, ids, **kw), fr, prob.intr,
                                           prob.init[ids], solver.sparse_pairs_for(prob, ids), prm)
        assert st["energy"] == stats[k]["energy"]
        np.testing.assert_array_equal(P, poses[k])
        rel = np.abs(np.array(st["energy"]) - ref.energy) / np.abs(ref.energy)
        assert rel.max() <= ENERGY_RTOL, (k, rel)
        for f in range(len(ids)):
            rot, tr = lie.pose_error(P[f], ref.poses[f])
            assert rot <= ROT_TOL and tr <= TRANS_TOL, (k, f, rot, tr)


def test_persistent_edge_cases(bf, batch80):
    """A one-frame chunk (no pairs: its stages go straight to the solve), n_gn = 0 (only the final
    energy), and a dense-free solve (sparse segments only) inside the same kind of batch."""
    ctx = make_ctx(bf, batch80)
    lists = [c.tolist() for c in batch80.chunks]
    lists_1 = lists[:3] + [[lists[3][0]]] + lists[4:]
    ids = list(range(len(lists_1)))
    for kw in (dict(n_gn=2, n_pcg=5), dict(n_gn=0, n_pcg=5), dict(n_gn=2, n_pcg=5, dense_on=0)):
        ref = ctx.solve_local_batch(ids, lists_1, tile_px=1200, **kw)
        pref = [ctx.get_poses(c) for c in lists_1]
        got = ctx.solve_local_batch(ids, lists_1, tile_px=1200, persistent=1, **kw)
        pgot = [ctx.get_poses(c) for c in lists_1]
        assert_bitwise((got, pgot), (ref, pref))
        assert got[3]["n_gn"] == kw["n_gn"] and len(got[3]["energy"]) == kw["n_gn"] + 1


def test_persistent_falls_back_where_it_does_not_apply(bf, batch80):
    """With the target frame staged in shared memory (tile_px = 0 at 80x60) the launch sequence runs."""
    ctx = make_ctx(bf, batch80)
    ctx.reset_profile()
    ctx.set_profiling(True)
    solve_batch(ctx, batch80, n_gn=2, n_pcg=5, persistent=1)
    k = ctx.profile()["kernels"]
    assert k["batch"]["count"] == 0 and k["dense"]["count"] == 3
