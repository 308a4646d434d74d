"""GPU checks of the solve-table reuse: a context keeps the last tables it built and reuses them
(with the new initial poses) for a solve over the same problems, pairs, frame slots, dense
decomposition and dense set E (Sec. 4.3's angle test at the new initial poses).  Whatever the
reuse decides, every solve must equal, bit for bit, the same solve in a fresh context, which
builds its tables from scratch: after repeats, after a pair is removed or correspondences are
added, after initial poses that change E, and when problems of the same sizes alternate (the
captured graph must follow the tables, not only their sizes).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

KW = dict(n_gn=3, n_pcg=8, w_dense=0.5)


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


@pytest.fixture(scope="module")
def prob():
    return synth.chunk_problem(4401, 9, 80, 60, (60, 120), name="cache9")


def make_ctx(bf, prob, init=None, skip=()):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], max_frames_hint=prob.n_frames)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init if init is None else init)
    for k, (i, j) in enumerate(prob.pairs):
        if (int(i), int(j)) in skip:
            continue
        p, q = prob.pair_corr(k)
        ctx.add_correspondences(int(i), int(j), p, q)
    return ctx


def solve(ctx, prob, ids, init=None, graph=1):
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init if init is None else init)
    st = ctx.solve_global(ids, use_graph=graph, **KW)
    return st, ctx.get_poses(ids)


def fresh(bf, prob, ids, init=None, skip=(), graph=1):
    ctx = make_ctx(bf, prob, init, skip)
    out = solve(ctx, prob, ids, init, graph)
    ctx.close()
    return out


def assert_same(a, b):
    (sa, pa), (sb, pb) = a, b
    assert sa["energy"] == sb["energy"]
    assert sa["n_dense"] == sb["n_dense"] and sa["flags"] == sb["flags"]
    np.testing.assert_array_equal(pa, pb)


@pytest.mark.parametrize("graph", [0, 1])
def test_repeated_solves_equal_a_fresh_context(bf, prob, graph):
    ids = list(range(prob.n_frames))
    ref = fresh(bf, prob, ids, graph=graph)
    ctx = make_ctx(bf, prob)
    for _ in range(3):
        assert_same(solve(ctx, prob, ids, graph=graph), ref)


def test_removed_pair_and_new_correspondences_rebuild(bf, prob):
    ids = list(range(prob.n_frames))
    ctx = make_ctx(bf, prob)
    solve(ctx, prob, ids)
    i, j = (int(x) for x in prob.pairs[3])
    ctx.remove_pair(i, j)
    assert_same(solve(ctx, prob, ids), fresh(bf, prob, ids, skip={(i, j)}))
    # the pair's correspondences back, appended as a new segment
    p, q = prob.pair_corr(3)
    ctx.add_correspondences(i, j, p, q)
    got = solve(ctx, prob, ids)
    ref_ctx = make_ctx(bf, prob, skip={(i, j)})
    ref_ctx.add_correspondences(i, j, p, q)
    assert_same(got, solve(ref_ctx, prob, ids))


def test_initial_poses_that_change_the_dense_set_rebuild(bf, prob):
    """Frame 4 turned by 90 degrees about its x axis: its pairs leave E (max angle 30 degrees)."""
    ids = list(range(prob.n_frames))
    init2 = prob.init.copy()
    c, s = np.cos(np.pi / 2), np.sin(np.pi / 2)
    init2[4, :3, :3] = init2[4, :3, :3] @ np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    ctx = make_ctx(bf, prob)
    a = solve(ctx, prob, ids)
    b = solve(ctx, prob, ids, init=init2)
    assert b[0]["n_dense"] < a[0]["n_dense"]
    assert_same(b, fresh(bf, prob, ids, init=init2))
    assert_same(solve(ctx, prob, ids), a)


def test_alternating_problems_of_equal_size(bf, prob):
    """Two 5-frame subsets (every pair matched, so equal table sizes) solved in turn, graph on."""
    s1, s2 = [0, 1, 2, 3, 4], [4, 5, 6, 7, 8]
    r1, r2 = fresh(bf, prob, s1), fresh(bf, prob, s2)
    ctx = make_ctx(bf, prob)
    for _ in range(2):
        assert_same(solve(ctx, prob, s1), r1)
        assert_same(solve(ctx, prob, s2), r2)


def test_reuploaded_correspondences(bf, prob):
    """Cleared and uploaded again: in the same layout (the tables may be reused, the points are
    read afresh) and in reversed pair order (a different layout); both equal a fresh context
    loaded the same way."""
    ids = list(range(prob.n_frames))
    ctx = make_ctx(bf, prob)
    ref = solve(ctx, prob, ids)
    order = list(range(len(prob.pairs)))
    for rev in (False, True, False):
        ks = order[::-1] if rev else order
        ctx.clear_correspondences()
        for k in ks:
            i, j = (int(x) for x in prob.pairs[k])
            p, q = prob.pair_corr(k)
            ctx.add_correspondences(i, j, p, q)
        got = solve(ctx, prob, ids)
        if not rev:
            assert_same(got, ref)
        else:
            fresh_ctx = make_ctx(bf, prob, skip={(int(i), int(j)) for i, j in prob.pairs})
            for k in ks:
                i, j = (int(x) for x in prob.pairs[k])
                p, q = prob.pair_corr(k)
                fresh_ctx.add_correspondences(i, j, p, q)
            assert_same(got, solve(fresh_ctx, prob, ids))


def test_new_points_in_the_same_layout_are_used(bf, prob):
    """Points moved by 2 mm and uploaded into the same layout: the solve sees the new points (it
    equals a fresh context loaded with them and differs from the solve on the old ones)."""
    ids = list(range(prob.n_frames))
    ctx = make_ctx(bf, prob)
    old = solve(ctx, prob, ids)
    ctx.clear_correspondences()
    fresh_ctx = make_ctx(bf, prob, skip={(int(i), int(j)) for i, j in prob.pairs})
    for k, (i, j) in enumerate(prob.pairs):
        p, q = prob.pair_corr(k)
        p = p + np.float32(0.002)
        ctx.add_correspondences(int(i), int(j), p, q)
        fresh_ctx.add_correspondences(int(i), int(j), p, q)
    got = solve(ctx, prob, ids)
    assert_same(got, solve(fresh_ctx, prob, ids))
    assert got[0]["energy"] != old[0]["energy"]


def test_failed_solve_leaves_the_cache_usable(bf, prob):
    """A solve that the table build rejects (a pair with 2 correspondences: Sec. 4.1.1 needs 3),
    then the pair removed: the next solves equal a fresh context's."""
    ids = list(range(prob.n_frames))
    ref = fresh(bf, prob, ids)
    ctx = make_ctx(bf, prob)
    assert_same(solve(ctx, prob, ids), ref)
    # the first pair keeps only 2 of its correspondences
    i, j = (int(x) for x in prob.pairs[0])
    ctx.remove_pair(i, j)
    p, q = prob.pair_corr(0)
    ctx.add_correspondences(i, j, p[:2], q[:2])
    with pytest.raises(bf.BFError):
        solve(ctx, prob, ids)
    ctx.remove_pair(i, j)
    ctx.add_correspondences(i, j, p, q)
    assert_same(solve(ctx, prob, ids), ref)
    assert_same(solve(ctx, prob, ids), ref)
