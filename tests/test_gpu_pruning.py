"""GPU parity of the Sec. 4.4.1 correspondence pruning loop against the oracle.

Chunks of 80x60 frames with 5 mm correspondence noise and no random outliers, plus one pair
whose matches are half wrong (shifted 0.3 m in frame j: no rigid motion explains them).  Both
sides must remove the same pairs in the same order and end at the same poses (within the
accuracy targets), and frames left without pairs are reported invalid.
"""
import copy

import numpy as np
import pytest

import replay
import synth
from oracle import frames as ofr, lie, solver
from oracle.system import SolveParams

pytestmark = pytest.mark.gpu

PRUNE = 0.05  # Sec. 4.4.1


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


def corrupt(prob, pair):
    """Copy of prob with half the matches of `pair` moved 0.3 m in camera j."""
    out = copy.copy(prob)
    out.p_j = prob.p_j.copy()
    k = [tuple(map(int, p)) for p in prob.pairs].index(pair)
    a, b = prob.corr_off[k], prob.corr_off[k + 1]
    out.p_j[a:b:2] += np.array([0.0, 0.3, 0.0], dtype=np.float32)
    return out


def make_ctx(bf, prob):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"])
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    for k, (i, j) in enumerate(prob.pairs):
        p, q = prob.pair_corr(k)
        ctx.add_correspondences(int(i), int(j), p, q)
    return ctx


@pytest.fixture(scope="module")
def bad_chunk():
    prob = synth.chunk_problem(91, 6, 80, 60, (60, 120), sigma=0.005, outlier_frac=0.0, name="chunk6_prune")
    return corrupt(prob, (1, 4))


def test_pruning_matches_oracle(bf, bad_chunk):
    prob = bad_chunk
    n = prob.n_frames
    fr = [ofr.Frame(prob.depth[k], prob.lum[k], prob.intr) for k in range(n)]
    prm = SolveParams(n_gn=4, n_pcg=12, w_dense=0.5)
    rep = replay.from_ctx(make_ctx(bf, prob), range(n), prob.intr["W"], prob.intr["H"])
    ref = solver.gauss_newton_pruned(fr, prob.intr, prob.init, solver.sparse_pairs_for(prob, range(n)), prm, PRUNE,
                                     assoc=rep)
    assert ref.pruned == [(1, 4)] and ref.rounds == 2  # the scenario does what it is meant to
    ctx = make_ctx(bf, prob)
    st = ctx.solve_local(3, list(range(n)), n_gn=4, n_pcg=12, w_dense=0.5, prune_rmax=PRUNE)
    assert st["pruned"] == ref.pruned and st["solves"] == ref.rounds and st["invalid"] == ref.invalid
    assert st["r_max"] <= PRUNE
    e = np.array(st["energy"])
    assert np.abs(e - ref.result.energy).max() <= 1e-5 * np.abs(ref.result.energy).max()
    P = ctx.get_poses(list(range(n)))
    for k in range(n):
        rot, tr = lie.pose_error(P[k], ref.result.poses[k])
        assert rot <= 1e-4 and tr <= 1e-5, (k, rot, tr)
    # the pair is gone from the context: solving again prunes nothing
    st2 = ctx.solve_local(3, list(range(n)), n_gn=4, n_pcg=12, w_dense=0.5, prune_rmax=PRUNE)
    assert st2["pruned"] == [] and st2["solves"] == 1


def test_batch_prunes_only_the_chunk_that_needs_it(bf, bad_chunk):
    """Three chunks in one batch, one with a false pair: only that chunk is re-solved; the others
    keep exactly (bitwise) their unpruned result."""
    good = [synth.chunk_problem(s, 5, 80, 60, (60, 120), sigma=0.005, outlier_frac=0.0) for s in (92, 93)]
    probs = [good[0], bad_chunk, good[1]]
    intr = bad_chunk.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"])
    base = 0
    lists = []
    for pr in probs:
        ctx.add_frames(base, pr.depth, pr.lum)
        for k, (i, j) in enumerate(pr.pairs):
            p, q = pr.pair_corr(k)
            ctx.add_correspondences(base + int(i), base + int(j), p, q)
        lists.append(list(range(base, base + pr.n_frames)))
        base += pr.n_frames
    kw = dict(n_gn=4, n_pcg=12, w_dense=0.5)
    plain = ctx.solve_local_batch([10, 11, 12], lists, **kw)
    P_plain = [ctx.get_poses(l) for l in lists]
    st = ctx.solve_local_batch([10, 11, 12], lists, prune_rmax=PRUNE, **kw)
    off = lists[1][0]
    assert [s["solves"] for s in st] == [1, 2, 1]
    assert st[1]["pruned"] == [(off + 1, off + 4)] and st[0]["pruned"] == [] and st[2]["pruned"] == []
    for c in (0, 2):
        np.testing.assert_array_equal(ctx.get_poses(lists[c]), P_plain[c])
        assert st[c]["energy"] == plain[c]["energy"]


def test_frame_left_without_pairs_is_invalid(bf):
    """A frame tied to the chunk by a single bad pair becomes invalid and stays where it started."""
    prob = synth.chunk_problem(94, 5, 80, 60, (60, 120), sigma=0.005, outlier_frac=0.0)
    keep = [k for k, (i, j) in enumerate(prob.pairs) if not (j == 4 and i != 3)]
    sub = copy.copy(prob)
    sub.pairs = prob.pairs[keep]
    sub.corr_off = np.concatenate([[0], np.cumsum([prob.corr_off[k + 1] - prob.corr_off[k] for k in keep])])
    sub.p_i = np.concatenate([prob.pair_corr(k)[0] for k in keep])
    sub.p_j = np.concatenate([prob.pair_corr(k)[1] for k in keep])
    sub = corrupt(sub, (3, 4))
    ctx = make_ctx(bf, sub)
    st = ctx.solve_local(5, list(range(5)), n_gn=3, n_pcg=10, w_dense=0.5, prune_rmax=PRUNE)
    assert st["pruned"] == [(3, 4)] and st["invalid"] == [4] and st["n_invalid"] == 1
    np.testing.assert_array_equal(ctx.get_poses([4])[0], np.eye(4))  # local solves start at identity
