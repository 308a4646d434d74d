"""Serving: continuous batching on a persistent context (bf_serve_start / bf_submit / bf_wait)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available()
    import paper_1604_01093_b300 as bf
    return bf


@pytest.fixture(scope="module")
def chunks():
    return synth.chunk_batch(91, n_chunks=12, W=80, H=60, length=(3, 9), n_corr=(50, 120), name="serve")


def make_ctx(bf, prob, **kw):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], **kw)
    ctx.add_frames(0, prob.depth, prob.lum)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, prob.p_i, prob.p_j)
    return ctx


def test_each_result_is_the_same_alone_and_in_the_mix(bf, chunks):
    lists = [c.tolist() for c in chunks.chunks]
    alone = make_ctx(bf, chunks)
    ref_stats, ref_poses = [], []
    for k, ids in enumerate(lists):
        ref_stats.append(alone.solve_local(k, ids, n_gn=3, n_pcg=8))
        ref_poses.append(alone.get_poses(ids))
    ctx = make_ctx(bf, chunks)
    ctx.serve_start(n_slots=2, max_batch=5)
    tickets = [ctx.submit(ids, chunk_id=k, n_gn=3, n_pcg=8) for k, ids in enumerate(lists)]
    for k, t in enumerate(tickets):
        code, st = ctx.wait(t, timeout_ms=60000)
        assert code == 0, code
        assert st["energy"] == ref_stats[k]["energy"]
        assert st["ms"] > 0
        np.testing.assert_array_equal(ctx.get_poses(lists[k]), ref_poses[k])
    ctx.serve_stop()


def test_global_request_and_mixed_queue(bf, chunks):
    lists = [c.tolist() for c in chunks.chunks]
    keyframes = [ids[0] for ids in lists[:6]]
    ctx = make_ctx(bf, chunks)
    ctx.serve_start(n_slots=2, max_batch=4)
    t_local = [ctx.submit(ids, chunk_id=k, n_gn=2, n_pcg=6) for k, ids in enumerate(lists[:6])]
    for t in t_local:
        assert ctx.wait(t, 60000)[0] == 0
    t_glob = ctx.submit(keyframes, kind=bf._lib.BF_REQ_GLOBAL, n_gn=2, n_pcg=6, dense_on=0)
    code, st = ctx.wait(t_glob, 60000)
    assert code == 0 and st["n_frames"] == len(keyframes)
    assert ctx.wait(t_glob, 0)[0] == 4  # collected already
    ctx.serve_stop()


def test_poll_timeout_and_full_queue(bf, chunks):
    lists = [c.tolist() for c in chunks.chunks]
    ctx = make_ctx(bf, chunks)
    ctx.serve_start(n_slots=1, max_batch=1, max_queue=4)
    tickets, busy = [], 0
    for r in range(60):
        try:
            tickets.append(ctx.submit(lists[r % len(lists)], chunk_id=r, n_gn=4, n_pcg=10))
        except bf.BFError as e:
            assert e.status == 7  # BF_ERR_BUSY
            busy += 1
    assert busy > 0
    assert ctx.wait(tickets[-1], 0)[0] in (0, 6)
    for t in tickets:
        assert ctx.wait(t, 60000)[0] == 0
    ctx.serve_stop()


def test_budget_refusal_completes_with_out_of_memory(bf, chunks):
    lists = [c.tolist() for c in chunks.chunks]
    intr = chunks.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                     max_frames_hint=chunks.n_frames)
    ctx.add_frames(0, chunks.depth, chunks.lum)
    ctx.add_correspondences_batch(chunks.pairs, chunks.corr_off, chunks.p_i, chunks.p_j)
    used = ctx.device_bytes()
    ctx.close()
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                     max_frames_hint=chunks.n_frames, hbm_budget_bytes=used + 1024)
    ctx.add_frames(0, chunks.depth, chunks.lum)
    ctx.add_correspondences_batch(chunks.pairs, chunks.corr_off, chunks.p_i, chunks.p_j)
    ctx.serve_start(n_slots=1)
    t = ctx.submit(lists[0], chunk_id=0, n_gn=2)
    assert ctx.wait(t, 60000)[0] == 2  # BF_ERR_OUT_OF_MEMORY
    ctx.serve_stop()
