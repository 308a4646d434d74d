"""The allocation-free entry point bf_dense_pair_noalloc against the context path.

Callers that cannot allocate device memory where they need these blocks (real-time loops that
cannot pay cudaMalloc's implicit device-wide synchronisation, processes whose memory manager
already owns the GPU's memory, plugins handed their buffers by the embedding application) use
bf_dense_pair_noalloc; it keeps its intermediates in a fixed device array built into the library.
Its pair blocks must equal the ones the regular solver assembles for the same pair.  This file
runs last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import synth
from oracle import lie

pytestmark = pytest.mark.gpu

TOL = 2e-5  # normal equations: the tolerance of the parity tests (of the largest entry)


def perturbed(poses, seed):
    rng = np.random.default_rng(seed)
    out = poses.copy()
    for k in range(len(out)):
        R, t = lie.apply_update(out[k][:3, :3], out[k][:3, 3], np.r_[rng.normal(0, 0.01, 3), rng.normal(0, 0.02, 3)])
        out[k] = lie.to44(R, t)
    return out


def unpack(o):
    A = np.zeros((12, 12))
    A[:6, :6] = o[0:36].reshape(6, 6)
    A[:6, 6:] = o[36:72].reshape(6, 6)
    A[6:, :6] = o[36:72].reshape(6, 6).T
    A[6:, 6:] = o[72:108].reshape(6, 6)
    return A, o[108:120]


def check_pair_against_context(prob, i, j, poses):
    """Blocks of the pair (i, j) from two calls of bf_dense_pair_noalloc in a row against the
    context path's normal equations for the same pair (a gauge frame without pairs plus i and j,
    w_sparse = 0 so that only the dense term enters A and b)."""
    import torch

    import paper_1604_01093_b300 as bf

    assert torch.cuda.is_available()
    intr = prob.intr
    g = 999
    weights = dict(w_sparse=0.0, w_dense=0.5, w_photo=0.1, w_geo=1.0)
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"])
    ctx.add_frames(0, prob.depth, prob.lum)
    ctx.add_frames(g, prob.depth[:1], prob.lum[:1])
    k = int(np.flatnonzero((prob.pairs[:, 0] == i) & (prob.pairs[:, 1] == j))[0])
    p, q = prob.pair_corr(k)
    ctx.add_correspondences(i, j, p, q)
    ref = ctx.build_system([g, i, j], np.stack([np.eye(4), poses[i], poses[j]]), **weights)
    A_ref, b_ref = ref["A"], ref["b"]
    assert ref["n_dense"] > 100

    dev = torch.device("cuda", 0)
    d_i = torch.from_numpy(prob.depth[i]).to(dev)
    l_i = torch.from_numpy(prob.lum[i]).to(dev)
    d_j = torch.from_numpy(prob.depth[j]).to(dev)
    l_j = torch.from_numpy(prob.lum[j]).to(dev)
    out = torch.full((124,), float("nan"), dtype=torch.float64, device=dev)
    for call in range(2):  # two calls in a row share the scratch array
        bf._lib.dense_pair_noalloc(d_i, l_i, d_j, l_j, poses[i], poses[j], out, intr["W"], intr["H"], intr["fx"],
                                   intr["fy"], intr["cx"], intr["cy"], **weights)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        A, b = unpack(o)
        np.testing.assert_allclose(A, A_ref, rtol=0, atol=TOL * np.abs(A_ref).max())
        np.testing.assert_allclose(b, b_ref, rtol=0, atol=TOL * np.abs(b_ref).max())
        assert abs(o[121] - ref["e_photo"]) <= TOL * ref["e_photo"]
        assert abs(o[122] - ref["e_geo"]) <= TOL * ref["e_geo"]
        assert int(round(o[123])) == ref["n_dense"]
        out.fill_(float("nan"))


def test_noalloc_pair_blocks_match_context_path():
    prob = synth.cfg1()
    check_pair_against_context(prob, 2, 6, perturbed(prob.gt, 31))


def test_noalloc_at_the_largest_frame_size():
    """160 x 120, the largest size the scratch array holds: its tile table is exactly full."""
    prob = synth.chunk_problem(95, 3, 160, 120, (80, 120), name="chunk3_160x120")
    check_pair_against_context(prob, 0, 1, perturbed(prob.gt, 32))


def test_noalloc_rejects_oversized_frames():
    import torch

    import paper_1604_01093_b300 as bf

    dev = torch.device("cuda", 0)
    big = torch.zeros((240, 320), dtype=torch.float32, device=dev)
    out = torch.zeros(124, dtype=torch.float64, device=dev)
    with pytest.raises(bf.BFError) as e:
        bf._lib.dense_pair_noalloc(big, big, big, big, np.eye(4), np.eye(4), out, 320, 240, 262.5, 262.5, 159.5,
                                   119.5)
    assert e.value.status == 1
