"""GPU parity of the dense verification (Sec. 4.1.1) and chunk validation (Sec. 4.2) kernels.

The gate decisions are FP32 with the oracle's operation order, so kept-correspondence counts
agree exactly except where the normal gate sits within FP32 rounding of tau_n (the two sides
round their normals independently): at most max(2, 1e-3 n) differences.  Distance sums are
FP32 per pixel and thread, FP64 across warps: relative 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle import frames as ofr, lie, verification

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


@pytest.fixture(scope="module")
def cfg1():
    return synth.cfg1()


def make_ctx(bf, prob, storage=0):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], storage=storage)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    for k, (i, j) in enumerate(prob.pairs):
        p, q = prob.pair_corr(k)
        ctx.add_correspondences(int(i), int(j), p, q)
    return ctx


def close_counts(a, b):
    return abs(a - b) <= max(2, int(1e-3 * max(a, b)))


def perturbed_rel(T, seed, rot=0.02, trans=0.03):
    rng = np.random.default_rng(seed)
    out = T.copy()
    out[:3, :3] = lie.exp_so3(rng.normal(scale=rot, size=3)) @ T[:3, :3]
    out[:3, 3] += rng.normal(scale=trans, size=3)
    return out


@pytest.mark.parametrize("kind", ["fp32", "bf16"])
def test_verify_pairs_matches_oracle(bf, cfg1, kind):
    storage = {"fp32": bf.BF_STORE_FP32, "bf16": bf.BF_STORE_BF16}[kind]
    ctx = make_ctx(bf, cfg1, storage)
    fr = [ofr.Frame(cfg1.depth[k], cfg1.lum[k], cfg1.intr, storage=None if kind == "fp32" else kind)
          for k in range(cfg1.n_frames)]
    pairs, rels = [], []
    for (i, j), seed in (((0, 1), 1), ((2, 9), 2), ((3, 7), 3), ((10, 4), 4)):
        T = np.linalg.inv(cfg1.gt[j]) @ cfg1.gt[i]
        for rel in (T, perturbed_rel(T, seed), perturbed_rel(T, seed + 10, 0.1, 0.3)):
            pairs.append((i, j))
            rels.append(rel)
    got = ctx.verify_pairs(pairs, np.stack(rels))
    n_checked = 0
    for (i, j), rel, g in zip(pairs, rels, got):
        ref = verification.verify_pair(fr[i], fr[j], rel, cfg1.intr)
        assert close_counts(g["n_ij"], ref.n_ij) and close_counts(g["n_ji"], ref.n_ji), (i, j, g, ref)
        for ge, re_, gn, rn in ((g["err_ij"], ref.e_ij, g["n_ij"], ref.n_ij), (g["err_ji"], ref.e_ji, g["n_ji"], ref.n_ji)):
            if gn == rn:
                assert abs(ge - re_) <= 1e-5 * max(re_, 1e-9), (ge, re_)
        if g["n_ij"] == ref.n_ij and g["n_ji"] == ref.n_ji:
            assert g["valid"] == verification.pair_valid(ref, cfg1.intr)
            n_checked += 1
    assert n_checked >= len(pairs) - 2
    assert any(g["valid"] for g in got) and not all(g["valid"] for g in got)  # both outcomes exercised


def test_verify_identity_pair_is_exact(bf, cfg1):
    """A frame against itself under the identity: every valid pixel kept, distance exactly 0."""
    ctx = make_ctx(bf, cfg1)
    fr0 = ofr.Frame(cfg1.depth[0], cfg1.lum[0], cfg1.intr)
    g = ctx.verify_pairs([(0, 0)], np.eye(4)[None])[0]
    n = int((fr0.valid & fr0.nvalid).sum())
    assert g["n_ij"] == g["n_ji"] == n and g["err_ij"] == 0.0 and g["err_ji"] == 0.0 and g["valid"]


def test_chunk_validation_matches_oracle(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    fr = [ofr.Frame(cfg1.depth[k], cfg1.lum[k], cfg1.intr) for k in range(cfg1.n_frames)]
    ids = list(range(11))
    ctx.solve_local(0, ids, **dict(cfg1.solve))
    g = ctx.validate_chunk(0)
    local = ctx.get_poses(ids)
    local = np.einsum("ab,kbc->kac", np.linalg.inv(local[0]), local)
    ok, worst, arg, _ = verification.validate_chunk(fr, local, cfg1.intr)
    assert g["valid"] == ok and ok
    assert abs(g["worst_err"] - worst) <= 1e-4 * worst  # the poses went through the 4x4 round trip
    # an unsolved chunk (no Gauss-Newton step: every frame at the identity) fails validation
    ctx.solve_local(1, ids, n_gn=0)
    bad = ctx.validate_chunk(1)
    ref_bad = verification.validate_chunk(fr, np.tile(np.eye(4), (11, 1, 1)), cfg1.intr)
    assert not bad["valid"] and not ref_bad[0]
    assert abs(bad["worst_err"] - ref_bad[1]) <= 1e-5 * ref_bad[1] and bad["worst_pair"] == ref_bad[2]


def test_validate_unknown_chunk(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    with pytest.raises(bf.BFError):
        ctx.validate_chunk(12345)
