"""GPU parity of the dense verification (Sec. 4.1.1) and chunk validation (Sec. 4.2) kernels.

The library decides the gates in FP32, the oracle in FP64; they agree except on ties (a value
within FP32 rounding of its threshold, which either side may decide either way).  So the
library's kept count must lie between the oracle's count of kept non-tie pixels and that plus
the ties, and its distance sum between the non-tie sum and that plus tau_d per tie (a kept pixel is
closer than tau_d), up to the FP32 summation's rounding (relative 1e-5).  With no tie the two must
agree exactly in count.
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


def mean_bounds(chk):
    """Range of a pair's two-sided mean error over every way of deciding its ties."""
    n_lo = chk.bounds("ij")[0] + chk.bounds("ji")[0]
    n_hi = chk.bounds("ij")[1] + chk.bounds("ji")[1]
    e_lo = chk.bounds("ij")[2] + chk.bounds("ji")[2]
    e_hi = chk.bounds("ij")[3] + chk.bounds("ji")[3]
    return e_lo / max(n_hi, 1), e_hi / max(n_lo, 1)


def within_bounds(ref, direction, n, e, rtol=1e-5):
    n_lo, n_hi, e_lo, e_hi = ref.bounds(direction)
    return n_lo <= n <= n_hi and e_lo * (1 - rtol) - 1e-9 <= e <= e_hi * (1 + rtol) + 1e-9


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
    n_decided = 0
    for (i, j), rel, g in zip(pairs, rels, got):
        ref = verification.verify_pair(fr[i], fr[j], rel, cfg1.intr)
        assert within_bounds(ref, "ij", g["n_ij"], g["err_ij"]), (i, j, g, ref)
        assert within_bounds(ref, "ji", g["n_ji"], g["err_ji"]), (i, j, g, ref)
        # validity where no way of deciding the ties could change it
        lo, hi = mean_bounds(ref)
        n_lo = ref.bounds("ij")[0] + ref.bounds("ji")[0]
        n_hi = ref.bounds("ij")[1] + ref.bounds("ji")[1]
        min_n = 0.02 * cfg1.intr["W"] * cfg1.intr["H"]
        if (hi <= 0.075 and n_lo >= min_n) or lo > 0.075 or n_hi < min_n:
            assert g["valid"] == verification.pair_valid(ref, cfg1.intr), (i, j, g, ref)
            n_decided += 1
    assert n_decided >= len(pairs) - 2
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
    ok, worst, arg, checks = verification.validate_chunk(fr, local, cfg1.intr)
    assert g["valid"] == ok and ok
    # the worst pair's mean error within what the ties allow (the poses went through the 4x4 round trip)
    bounds = [mean_bounds(c) for c in checks.values() if c.n_ij + c.n_ji > 0]
    lo, hi = max(b[0] for b in bounds), max(b[1] for b in bounds)
    assert lo * (1 - 1e-4) <= g["worst_err"] <= hi * (1 + 1e-4), (g["worst_err"], lo, hi, worst)
    # an unsolved chunk (no Gauss-Newton step: every frame at the identity) fails validation
    ctx.solve_local(1, ids, n_gn=0)
    bad = ctx.validate_chunk(1)
    ref_bad = verification.validate_chunk(fr, np.tile(np.eye(4), (11, 1, 1)), cfg1.intr)
    assert not bad["valid"] and not ref_bad[0]
    bounds = [mean_bounds(c) for c in ref_bad[3].values() if c.n_ij + c.n_ji > 0]
    lo, hi = max(b[0] for b in bounds), max(b[1] for b in bounds)
    assert lo * (1 - 1e-5) <= bad["worst_err"] <= hi * (1 + 1e-5)
    assert bad["worst_pair"] == ref_bad[2] or mean_bounds(ref_bad[3][tuple(bad["worst_pair"])])[1] >= lo


def test_validate_unknown_chunk(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    with pytest.raises(bf.BFError):
        ctx.validate_chunk(12345)
