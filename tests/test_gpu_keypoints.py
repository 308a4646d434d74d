"""GPU parity of the Sec. 4.1.1 key-point correspondence filter and surface-area filter.

Both sides decide in FP64 (the oracle with LAPACK's SVD, the kernel with Jacobi eigen-
decompositions), so the kept sets and statuses agree exactly and the fitted transforms to
~1e-9.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import keypoints

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


@pytest.fixture(scope="module")
def ctx(bf):
    return bf.Context(80, 60, 65.625, 65.625, 39.5, 29.5)


def make_pairs(seed, n_pairs=40):
    """Matched points with 3 mm noise, 0-40 % gross outliers anywhere in the match order, plus
    degenerate pairs: nearly collinear points, a small patch (area filter), too few matches."""
    rng = np.random.default_rng(seed)
    P_all, Q_all, off = [], [], [0]
    for k in range(n_pairs):
        kind = k % 8
        n = int(rng.integers(5, 300)) if kind < 5 else int(rng.integers(0, 40))
        if kind == 5:  # nearly collinear
            s = rng.uniform(-1, 1, n)
            P = np.stack([s, 0.5 * s, 2.0 + 0.3 * s], 1) + rng.normal(0, 1e-4, (n, 3))
        elif kind == 6:  # a 10 x 10 cm patch
            P = np.concatenate([rng.uniform(-0.05, 0.05, (n, 2)), rng.normal(2.0, 0.01, (n, 1))], 1)
        else:
            P = rng.uniform([-1.5, -1.0, 0.8], [1.5, 1.0, 4.0], (n, 3))
        n = len(P)
        R = Rotation.from_rotvec(rng.normal(0, 0.3, 3)).as_matrix()
        t = rng.normal(0, 0.5, 3)
        Q = P @ R.T + t + rng.normal(0, 0.003, (n, 3))
        if kind < 5 and n:
            bad = rng.random(n) < 0.4 * rng.random()
            Q[bad] += rng.normal(0, 0.4, (int(bad.sum()), 3))
        if kind == 7:
            P, Q = P[:int(rng.integers(0, 5))], Q[:0 + int(rng.integers(0, 5))]
            m = min(len(P), len(Q))
            P, Q = P[:m], Q[:m]
        P_all.append(P.astype(np.float32))
        Q_all.append(Q.astype(np.float32))
        off.append(off[-1] + len(P))
    return np.array(off), np.concatenate(P_all), np.concatenate(Q_all)


@pytest.mark.parametrize("seed", [71, 72])
def test_keypoint_filter_matches_oracle(ctx, seed):
    off, P, Q = make_pairs(seed)
    keep, T, status = ctx.filter_keypoints(off, P, Q)
    seen = set()
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        # the oracle sees exactly the FP32 inputs the device got, widened
        ref = keypoints.filter_pair(P[a:b].astype(np.float64), Q[a:b].astype(np.float64))
        assert status[k] == ref.status, (k, status[k], ref.status)
        seen.add(ref.status)
        got = np.flatnonzero(keep[a:b]).tolist()
        assert got == sorted(ref.keep), (k, got, ref.keep)
        if ref.status == 0:
            np.testing.assert_allclose(T[k][:3, :3], ref.R, atol=1e-9)
            np.testing.assert_allclose(T[k][:3, 3], ref.t, atol=1e-9)
            assert len(got) < b - a or len(got) == b - a
        else:
            assert not keep[a:b].any() and not T[k].any()
    assert seen == {0, 1, 2}  # every outcome exercised


def test_too_many_matches_rejected(ctx, bf):
    rng = np.random.default_rng(73)
    P = rng.uniform(-1, 1, (1025, 3)).astype(np.float32)
    with pytest.raises(bf.BFError):
        ctx.filter_keypoints([0, 1025], P, P)
    keep, T, status = ctx.filter_keypoints([0, 1024], P[:1024], P[:1024])
    assert status[0] == 0 and keep.all()
