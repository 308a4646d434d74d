"""GPU parity of the Sec. 5 TSDF integration / de-integration against the oracle.

The voxel sums are integers and every decision before them is FP32 in the oracle's operation
order, so the exported volume (block set and every S, W, SC) must equal the oracle's exactly.
"""
import numpy as np
import pytest

import synth
from oracle import frames as ofr, lie, tsdf

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


def make_ctx(bf, prob, storage=0, poses=None):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], storage=storage)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=poses)
    return ctx


def oracle_frames(prob, storage=None):
    return [ofr.Frame(prob.depth[k], prob.lum[k], prob.intr, storage=storage) for k in range(prob.n_frames)]


def assert_same_volume(got, ref):
    ref = {k: v for k, v in ref.items()}
    assert set(got) == set(ref), (len(got), len(ref), len(set(got) ^ set(ref)))
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=str(k))


@pytest.mark.parametrize("voxel", [0.01, 0.004])
def test_integrate_matches_oracle(bf, cfg1, voxel):
    ctx = make_ctx(bf, cfg1)
    ctx.tsdf_init(voxel_size=voxel, trunc_voxels=5, table_log2=20, max_blocks=1 << 16)
    fr = oracle_frames(cfg1)
    prm = tsdf.Params(voxel, 5)
    ref = {}
    for k in ((0, 3, 7) if voxel > 0.005 else (0,)):
        ctx.tsdf_integrate(k, cfg1.gt[k])
        tsdf.integrate(ref, fr[k].D32, fr[k].C32, cfg1.intr, cfg1.gt[k], prm)
    got = ctx.tsdf_export()
    assert len(got) > 100
    assert_same_volume(got, ref)


def test_deintegration_is_the_exact_inverse(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    ctx.tsdf_init(voxel_size=0.01)
    fr = oracle_frames(cfg1)
    prm = tsdf.Params(0.01, 5)
    ref = {}
    for k in (1, 4, 9):
        ctx.tsdf_integrate(k, cfg1.gt[k])
        tsdf.integrate(ref, fr[k].D32, fr[k].C32, cfg1.intr, cfg1.gt[k], prm)
    ctx.tsdf_deintegrate(4)
    tsdf.integrate(ref, fr[4].D32, fr[4].C32, cfg1.intr, cfg1.gt[4], prm, sign=-1)
    assert_same_volume(ctx.tsdf_export(), ref)
    with pytest.raises(bf.BFError):
        ctx.tsdf_deintegrate(4)  # no longer integrated
    ctx.tsdf_deintegrate(1)
    ctx.tsdf_deintegrate(9)
    got = ctx.tsdf_export()
    assert len(got) > 0 and all(not v.any() for v in got.values())  # every sum back to 0


def test_bf16_storage_volume(bf, cfg1):
    """16-bit storage keeps depth exact; the intensity is the BF16-rounded one on both sides."""
    ctx = make_ctx(bf, cfg1, storage=bf.BF_STORE_BF16)
    ctx.tsdf_init(voxel_size=0.01)
    fr = oracle_frames(cfg1, "bf16")
    prm = tsdf.Params(0.01, 5)
    ref = {}
    for k in (2, 6):
        ctx.tsdf_integrate(k, cfg1.gt[k])
        tsdf.integrate(ref, fr[k].D32, fr[k].C32, cfg1.intr, cfg1.gt[k], prm)
    assert_same_volume(ctx.tsdf_export(), ref)


def test_reintegration_follows_the_largest_pose_changes(bf, cfg1):
    """Frames integrated at perturbed poses; their optimised (world) poses are the ground truth.
    The update re-integrates the n_fix frames whose poses moved most, in that order."""
    ctx = make_ctx(bf, cfg1, poses=cfg1.gt)
    ctx.tsdf_init(voxel_size=0.01)
    rng = np.random.default_rng(81)
    fr = oracle_frames(cfg1)
    prm = tsdf.Params(0.01, 5)
    integ = {}
    for k in range(6):
        T = cfg1.gt[k].copy()
        T[:3, :3] = lie.exp_so3(rng.normal(scale=0.02 * (k + 1), size=3)) @ T[:3, :3]
        T[:3, 3] += rng.normal(scale=0.01 * (k + 1), size=3)
        integ[k] = T
        ctx.tsdf_integrate(k, T)
    order = tsdf.reintegration_order(integ, {k: cfg1.gt[k] for k in integ}, n_fix=3)
    assert ctx.tsdf_reintegrate(3) == order
    ref = {}
    for k in range(6):
        T = cfg1.gt[k] if k in order else integ[k]
        tsdf.integrate(ref, fr[k].D32, fr[k].C32, cfg1.intr, T, prm)
    got = ctx.tsdf_export()
    # compare the non-empty voxels (de-integration leaves the old pose's blocks allocated)
    for k in set(got) | set(ref):
        a = got.get(k, np.zeros((3, 512), np.int64))
        b = ref.get(k, np.zeros((3, 512), np.int64))
        np.testing.assert_array_equal(a, b, err_msg=str(k))


def test_full_table_is_an_error_not_a_hang(bf, cfg1):
    ctx = make_ctx(bf, cfg1)
    ctx.tsdf_init(voxel_size=0.004, table_log2=8, max_blocks=64)
    with pytest.raises(bf.BFError) as e:
        ctx.tsdf_integrate(0, cfg1.gt[0])
    assert e.value.status == 2  # BF_ERR_OUT_OF_MEMORY
    ctx.tsdf_init(voxel_size=0.01)  # a fresh volume works
    ctx.tsdf_integrate(0, cfg1.gt[0])
    assert len(ctx.tsdf_export()) > 0
