"""Full-size parity: the 300-keyframe global solve in the launch configuration bench.py times
(mixed precision, target frames staged in shared memory, cluster PCG, the Gauss-Newton loop
replayed as a CUDA graph) against the FP64 oracle's first Gauss-Newton step on the same workload.

The oracle's step takes about a minute at this size, so its result is stored in
tests/golden/global300_oracle.json, written by tests/golden/make_global300_oracle.py from the
oracle and the seeded scene generator alone.  Tolerances are the spec ones.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import lie

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROT_TOL, TRANS_TOL, ENERGY_RTOL = 1e-4, 1e-5, 1e-5


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1604_01093_b300 as bf
    return bf


@pytest.fixture(scope="module")
def global300():
    return synth.cfg2()


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "global300_oracle.json")) as f:
        return json.load(f)


def make_ctx(bf, prob):
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                     max_frames_hint=prob.n_frames)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, prob.p_i, prob.p_j)
    return ctx


def params(prob, n_gn):
    d = prob.solve
    return dict(n_gn=n_gn, n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
                w_geo=d["w_geo"], use_graph=1)


def test_golden_matches_the_workload(global300, golden):
    assert golden["workload"] == global300.name and golden["n_frames"] == global300.n_frames
    assert golden["pairs"] == len(global300.pairs) and golden["n_pcg"] == global300.solve["n_pcg"]


def test_global300_first_step_matches_oracle(bf, global300, golden):
    ctx = make_ctx(bf, global300)
    ids = list(range(global300.n_frames))
    for _ in range(2):  # capture, then replay the graph
        ctx.add_frames(0, global300.depth, global300.lum, init_pose=global300.init)
        st = ctx.solve_global(ids, **params(global300, 1))
        assert st["flags"] == 0
        rel = np.abs(np.array(st["energy"]) - np.array(golden["energy"])) / np.array(golden["energy"])
        assert rel.max() <= ENERGY_RTOL, rel
        P = ctx.get_poses(ids)
        worst_rot = worst_tr = 0.0
        for k in range(len(ids)):
            ref = np.eye(4)
            ref[:3, :] = np.array(golden["poses"][k]).reshape(3, 4)
            rot, tr = lie.pose_error(P[k], ref)
            worst_rot, worst_tr = max(worst_rot, rot), max(worst_tr, tr)
        assert worst_rot <= ROT_TOL and worst_tr <= TRANS_TOL, (worst_rot, worst_tr)


def test_global300_bench_solve_starts_at_the_oracle_energy(bf, global300, golden):
    """The bench's own solve (8 GN x 20 PCG): its first energy is the oracle's at the initial poses and
    the energy falls from there."""
    ctx = make_ctx(bf, global300)
    st = ctx.solve_global(list(range(global300.n_frames)), **params(global300, global300.solve["n_gn"]))
    assert st["flags"] == 0 and st["n_gn"] == global300.solve["n_gn"]
    assert abs(st["energy"][0] - golden["energy"][0]) <= ENERGY_RTOL * golden["energy"][0]
    assert abs(st["energy"][1] - golden["energy"][1]) <= ENERGY_RTOL * golden["energy"][1]
    assert st["energy"][-1] < 0.8 * st["energy"][0]
