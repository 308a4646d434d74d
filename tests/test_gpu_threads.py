"""Several contexts driven from several host threads.

Kernel attributes (the staged dense kernel's and the cluster PCG's shared-memory opt-ins, the
cluster size) and occupancy queries are per-device one-time setups kept behind a mutex.  This test
runs, in a fresh process so that those setups happen during the race, two contexts on device 0 from
two host threads at once: the 11-frame chunk (staged dense kernel, target frames in shared memory)
and the 48-keyframe global solve (16-CTA cluster PCG).  Each result must be bitwise the result of
the same solve run alone afterwards.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys, threading
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_1604_01093_b300 as bf
import synth

probs = [synth.cfg1(), synth.global_problem(77, n_kf=48, outer=(12.0, 2.8, 9.0), inner=(6.0, 3.0),
                                            n_corr=(40, 100), name="global48")]

def run(k, out, barrier=None):
    prob = probs[k]
    intr = prob.intr
    ctx = bf.Context(intr["W"], intr["H"], intr["fx"], intr["fy"], intr["cx"], intr["cy"], max_frames_hint=prob.n_frames)
    ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
    ctx.add_correspondences_batch(prob.pairs, prob.corr_off, prob.p_i, prob.p_j)
    ids = list(range(prob.n_frames))
    if barrier is not None:
        barrier.wait()
    res = []
    for rep in range(3):
        ctx.add_frames(0, prob.depth, prob.lum, init_pose=prob.init)
        if k == 0:
            st = ctx.solve_local(0, ids, tile_px=0, **dict(prob.solve))
        else:
            st = ctx.solve_global(ids, n_gn=3, n_pcg=15, pcg_variant=3)
        res.append((st["energy"], ctx.get_poses(ids)))
    out[k] = res
    ctx.close()

conc = {}
barrier = threading.Barrier(2)
th = [threading.Thread(target=run, args=(k, conc, barrier)) for k in range(2)]
for t in th:
    t.start()
for t in th:
    t.join()
serial = {}
for k in range(2):
    run(k, serial)
for k in range(2):
    assert len(conc[k]) == 3
    for (e1, P1), (e2, P2) in zip(conc[k], serial[k]):
        assert e1 == e2, (k, e1, e2)
        assert np.array_equal(P1, P2), k
print("threads ok")
'''


def test_two_contexts_on_two_threads_match_serial_runs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "threads ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
