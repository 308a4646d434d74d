"""Write global300_oracle.json: the FP64 oracle on the 300-keyframe 80x60 corridor workload from its
initial poses: its first Gauss-Newton step (20 block-Jacobi PCG iterations) and its whole solve as
the benchmark runs it (8 Gauss-Newton x 20 PCG): the Sec. 4.3 energy before every step and after
the last, and every keyframe's pose at the iterates X_1, X_3, X_7 and at the end.  Only the oracle and the
seeded scene generator run here; the GPU tests compare the library's full-size solve with these.

    python tests/golden/make_global300_oracle.py [processes]
"""
import json
import os
import sys

# pool workers run one BLAS thread each (they inherit this environment; set before numpy loads)
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import frames as ofr, solver, system  # noqa: E402
from oracle.system import SolveParams  # noqa: E402


KEEP = (1, 3, 7)  # X_1 pins the oracle itself; the GPU tests start single steps at X_0 = init, X_3, X_7


def poses34(P):
    return [[float(v) for v in T[:3, :].ravel()] for T in P]


def main(processes=None):
    prob = synth.cfg2()
    d = prob.solve
    frames = [ofr.Frame(prob.depth[k], prob.lum[k], prob.intr) for k in range(prob.n_frames)]
    prm = SolveParams(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"],
                      w_photo=d["w_photo"], w_geo=d["w_geo"])
    with system.frame_pool(frames, processes) as pool:
        res = solver.gauss_newton(frames, prob.intr, prob.init, solver.sparse_pairs_for(prob, range(prob.n_frames)),
                                  prm, pmap=lambda f, tasks: pool.map(f, tasks, chunksize=16))
    out = {"workload": prob.name, "n_frames": prob.n_frames, "pairs": int(len(prob.pairs)),
           "n_gn": d["n_gn"], "n_pcg": d["n_pcg"], "weights": {k: d[k] for k in ("w_sparse", "w_dense", "w_photo", "w_geo")},
           "energy": [float(e) for e in res.energy], "n_dense": [int(n) for n in res.n_dense],
           "iterates": {str(k): poses34(res.pose_history[k]) for k in KEEP}, "poses": poses34(res.poses)}
    with open(os.path.join(HERE, "global300_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else None)
