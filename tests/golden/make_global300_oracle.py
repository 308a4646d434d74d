"""Write global300_oracle.json: the FP64 oracle's first Gauss-Newton step (20 block-Jacobi PCG
iterations, the Sec. 4.3 energy before and after it) on the 300-keyframe 80x60 corridor workload,
from its initial poses.  Only the oracle and the seeded scene generator run here; the GPU tests
compare the library's full-size solve with these values.

    python tests/golden/make_global300_oracle.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import frames as ofr, solver  # noqa: E402
from oracle.system import SolveParams  # noqa: E402


def main():
    prob = synth.cfg2()
    d = prob.solve
    frames = [ofr.Frame(prob.depth[k], prob.lum[k], prob.intr) for k in range(prob.n_frames)]
    prm = SolveParams(n_gn=1, n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
                      w_geo=d["w_geo"])
    res = solver.gauss_newton(frames, prob.intr, prob.init, solver.sparse_pairs_for(prob, range(prob.n_frames)), prm)
    out = {"workload": prob.name, "n_frames": prob.n_frames, "pairs": int(len(prob.pairs)), "n_gn": 1,
           "n_pcg": d["n_pcg"], "weights": {k: d[k] for k in ("w_sparse", "w_dense", "w_photo", "w_geo")},
           "energy": [float(e) for e in res.energy],
           "poses": [[float(v) for v in P[:3, :].ravel()] for P in res.poses]}
    with open(os.path.join(HERE, "global300_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
