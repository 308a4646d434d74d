"""Write global2000_oracle.json: the FP64 oracle's first Gauss-Newton step (30 block-Jacobi PCG
iterations, the Sec. 4.3 energy before and after it) on the 2000-keyframe 160x120 corridor
workload, from its initial poses, on the BF16-rounded frame planes the library stores for it.
The explicitly assembled system has 11994 unknowns (1.15 GB); the run takes most of an hour.
Kept: both energies and the poses of every 32nd keyframe.  Only the oracle and the seeded scene
generator run here; the GPU tests compare the library's full-size solve with these values.

    python tests/golden/make_global2000_oracle.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import frames as ofr, solver  # noqa: E402
from oracle.system import SolveParams  # noqa: E402

STRIDE = 32


def main():
    prob = synth.cfg5()
    d = prob.solve
    frames = [ofr.Frame(prob.depth[k], prob.lum[k], prob.intr, storage="bf16") for k in range(prob.n_frames)]
    prm = SolveParams(n_gn=1, n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
                      w_geo=d["w_geo"])
    res = solver.gauss_newton(frames, prob.intr, prob.init, solver.sparse_pairs_for(prob, range(prob.n_frames)), prm)
    keep = list(range(0, prob.n_frames, STRIDE))
    out = {"workload": prob.name, "n_frames": prob.n_frames, "pairs": int(len(prob.pairs)), "storage": "bf16",
           "n_gn": 1, "n_pcg": d["n_pcg"], "weights": {k: d[k] for k in ("w_sparse", "w_dense", "w_photo", "w_geo")},
           "energy": [float(e) for e in res.energy], "frames_kept": keep,
           "poses": [[float(v) for v in res.poses[k][:3, :].ravel()] for k in keep]}
    with open(os.path.join(HERE, "global2000_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
