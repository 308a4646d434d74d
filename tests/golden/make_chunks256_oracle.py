"""Write chunks256_oracle.json: the FP64 oracle's local solves (6 GN x 10 PCG, Sec. 4.2 chunk
solves, identity start) of two chunks of the 256-chunk 320x240 batch workload: the first 3-frame
chunk and the first 11-frame chunk.  Only the oracle and the seeded scene generator run here; the
GPU tests compare the library's full batch with these values.

    python tests/golden/make_chunks256_oracle.py
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
    prob = synth.cfg3()
    d = prob.solve
    prm = SolveParams(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"],
                      w_photo=d["w_photo"], w_geo=d["w_geo"])
    lens = [len(c) for c in prob.chunks]
    picks = [lens.index(3), lens.index(11)]
    out = {"workload": prob.name, "chunks": len(prob.chunks), "n_gn": d["n_gn"], "n_pcg": d["n_pcg"], "samples": []}
    for k in picks:
        ids = [int(f) for f in prob.chunks[k]]
        frames = [ofr.Frame(prob.depth[f], prob.lum[f], prob.intr) for f in ids]
        res = solver.gauss_newton(frames, prob.intr, prob.init[ids], solver.sparse_pairs_for(prob, ids), prm)
        out["samples"].append({"chunk": k, "frames": ids, "energy": [float(e) for e in res.energy],
                               "poses": [[float(v) for v in P[:3, :].ravel()] for P in res.poses]})
    with open(os.path.join(HERE, "chunks256_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
