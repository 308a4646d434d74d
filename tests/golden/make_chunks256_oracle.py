"""Write chunks256_oracle.json: the FP64 oracle's local solves (6 GN x 10 PCG, Sec. 4.2 chunk solves
from the identity) of 18 chunks of the 256-chunk 320x240 batch workload, two of every length 3..11
(the first two chunks of that length), on the frames as given ("fp32") and on the BF16-rounded
planes the library stores with BF16 storage ("bf16").  Only the oracle and the seeded scene
generator run here; the GPU tests compare the library's full batch with these values.

    python tests/golden/make_chunks256_oracle.py [processes]
"""
import json
import multiprocessing as mp
import os
import sys

# pool workers run one BLAS thread each (they inherit this environment; set before numpy loads)
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import frames as ofr, solver  # noqa: E402
from oracle.system import SolveParams  # noqa: E402


def picks(prob):
    out = []
    for n in range(3, 12):
        out += [k for k, c in enumerate(prob.chunks) if len(c) == n][:2]
    return out


_PROB = None


def workload():
    """The batch workload, generated once per process."""
    global _PROB
    if _PROB is None:
        _PROB = synth.cfg3()
    return _PROB


def solve_one(args):
    k, storage = args
    prob = workload()
    d = prob.solve
    prm = SolveParams(n_gn=d["n_gn"], n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"],
                      w_photo=d["w_photo"], w_geo=d["w_geo"])
    ids = [int(f) for f in prob.chunks[k]]
    st = None if storage == "fp32" else storage
    frames = [ofr.Frame(prob.depth[f], prob.lum[f], prob.intr, storage=st) for f in ids]
    res = solver.gauss_newton(frames, prob.intr, prob.init[ids], solver.sparse_pairs_for(prob, ids), prm)
    return {"chunk": k, "storage": storage, "frames": ids, "energy": [float(e) for e in res.energy],
            "poses": [[float(v) for v in P[:3, :].ravel()] for P in res.poses]}


def main(processes=None):
    prob = workload()
    d = prob.solve
    jobs = [(k, s) for s in ("fp32", "bf16") for k in picks(prob)]
    # longest chunks first so that the pool's last wave is short
    jobs.sort(key=lambda j: -len(prob.chunks[j[0]]))
    with mp.get_context("spawn").Pool(processes) as pool:
        samples = pool.map(solve_one, jobs, chunksize=1)
    samples.sort(key=lambda s: (s["storage"], len(s["frames"]), s["chunk"]))
    out = {"workload": prob.name, "chunks": len(prob.chunks), "n_gn": d["n_gn"], "n_pcg": d["n_pcg"],
           "samples": samples}
    with open(os.path.join(HERE, "chunks256_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else None)
