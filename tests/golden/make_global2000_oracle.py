"""Write global2000_oracle.json: the FP64 oracle's first Gauss-Newton step (30 block-Jacobi PCG
iterations, the Sec. 4.3 energy before and after it) on the 2000-keyframe 160x120 corridor
workload from its initial poses, twice: on the BF16-rounded frame planes the library stores for it
("bf16", the parity reference) and on the frames as given ("fp32", the reference for the error
of BF16 storage).  The explicitly assembled system has 11994 unknowns (1.15 GB).  Kept: both
energies, the pose of every keyframe for "bf16" and of every 32nd keyframe for "fp32" (poses
written with 12 significant digits).  Only the oracle and the seeded scene generator run
here; the GPU tests compare the library's full-size solve with these values.

    python tests/golden/make_global2000_oracle.py [processes]
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

FP32_STRIDE = 32


def pose_rows(P):
    """The top 3x4 of each pose, 12 significant digits."""
    return [[float(f"{v:.12g}") for v in T[:3, :].ravel()] for T in P]


def main(processes=None):
    prob = synth.cfg5()
    d = prob.solve
    prm = SolveParams(n_gn=1, n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
                      w_geo=d["w_geo"])
    keep = {"bf16": list(range(prob.n_frames)), "fp32": list(range(0, prob.n_frames, FP32_STRIDE))}
    out = {"workload": prob.name, "n_frames": prob.n_frames, "pairs": int(len(prob.pairs)), "n_gn": 1,
           "n_pcg": d["n_pcg"], "weights": {k: d[k] for k in ("w_sparse", "w_dense", "w_photo", "w_geo")}}
    sp = solver.sparse_pairs_for(prob, range(prob.n_frames))
    for storage in ("bf16", "fp32"):
        frames = [ofr.Frame(prob.depth[k], prob.lum[k], prob.intr, storage=None if storage == "fp32" else storage)
                  for k in range(prob.n_frames)]
        with system.frame_pool(frames, processes) as pool:
            res = solver.gauss_newton(frames, prob.intr, prob.init, sp, prm,
                                      pmap=lambda f, tasks: pool.map(f, tasks, chunksize=64))
        out[storage] = {"energy": [float(e) for e in res.energy], "n_dense": [int(n) for n in res.n_dense],
                        "frames_kept": keep[storage], "poses": pose_rows(res.poses[keep[storage]])}
    with open(os.path.join(HERE, "global2000_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else None)
