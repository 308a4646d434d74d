"""Explicit Gauss-Newton normal equations (oracle, FP64).

Sec. 4.4 linearises the stacked residual vector F at X^{k-1} and solves
J_F^T J_F dX = -J_F^T F.  Here every residual carries its energy weight w, so the
system is A = sum w J^T J, b = -sum w J^T r, assembled as one dense
(6 n_free) x (6 n_free) matrix.  The first frame of the solve is the gauge
(Sec. 4.3: T_0 is not a free variable), so frame a >= 1 owns unknowns 6(a-1)..6a-1.

Readings:
* E = w_sparse sum_corr w_c ||r_s||^2 + w_dense (w_photo sum r_p^2 + w_geo sum r_g^2), plain
  L2 with no normalisation by residual counts;
* each unordered pair's correspondences are counted once;
* the dense set E holds unordered pairs; both directions i->j and j->i are evaluated
  (Sec. 4.4 counts one photometric and one geometric residual per pixel per element);
* E = the sparse pairs whose camera viewing directions differ by less than max_angle_deg
  (Sec. 4.3: within 60 degrees), tested once at the solve's initial poses, in FP64, as
  z_i . z_j > cos(max_angle) on the third columns of R;
* w_dense ramps linearly, w_dense(k) = w_dense (k+1)/n_gn, when dense_ramp is set
  (Sec. 4.3 says it is linearly increased; the schedule is a reading).
"""
import dataclasses
import math

import numpy as np

from . import association, residuals


@dataclasses.dataclass
class SolveParams:
    n_gn: int = 4
    n_pcg: int = 10
    w_sparse: float = 1.0
    w_dense: float = 0.5
    w_photo: float = 0.1
    w_geo: float = 1.0
    dense_ramp: bool = False
    tau_dist: float = 0.15
    tau_normal: float = 0.9
    max_angle_deg: float = 60.0
    precond: str = "block"      # "block" (6x6 block-Jacobi) or "jacobi" (diagonal)
    dense_on: bool = True

    def w_dense_at(self, k):
        if self.dense_ramp:
            return self.w_dense * (k + 1) / self.n_gn
        return self.w_dense


@dataclasses.dataclass
class SparsePair:
    """Correspondences of an unordered pair a < b (local frame indices of the solve)."""
    a: int
    b: int
    p: np.ndarray        # (N,3) camera coordinates of frame a
    q: np.ndarray        # (N,3) camera coordinates of frame b
    w: np.ndarray | None = None


def dense_pair_set(poses, sparse_pairs, max_angle_deg):
    """Pairs of E: sparse pairs whose optical axes are within max_angle_deg (Sec. 4.3)."""
    c = math.cos(math.radians(max_angle_deg))
    out = []
    for sp in sparse_pairs:
        za = poses[sp.a][:3, 2]
        zb = poses[sp.b][:3, 2]
        dot = (za[0] * zb[0] + za[1] * zb[1]) + za[2] * zb[2]
        if dot > c:
            out.append((sp.a, sp.b))
    return out


def row_products(Ja, Jb, r, w):
    """For rows r (N,) with Jacobians Ja, Jb (N,6) w.r.t. two frames and weights w (N,): the blocks
    sum w J_x^T J_y (x, y in {a, b}) and the right-hand sides -sum w J_x^T r."""
    Ja = np.asarray(Ja, dtype=np.float64)
    Jb = np.asarray(Jb, dtype=np.float64)
    wr = w * r
    Wa, Wb = Ja * w[:, None], Jb * w[:, None]
    return dict(aa=Wa.T @ Ja, ab=Wa.T @ Jb, ba=Wb.T @ Ja, bb=Wb.T @ Jb, ga=-(Ja.T @ wr), gb=-(Jb.T @ wr))


class System:
    def __init__(self, n_frames):
        self.n = n_frames
        m = 6 * (n_frames - 1)
        self.A = np.zeros((m, m))
        self.b = np.zeros(m)
        self.e_sparse = 0.0
        self.e_geo = 0.0
        self.e_photo = 0.0
        self.n_sparse = 0
        self.n_dense = 0

    def add_products(self, a, b, P):
        """Add row_products of frames a, b into the system; the gauge frame 0 has no unknowns."""
        for fx, kx in ((a, "a"), (b, "b")):
            if fx == 0:
                continue
            ix = 6 * (fx - 1)
            self.b[ix:ix + 6] += P["g" + kx]
            for fy, ky in ((a, "a"), (b, "b")):
                if fy == 0:
                    continue
                iy = 6 * (fy - 1)
                self.A[ix:ix + 6, iy:iy + 6] += P[kx + ky]

    def add(self, a, Ja, b, Jb, r, w):
        """Accumulate rows r (N,) with Jacobians Ja, Jb (N,6) for frames a, b and weights w (N,)."""
        self.add_products(a, b, row_products(Ja, Jb, r, w))


# Frames of the solve in a worker process of a parallel assembly (set by init_worker).
_WORKER_FRAMES = None


def init_worker(frames):
    """Initializer of a worker pool for assemble(pmap=...): the solve's frames, sent once."""
    global _WORKER_FRAMES
    _WORKER_FRAMES = frames


def dense_pair(frames, task):
    """Dense photometric and geometric contribution of one directed pair i -> j (Sec. 4.3).

    task = (i, j, poses (4x4 of i and j), intr, tau_d, tau_n, w_geo, w_photo, asc): weights already
    multiplied by w_dense (0 = energies only); asc None = this oracle's own association, a dict = a
    given association, ("replay", target, W, H, eps, check_poses) = another implementation's
    decisions to check against this oracle's (at check_poses = (T_i, T_j), or at the task's poses
    if None) and replay at the task's poses (association.check_replay; the result's "check" holds
    the valid count, the flips and the first disagreement).
    Returns the residual count, both energies and the row products of the two residual kinds."""
    i, j, Ti, Tj, intr, tau_d, tau_n, w_geo, w_photo, asc = task
    Ri, ti, Rj, tj = Ti[:3, :3], Ti[:3, 3], Tj[:3, :3], Tj[:3, 3]
    check = None
    if asc is None or (isinstance(asc, tuple) and asc[0] == "replay"):
        own = association.associate(frames[i], frames[j], association.relative_transform(Ri, ti, Rj, tj), intr,
                                    tau_d, tau_n)
        if asc is None:
            asc = own
        else:  # another implementation's decisions, checked here (association.check_replay)
            _, target, W, H, eps, cp = asc
            own_c = own
            if cp is not None:  # checked at the poses they were taken at
                Ci, Cj = cp
                own_c = association.associate(frames[i], frames[j], association.relative_transform(
                    Ci[:3, :3], Ci[:3, 3], Cj[:3, :3], Cj[:3, 3]), intr, tau_d, tau_n)
            asc, nv, nf, err = association.check_replay(own_c, target, W, H, eps, own_replay=own)
            check = (nv, nf, err)
    d = residuals.dense_terms(frames[i], frames[j], Ri, ti, Rj, tj, asc)
    k = len(d["idx"])
    out = dict(k=k, e_geo=float(np.sum(d["r_geo"] ** 2)), e_photo=float(np.sum(d["r_photo"] ** 2)), check=check)
    if w_geo != 0.0 or w_photo != 0.0:
        out["geo"] = row_products(d["J_geo_i"], d["J_geo_j"], d["r_geo"], np.full(k, w_geo))
        out["photo"] = row_products(d["J_photo_i"], d["J_photo_j"], d["r_photo"], np.full(k, w_photo))
    return out


def _dense_pair_worker(task):
    return dense_pair(_WORKER_FRAMES, task)


def frame_pool(frames, processes=None):
    """A process pool (spawn start method) whose workers hold the solve's frames (a list, or e.g. a
    frames.FrameCache over a whole problem, with assemble's frame_keys); pass
    ``lambda f, tasks: pool.map(f, tasks, chunksize=8)`` as assemble's pmap."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(processes, initializer=init_worker, initargs=(frames,))


def assemble(frames, intr, poses, sparse_pairs, dense_pairs, params: SolveParams, w_dense, assoc=None, pmap=None,
             frame_keys=None):
    """Normal equations and energy at the given poses.

    frames: preprocessed frames (frames.Frame) of the solve, index 0 = gauge frame.
    poses: (n,4,4) camera->world.  Returns a System.
    assoc: optional association.CheckedReplay: another implementation's decisions, checked
    against this oracle's own (ties may differ) and replayed in place of them; None keeps the
    oracle's decisions.
    pmap: optional order-preserving map (e.g. a process pool's, initialised with init_worker(frames))
    over the directed pairs; each pair is evaluated alone and the sums are taken in pair order.
    frame_keys: with pmap, the key under which the workers' frames hold local frame k (default k).
    """
    S = System(len(frames))
    R = [P[:3, :3] for P in poses]
    t = [P[:3, 3] for P in poses]
    for sp in sparse_pairs:
        a, b = sp.a, sp.b
        N = sp.p.shape[0]
        w = np.ones(N) if sp.w is None else np.asarray(sp.w, dtype=np.float64)
        r = residuals.sparse_residuals(R[a], t[a], R[b], t[b], sp.p, sp.q)
        Ja, Jb = residuals.sparse_jacobians(R[a], t[a], R[b], t[b], sp.p, sp.q)
        S.e_sparse += float(np.sum(w * np.sum(r * r, axis=1)))
        S.n_sparse += 3 * N
        for row in range(3):
            S.add(a, Ja[:, row, :], b, Jb[:, row, :], r[:, row], params.w_sparse * w)
    if params.dense_on:
        # zero dense weight: energies still reported, no contribution to the system
        wg, wp = w_dense * params.w_geo, w_dense * params.w_photo
        tasks, order = [], []
        for (a, b) in dense_pairs:
            for (i, j) in ((a, b), (b, a)):
                asc = None
                if assoc is not None:
                    # checked replay (dense_pair compares the fetched decisions with its own)
                    asc = ("replay", np.asarray(assoc.fetch(i, j, poses)), assoc.W, assoc.H, assoc.eps,
                           assoc.check_poses(i, j))
                tasks.append((i, j, poses[i], poses[j], intr, params.tau_dist, params.tau_normal, wg, wp, asc))
                order.append((i, j))
        if pmap is not None:
            if frame_keys is not None:
                tasks = [(frame_keys[tk[0]], frame_keys[tk[1]]) + tk[2:] for tk in tasks]
            results = pmap(_dense_pair_worker, tasks)
        else:
            results = (dense_pair(frames, tk) for tk in tasks)
        for (i, j), res in zip(order, results):
            if res["check"] is not None:
                assoc.record(*res["check"], i, j)
            S.n_dense += res["k"]
            S.e_geo += res["e_geo"]
            S.e_photo += res["e_photo"]
            if "geo" in res:
                S.add_products(i, j, res["geo"])
                S.add_products(i, j, res["photo"])
    S.energy = params.w_sparse * S.e_sparse + w_dense * (params.w_photo * S.e_photo + params.w_geo * S.e_geo)
    return S
