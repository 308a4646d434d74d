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

    def add(self, a, Ja, b, Jb, r, w):
        """Accumulate rows r (N,) with Jacobians Ja, Jb (N,6) for frames a, b and weights w (N,)."""
        Ja = np.asarray(Ja, dtype=np.float64)
        Jb = np.asarray(Jb, dtype=np.float64)
        wr = w * r
        blocks = [(a, Ja), (b, Jb)]
        for fa, Jx in blocks:
            if fa == 0:
                continue
            ia = 6 * (fa - 1)
            self.b[ia:ia + 6] -= Jx.T @ wr
            for fb, Jy in blocks:
                if fb == 0:
                    continue
                ib = 6 * (fb - 1)
                self.A[ia:ia + 6, ib:ib + 6] += (Jx * w[:, None]).T @ Jy


def assemble(frames, intr, poses, sparse_pairs, dense_pairs, params: SolveParams, w_dense):
    """Normal equations and energy at the given poses.

    frames: preprocessed frames (frames.Frame) of the solve, index 0 = gauge frame.
    poses: (n,4,4) camera->world.  Returns a System.
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
    if params.dense_on and w_dense != 0.0:
        for (a, b) in dense_pairs:
            for (i, j) in ((a, b), (b, a)):
                M32 = association.pair_transform32(R[i], t[i], R[j], t[j])
                asc = association.associate(frames[i], frames[j], M32, intr, params.tau_dist, params.tau_normal)
                d = residuals.dense_terms(frames[i], frames[j], R[i], t[i], R[j], t[j], asc)
                k = len(d["idx"])
                S.n_dense += k
                S.e_geo += float(np.sum(d["r_geo"] ** 2))
                S.e_photo += float(np.sum(d["r_photo"] ** 2))
                S.add(i, d["J_geo_i"], j, d["J_geo_j"], d["r_geo"], np.full(k, w_dense * params.w_geo))
                S.add(i, d["J_photo_i"], j, d["J_photo_j"], d["r_photo"], np.full(k, w_dense * params.w_photo))
    elif params.dense_on:
        # zero dense weight: energies still reported, no contribution to the system
        for (a, b) in dense_pairs:
            for (i, j) in ((a, b), (b, a)):
                M32 = association.pair_transform32(R[i], t[i], R[j], t[j])
                asc = association.associate(frames[i], frames[j], M32, intr, params.tau_dist, params.tau_normal)
                d = residuals.dense_terms(frames[i], frames[j], R[i], t[i], R[j], t[j], asc)
                S.n_dense += len(d["idx"])
                S.e_geo += float(np.sum(d["r_geo"] ** 2))
                S.e_photo += float(np.sum(d["r_photo"] ** 2))
    S.energy = params.w_sparse * S.e_sparse + w_dense * (params.w_photo * S.e_photo + params.w_geo * S.e_geo)
    return S
