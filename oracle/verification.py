"""Dense verification of a frame pair and chunk validation (oracle, FP64, Sec. 4.1.1 and Sec. 4.2).

TEST INFRASTRUCTURE ONLY: the CUDA library never imports this package.

Sec. 4.1.1 aligns frames f_i and f_j with a relative transform T_ij (camera i -> camera j),
re-projects every pixel of one frame into the other in both directions, and keeps a pixel
correspondence when its depth discrepancy, normal deviation and photoconsistency pass three
gates; the pair is rejected if the re-projection error of the kept correspondences is too
large or too few of them exist.  Sec. 4.2 applies the same test to every frame pair of a chunk
at its optimised local poses and discards the chunk if any pair's error is too large.

Readings (the paper states the gates and thresholds but not every detail):

* the correspondence of source pixel (x, y) is the nearest target pixel of u = pi(T_ij p),
  (floor(u_x + 1/2), floor(u_y + 1/2)) (the projective association of the dense energy, Sec. 4.3,
  without its bilinear border), inside the image, with valid depth and normal on both sides;
* gates: ||T_ij p - q|| < tau_d, (R_ij n_i) . n_j > tau_n, |C_i(x, y) - C_j(target)| < tau_c,
  where C is the frame's intensity (the luminance given with the depth);
* the re-projection error of the pair is the mean distance over the kept correspondences of
  both directions, sum(E_ij + E_ji) / (n_ij + n_ji); the pair is valid iff that mean is at most
  e_max (0.075 m) and n_ij + n_ji >= frac_min * w * h (frac_min = 0.02);
* chunk validation: every pair of the chunk's frames at the optimised local poses; the chunk is
  invalid if some pair with kept correspondences has a mean error above 0.05 m.

Everything is FP64.  As in association.py, a pixel whose decision sits within an FP32 evaluation's
rounding of a threshold is a tie; ``reproject`` counts the ties so that a comparison with an FP32
implementation can bound its count and distance sum (``PairCheck.bounds``).
"""
import dataclasses

import numpy as np

from .association import EPS_D, EPS_N, EPS_PX

# FP32 rounding of |C_i - C_j| for intensities in [0, 1]
EPS_C = 1e-6


def reproject(fi, fj, T, intr, tau_d=0.15, tau_n=0.9, tau_c=0.1):
    """One direction i -> j under T (4x4, camera i -> camera j).  Returns (n kept, sum of the kept
    correspondences' distances ||T p - q||, n ties, kept mask); ties are counted over the pixels
    whose outcome (kept or not, or which target) an FP32 evaluation may decide otherwise."""
    T = np.asarray(T, dtype=np.float64)
    R, t = T[:3, :3], T[:3, 3]
    W, H = intr["W"], intr["H"]
    fx, fy, cx, cy = (float(intr[k]) for k in ("fx", "fy", "cx", "cy"))
    ys, xs = np.divmod(np.arange(W * H), W)
    z = fi.D.ravel()
    d = np.stack([(xs - cx) * z / fx, (ys - cy) * z / fy, z], axis=1)
    y = d @ R.T + t
    ok = fi.valid.ravel() & fi.nvalid.ravel() & (y[:, 2] > 0)
    yz = np.where(ok, y[:, 2], 1.0)
    ux = np.where(ok, fx * y[:, 0] / yz + cx, -100.0)
    uy = np.where(ok, fy * y[:, 1] / yz + cy, -100.0)
    tie = ok & (np.minimum(np.abs(ux + 0.5 - np.round(ux + 0.5)), np.abs(uy + 0.5 - np.round(uy + 0.5))) < EPS_PX)
    nxf = np.floor(ux + 0.5)
    nyf = np.floor(uy + 0.5)
    ok &= (nxf >= 0) & (nxf <= W - 1) & (nyf >= 0) & (nyf <= H - 1)
    nx = np.where(ok, nxf, 0).astype(np.int64)
    ny = np.where(ok, nyf, 0).astype(np.int64)
    tgt = ny * W + nx
    ok &= fj.valid.ravel()[tgt] & fj.nvalid.ravel()[tgt]
    Dj = fj.D.ravel()[tgt]
    q = np.stack([(nx - cx) * Dj / fx, (ny - cy) * Dj / fy, Dj], axis=1)
    dist = np.sqrt(np.sum((y - q) ** 2, axis=1))
    ndot = np.sum((fi.N.reshape(-1, 3) @ R.T) * fj.N.reshape(-1, 3)[tgt], axis=1)
    dc = np.abs(fi.C.ravel() - fj.C.ravel()[tgt])
    tie |= ok & ((np.abs(dist - tau_d) < EPS_D) | (np.abs(ndot - tau_n) < EPS_N) | (np.abs(dc - tau_c) < EPS_C))
    ok &= (dist < tau_d) & (ndot > tau_n) & (dc < tau_c)
    return int(ok.sum()), float(dist[ok].sum()), int(tie.sum()), ok, tie, dist


@dataclasses.dataclass
class PairCheck:
    n_ij: int
    n_ji: int
    e_ij: float
    e_ji: float
    tie_ij: int = 0
    tie_ji: int = 0
    sure_ij: tuple = (0, 0.0)   # (count, distance sum) of the kept pixels that are not ties
    sure_ji: tuple = (0, 0.0)

    @property
    def mean(self):
        n = self.n_ij + self.n_ji
        return (self.e_ij + self.e_ji) / n if n else float("inf")

    def bounds(self, direction, tau_d=0.15):
        """(n_lo, n_hi, e_lo, e_hi): what an evaluation that may decide every tie either way can
        report for one direction ("ij" or "ji"); a kept tie's distance is below tau_d."""
        (n_s, e_s), n_t = (self.sure_ij, self.tie_ij) if direction == "ij" else (self.sure_ji, self.tie_ji)
        return n_s, n_s + n_t, e_s, e_s + n_t * tau_d


def _direction(fi, fj, T, intr, tau_d, tau_n, tau_c):
    n, e, nt, ok, tie, dist = reproject(fi, fj, T, intr, tau_d, tau_n, tau_c)
    sure = ok & ~tie
    return n, e, nt, (int(sure.sum()), float(dist[sure].sum()))


def verify_pair(fi, fj, T_ij, intr, tau_d=0.15, tau_n=0.9, tau_c=0.1):
    """Two-sided check of frames i, j under the relative transform T_ij (4x4, camera i -> j)."""
    T_ij = np.asarray(T_ij, dtype=np.float64)
    T_ji = np.linalg.inv(T_ij)
    n1, e1, t1, s1 = _direction(fi, fj, T_ij, intr, tau_d, tau_n, tau_c)
    n2, e2, t2, s2 = _direction(fj, fi, T_ji, intr, tau_d, tau_n, tau_c)
    return PairCheck(n1, n2, e1, e2, t1, t2, s1, s2)


def pair_valid(chk: PairCheck, intr, e_max=0.075, frac_min=0.02):
    return (chk.n_ij + chk.n_ji) >= frac_min * intr["W"] * intr["H"] and chk.mean <= e_max


def validate_chunk(frames, poses, intr, e_max=0.05, tau_d=0.15, tau_n=0.9, tau_c=0.1):
    """Sec. 4.2: every frame pair of a chunk at its local poses (n,4,4, camera -> chunk frame).
    Returns (valid, worst mean error, worst pair, per-pair checks)."""
    n = len(frames)
    worst, arg, checks = 0.0, (-1, -1), {}
    for i in range(n):
        for j in range(i + 1, n):
            chk = verify_pair(frames[i], frames[j], relative_from_poses(poses[i], poses[j]), intr, tau_d, tau_n, tau_c)
            checks[(i, j)] = chk
            if chk.n_ij + chk.n_ji > 0 and chk.mean > worst:
                worst, arg = chk.mean, (i, j)
    return worst <= e_max, worst, arg, checks


def relative_from_poses(Ti, Tj):
    """T_j^-1 T_i (FP64)."""
    return np.linalg.inv(np.asarray(Tj, dtype=np.float64)) @ np.asarray(Ti, dtype=np.float64)
