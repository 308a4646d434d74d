"""Key-point correspondence filter and surface-area filter (oracle, Sec. 4.1.1).

Test-infrastructure only: the CUDA library never imports this package.

For one frame pair with matched 3D points P (frame i) and Q (frame j), listed in order of match
distance, the filter grows a set of correspondences one at a time.  After each addition the
rigid transform T_ij (q ~ R p + t) minimising the RMSD over the set is fitted (Kabsch); the set
is rejected as it stands when the largest residual ||R p + t - q|| exceeds 0.02 m or the fit is
ambiguous (a condition number above 100), and then correspondences are removed, largest
residual first, until the set passes or fewer than 3 remain.  A pair keeps its correspondences
only if at least N_min = 5 survive (Sec. 4.1.1: 3 define a transform, 5 is the paper's choice).

Readings (the paper names the analysis but not its formulas):

* condition number of a 3x3 matrix M = sigma_1 / sigma_2, its two largest singular values, for
  M = the covariance of the set's P points, of its Q points, and their cross-covariance; a
  ratio above 100 means the points (or their correspondence) are nearly collinear, which leaves
  a rotation undetermined.  (sigma_1 / sigma_3 would reject every planar set, and a rigid
  transform is well defined by non-collinear points on a plane.)
* a tie for the largest residual removes the earliest correspondence of the set;
* surface area of a point set = area of its bounding rectangle in the plane of its two principal
  axes (the covariance's two leading eigenvectors); the pair is discarded if the area spanned
  by its kept P points or by its kept Q points is below 0.032 m^2.
"""
import dataclasses

import numpy as np


def kabsch(P, Q):
    """R, t minimising sum ||R p + t - q||^2 (SVD of the cross-covariance, reflection fixed)."""
    pc, qc = P.mean(axis=0), Q.mean(axis=0)
    H = (P - pc).T @ (Q - qc)
    U, _, Vt = np.linalg.svd(H)
    d = np.sign(np.linalg.det(Vt.T @ U.T))
    D = np.diag([1.0, 1.0, d if d != 0 else 1.0])
    R = Vt.T @ D @ U.T
    return R, qc - R @ pc


def cond12(M):
    """sigma_1 / sigma_2 of a 3x3 matrix (inf if sigma_2 is 0)."""
    s = np.linalg.svd(M, compute_uv=False)
    return s[0] / s[1] if s[1] > 0 else np.inf


def stable(P, Q, cond_max=100.0):
    Pc, Qc = P - P.mean(axis=0), Q - Q.mean(axis=0)
    return max(cond12(Pc.T @ Pc), cond12(Qc.T @ Qc), cond12(Pc.T @ Qc)) <= cond_max


@dataclasses.dataclass
class FilterResult:
    keep: list          # indices of the kept correspondences, in the set's order
    R: np.ndarray       # fitted T_ij (None when rejected)
    t: np.ndarray
    status: int         # 0 kept, 1 fewer than n_min survive, 2 surface area too small


def surface_area(X):
    """Bounding-rectangle area of the points in the plane of their two principal axes."""
    Xc = X - X.mean(axis=0)
    w, V = np.linalg.eigh(Xc.T @ Xc)
    e1, e2 = V[:, 2], V[:, 1]
    a, b = Xc @ e1, Xc @ e2
    return float((a.max() - a.min()) * (b.max() - b.min()))


def filter_pair(P, Q, max_residual=0.02, cond_max=100.0, n_min=5, min_area=0.032):
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    S = []
    for k in range(len(P)):
        S.append(k)
        while len(S) >= 3:
            R, t = kabsch(P[S], Q[S])
            res = np.linalg.norm(P[S] @ R.T + t - Q[S], axis=1)
            if res.max() <= max_residual and stable(P[S], Q[S], cond_max):
                break
            S.pop(int(np.argmax(res)))
    if len(S) < max(n_min, 3):
        return FilterResult([], None, None, 1)
    R, t = kabsch(P[S], Q[S])
    if min(surface_area(P[S]), surface_area(Q[S])) < min_area:
        return FilterResult([], None, None, 2)
    return FilterResult(S, R, t, 0)
