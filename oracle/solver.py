"""PCG, Gauss-Newton and the residual maximum (oracle, FP64).

Sec. 4.4: Gauss-Newton (no damping) whose normal equations are solved by a
preconditioned conjugate gradient with a Jacobi preconditioner.  Readings:
* the preconditioner is 6x6 block-Jacobi by default (inverse of each frame's diagonal
  block by Cholesky; a block that is not SPD falls back to its scalar diagonal; an
  all-zero block, a frame without constraints, gets a zero inverse so its update stays
  0); "jacobi" selects the paper's scalar diagonal;
* PCG starts at x = 0 and runs exactly n_pcg iterations, stopping early only if
  p.Ap <= 0 or r.z == 0;
* Gauss-Newton runs exactly n_gn iterations; the energy is recorded before every step
  and once more after the last one.
Sec. 4.4.1: r_max is the largest residual after the optimisation; read here as the
largest correspondence distance ||T_i p - T_j q|| (unweighted), with its pair.
"""
import dataclasses

import numpy as np

from . import lie, residuals, system
from .frames import Frame
from .system import SolveParams, SparsePair


def block_jacobi_inverse(A, kind="block"):
    """Preconditioner M^-1 as a dense matrix (block diagonal), plus per-block status flags."""
    m = A.shape[0]
    Minv = np.zeros_like(A)
    flags = []
    for k in range(m // 6):
        s = slice(6 * k, 6 * k + 6)
        B = A[s, s]
        if not np.any(B):
            flags.append("empty")
            continue
        if kind == "jacobi":
            d = np.diag(B)
            Minv[s, s] = np.diag(np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0))
            flags.append("ok")
            continue
        try:
            L = np.linalg.cholesky(B)
            Li = np.linalg.inv(L)
            Minv[s, s] = Li.T @ Li
            flags.append("ok")
        except np.linalg.LinAlgError:
            d = np.diag(B)
            Minv[s, s] = np.diag(np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0))
            flags.append("singular")
    return Minv, flags


def pcg(A, b, Minv, n_iter):
    """Preconditioned CG from x = 0 for exactly n_iter iterations (early stop on p.Ap <= 0 or r.z == 0)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = Minv @ r
    p = z.copy()
    rz = float(r @ z)
    iters = 0
    for _ in range(n_iter):
        if rz == 0.0:
            break
        Ap = A @ p
        pAp = float(p @ Ap)
        if pAp <= 0.0:
            break
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        z = Minv @ r
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        iters += 1
    return x, iters


def apply_step(poses, delta):
    """Frame a >= 1 takes delta[6(a-1):6a]; frame 0 (gauge) is unchanged."""
    out = poses.copy()
    for a in range(1, len(poses)):
        dlt = delta[6 * (a - 1): 6 * a]
        R, t = lie.apply_update(poses[a][:3, :3], poses[a][:3, 3], dlt)
        out[a] = lie.to44(R, t)
    return out


def r_max(poses, sparse_pairs):
    """Largest correspondence distance ||T_a p - T_b q|| and the (a, b) pair holding it."""
    best, arg = -1.0, (-1, -1)
    for sp in sparse_pairs:
        if sp.p.shape[0] == 0:
            continue
        r = residuals.sparse_residuals(poses[sp.a][:3, :3], poses[sp.a][:3, 3],
                                       poses[sp.b][:3, :3], poses[sp.b][:3, 3], sp.p, sp.q)
        d = np.sqrt(np.sum(r * r, axis=1))
        k = int(np.argmax(d))
        if d[k] > best:
            best, arg = float(d[k]), (sp.a, sp.b)
    return best, arg


@dataclasses.dataclass
class GNResult:
    poses: np.ndarray              # (n,4,4) final
    energy: list                   # n_gn + 1 values
    e_sparse: list
    e_geo: list
    e_photo: list
    n_dense: list
    deltas: list
    pose_history: list
    r_max: float
    r_max_pair: tuple
    pcg_iters: list


def gauss_newton(frames, intr, poses0, sparse_pairs, params: SolveParams, direct=False, assoc=None, pmap=None,
                 frame_keys=None):
    """Sec. 4.4 Gauss-Newton: n_gn linearisations, each solved by PCG (or Cholesky if direct).

    assoc, pmap, frame_keys: optional association provider (replayed decisions), parallel map over
    the directed pairs and the workers' frame keys, passed to system.assemble."""
    poses = np.array(poses0, dtype=np.float64)
    dense_pairs = system.dense_pair_set(poses, sparse_pairs, params.max_angle_deg) if params.dense_on else []
    res = GNResult(None, [], [], [], [], [], [], [poses.copy()], 0.0, (-1, -1), [])
    for k in range(params.n_gn):
        wd = params.w_dense_at(k)
        if assoc is not None:
            assoc.iteration = k
        S = system.assemble(frames, intr, poses, sparse_pairs, dense_pairs, params, wd, assoc, pmap, frame_keys)
        res.energy.append(S.energy)
        res.e_sparse.append(S.e_sparse)
        res.e_geo.append(S.e_geo)
        res.e_photo.append(S.e_photo)
        res.n_dense.append(S.n_dense)
        if direct:
            delta = np.linalg.solve(S.A, S.b)
            it = -1
        else:
            Minv, _ = block_jacobi_inverse(S.A, params.precond)
            delta, it = pcg(S.A, S.b, Minv, params.n_pcg)
        res.pcg_iters.append(it)
        res.deltas.append(delta)
        poses = apply_step(poses, delta)
        res.pose_history.append(poses.copy())
    wd = params.w_dense_at(params.n_gn - 1) if params.n_gn > 0 else params.w_dense
    if assoc is not None:
        assoc.iteration = params.n_gn
    S = system.assemble(frames, intr, poses, sparse_pairs, dense_pairs, params, wd, assoc, pmap, frame_keys)
    res.energy.append(S.energy)
    res.e_sparse.append(S.e_sparse)
    res.e_geo.append(S.e_geo)
    res.e_photo.append(S.e_photo)
    res.n_dense.append(S.n_dense)
    res.poses = poses
    res.r_max, res.r_max_pair = r_max(poses, sparse_pairs)
    res.dense_pairs = dense_pairs
    return res


# ------------------------------------------------------- problem-level helpers

def sparse_pairs_for(problem, frame_ids):
    """SparsePair list restricted to frame_ids (local index = position in frame_ids)."""
    loc = {int(f): k for k, f in enumerate(frame_ids)}
    out = []
    for k, (i, j) in enumerate(problem.pairs):
        if int(i) in loc and int(j) in loc:
            p, q = problem.pair_corr(k)
            a, b = loc[int(i)], loc[int(j)]
            if a < b:
                out.append(SparsePair(a, b, p, q))
            else:
                out.append(SparsePair(b, a, q, p))
    return out


def solve_frames(problem, frame_ids, init_poses, params: SolveParams, depth_min=0.1, depth_max=10.0,
                 frames_cache=None, direct=False, storage=None, assoc=None, pmap=None):
    """Gauss-Newton over the given frames (first one fixed) starting from init_poses (n,4,4);
    storage "bf16" / "fp16" evaluates the dense term on 16-bit stored frames."""
    if frames_cache is None:
        frames = [Frame(problem.depth[f], problem.lum[f], problem.intr, depth_min, depth_max, storage)
                  for f in frame_ids]
    else:
        frames = [frames_cache[f] for f in frame_ids]
    sp = sparse_pairs_for(problem, frame_ids)
    return gauss_newton(frames, problem.intr, init_poses, sp, params, direct=direct, assoc=assoc, pmap=pmap)


@dataclasses.dataclass
class PrunedResult:
    result: GNResult           # the last solve
    pruned: list               # (a, b) local pair indices removed, in order
    invalid: list              # local frame indices (not the fixed frame 0) left without any pair
    rounds: int                # solves run


def gauss_newton_pruned(frames, intr, poses0, sparse_pairs, params: SolveParams, prune_rmax, max_rounds=8, assoc=None):
    """Sec. 4.4.1 correspondence pruning around the solve.

    After a solve, r_max is the largest sparse correspondence distance ||T_a p - T_b q||.  If it
    exceeds prune_rmax, every correspondence of the pair (a, b) holding it is removed and the
    problem is solved again; at most max_rounds re-solves.  Reading (the paper does not say from
    where the next solve starts): each re-solve starts from the same initial poses, so the result
    is the solve of the pruned problem.  The dense pair set follows the remaining sparse pairs.
    A frame left with no pair is marked invalid (it keeps its initial pose: no constraint moves it).
    """
    sp = list(sparse_pairs)
    pruned = []
    rounds = 0
    while True:
        res = gauss_newton(frames, intr, poses0, sp, params, assoc=assoc)
        rounds += 1
        if not (res.r_max > prune_rmax) or rounds > max_rounds:
            break
        a, b = res.r_max_pair
        pruned.append((a, b))
        sp = [p for p in sp if not (p.a == a and p.b == b)]
    linked = set()
    for p in sp:
        if p.p.shape[0] > 0:
            linked.update((p.a, p.b))
    invalid = [k for k in range(1, len(frames)) if k not in linked]
    return PrunedResult(res, pruned, invalid, rounds)
