"""Dense projective association for a directed frame pair i -> j (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 4.3 (dense matching) maps the 3D point d_ik of source pixel k into frame j through
T_j^-1 T_i, projects it with pi, reads D_j there, ignores projections outside the frame, and
prunes ICP-style by distance and normal.  Readings used (the paper gives no numbers for this
pruning):

* the association is recomputed once per Gauss-Newton iteration at the current poses and held
  fixed inside the linearisation (projective, "ICP-like");
* y = T_j^-1 T_i d with d = pi^-1(x, y, D_i(x, y)); y_z must be positive;
* target pixel = nearest pixel of u = pi(y): (floor(u_x + 1/2), floor(u_y + 1/2)), with valid
  depth and a valid normal, on the 3-pixel interior (3 <= x <= W - 4, 3 <= y <= H - 4);
* the photometric term samples I_j and grad I_j bilinearly at u from the four pixels around it,
  (floor(u_x), floor(u_y)) and its +1 neighbours, which the 3-pixel interior of the nearest pixel
  keeps on the 2-pixel interior where grad I is defined.  (Every threshold on u then sits at a
  half-integer: an integer projection, as of every pixel of an identity relative pose, at which
  Sec. 4.2 starts every chunk, is never on one.  A test on the taps themselves would put the
  thresholds at integers, where identity poses place whole image columns and rows.)
* gates ||y - q|| < tau_d (q = pi^-1 of the target pixel; the distance of Sec. 4.1.1 between the
  world points T_i d and T_j q, measured in camera j) and (R n_i) . n_j > tau_n with the dense
  verification constants of Sec. 4.1.1 (tau_d = 0.15 m, tau_n = 0.9);
* the photometric and geometric residuals share one validity mask;
* the source pixel needs valid depth and a valid normal.

Everything here is FP64 from the frames' FP64 planes.  Every decision is a comparison of a
computed value with a threshold; ``associate`` also returns each pixel's distance to the
nearest threshold it was compared with (``margin_px`` in pixels for the rounding and interior
tests, ``margin_d`` in metres for the distance gate, ``margin_n`` for the normal gate),
so that a caller comparing with an implementation in lower precision can tell a decision that
sits within that precision's rounding of its threshold (either outcome is correct there) from a
real disagreement (see ``ties``).
"""
import numpy as np


def relative_transform(Ri, ti, Rj, tj):
    """T_j^-1 T_i as (R, t): R = R_j^T R_i, t = R_j^T (t_i - t_j) (FP64)."""
    Ri, ti, Rj, tj = (np.asarray(v, dtype=np.float64) for v in (Ri, ti, Rj, tj))
    return Rj.T @ Ri, Rj.T @ (ti - tj)


def associate(fi, fj, M, intr, tau_d=0.15, tau_n=0.9):
    """Association of every source pixel of frame i into frame j under M = T_j^-1 T_i.

    fi, fj: frames.Frame; M: (R, t) from relative_transform.  Returns a dict of flat arrays over
    the source pixels (row-major): valid (bool), nx, ny (nearest target pixel), bx, by (bilinear
    base tap), ux, uy (the projection), and the decision margins margin_px, margin_d, margin_n
    (+inf where a test was not reached).
    """
    R, t = (np.asarray(v, dtype=np.float64) for v in M)
    W, H = intr["W"], intr["H"]
    fx, fy, cx, cy = (float(intr[k]) for k in ("fx", "fy", "cx", "cy"))
    n_px = W * H
    ys, xs = np.divmod(np.arange(n_px), W)
    z = fi.D.ravel()
    d = np.stack([(xs - cx) * z / fx, (ys - cy) * z / fy, z], axis=1)
    y = d @ R.T + t
    ok = fi.valid.ravel() & fi.nvalid.ravel() & (y[:, 2] > 0)
    yz = np.where(ok, y[:, 2], 1.0)
    ux = np.where(ok, fx * y[:, 0] / yz + cx, -100.0)
    uy = np.where(ok, fy * y[:, 1] / yz + cy, -100.0)
    margin_px = np.full(n_px, np.inf)
    margin_d = np.full(n_px, np.inf)
    margin_n = np.full(n_px, np.inf)
    # nearest pixel on the 3-pixel interior; the rounding boundaries (u + 1/2 an integer) include
    # the interior's edges 2.5 and W - 3.5
    nxf = np.floor(ux + 0.5)
    nyf = np.floor(uy + 0.5)
    mr = np.minimum(np.abs(ux + 0.5 - np.round(ux + 0.5)), np.abs(uy + 0.5 - np.round(uy + 0.5)))
    margin_px = np.where(ok, mr, margin_px)
    ok &= (nxf >= 3) & (nxf <= W - 4) & (nyf >= 3) & (nyf <= H - 4)
    # bilinear base tap; floor(u) >= nearest - 1 >= 2 and floor(u) + 1 <= nearest + 1 <= W - 3
    bxf = np.floor(ux)
    byf = np.floor(uy)
    nx = np.where(ok, nxf, 0).astype(np.int64)
    ny = np.where(ok, nyf, 0).astype(np.int64)
    bx = np.where(ok, bxf, 0).astype(np.int64)
    by = np.where(ok, byf, 0).astype(np.int64)
    tgt = ny * W + nx
    ok &= fj.valid.ravel()[tgt] & fj.nvalid.ravel()[tgt]
    Dj = fj.D.ravel()[tgt]
    q = np.stack([(nx - cx) * Dj / fx, (ny - cy) * Dj / fy, Dj], axis=1)
    dist = np.sqrt(np.sum((y - q) ** 2, axis=1))
    margin_d = np.where(ok, np.abs(dist - tau_d), margin_d)
    ok &= dist < tau_d
    ndot = np.sum((fi.N.reshape(-1, 3) @ R.T) * fj.N.reshape(-1, 3)[tgt], axis=1)
    margin_n = np.where(ok, np.abs(ndot - tau_n), margin_n)
    ok &= ndot > tau_n
    return dict(valid=ok, nx=nx, ny=ny, bx=bx, by=by, ux=ux, uy=uy,
                margin_px=margin_px, margin_d=margin_d, margin_n=margin_n)


def targets(asc, W):
    """Flat target index per source pixel, -1 where the pixel has no association."""
    return np.where(asc["valid"], asc["ny"] * W + asc["nx"], -1)


def ties(asc, eps_px, eps_d, eps_n):
    """Pixels whose outcome depends on a comparison within (eps_px, eps_d, eps_n) of its threshold.

    Any decision taken on such a pixel by an evaluation whose rounding error stays below those
    bounds is as correct as this one; everywhere else both must agree."""
    return (asc["margin_px"] < eps_px) | (asc["margin_d"] < eps_d) | (asc["margin_n"] < eps_n)


def replay(asc_own, target, W, H):
    """An association with the decisions given by ``target`` (flat target index or -1 per source
    pixel, e.g. another implementation's) and this oracle's own projection for the bilinear taps.

    Used to compare residual and normal-equation arithmetic on identical decisions; the given
    decisions must first be checked against ``asc_own`` (they may differ only on ties)."""
    target = np.asarray(target).ravel()
    valid = target >= 0
    ny, nx = np.divmod(np.where(valid, target, 0), W)
    # the base tap of a pixel that another evaluation kept next to the interior's edge may round to
    # the other side here; clamping moves it by one pixel, where the bilinear weight is within
    # rounding of 0 or 1 and the interpolated value is the same
    bx = np.where(valid, np.clip(np.floor(np.where(valid, asc_own["ux"], 2.0)), 2, W - 4), 0).astype(np.int64)
    by = np.where(valid, np.clip(np.floor(np.where(valid, asc_own["uy"], 2.0)), 2, H - 4), 0).astype(np.int64)
    return dict(valid=valid, nx=nx.astype(np.int64), ny=ny.astype(np.int64), bx=bx, by=by,
                ux=asc_own["ux"], uy=asc_own["uy"])


# Rounding-error bounds of an FP32 evaluation of the decisions above, at the workloads' scales
# (depths 0.1-10 m, focal lengths up to 262.5 px, relative motions of metres): the projection u
# within EPS_PX pixels, the distance ||y - q|| within EPS_D metres and the normal cosine within
# EPS_N (FP32 normals from central differences of FP32 points: the cancellation of
# P(x+1) - P(x-1) leaves ~1e-5).  A decision whose margin is below its bound is a tie.
EPS_PX, EPS_D, EPS_N = 5e-4, 2e-5, 2e-4


def check_replay(own, target, W, H, eps=(EPS_PX, EPS_D, EPS_N), own_replay=None):
    """Check another implementation's decisions ``target`` (flat target index or -1 per source pixel)
    against this oracle's association ``own`` (taken at the poses those decisions were taken at):
    they may differ only on ties.  Returns the replayed association (with the bilinear taps of
    ``own_replay``, this oracle's association at its own poses, default ``own``), the number of
    valid pixels (of own), the number of differing decisions (flips), and None or the description
    of the first disagreement outside the rounding bounds."""
    target = np.asarray(target).ravel()
    ref = targets(own, W)
    diff = target != ref
    bad = np.flatnonzero(diff & ~ties(own, *eps))
    err = None
    if len(bad):
        k = bad[0]
        err = (f"{len(bad)} decisions differ outside the rounding bounds; first at pixel {k}: other {target[k]}, "
               f"oracle {ref[k]} (u = {own['ux'][k]:.6f}, {own['uy'][k]:.6f}; margins {own['margin_px'][k]:.3g} px, "
               f"{own['margin_d'][k]:.3g} m, {own['margin_n'][k]:.3g})")
    return replay(own if own_replay is None else own_replay, target, W, H), int((ref >= 0).sum()), int(diff.sum()), err


class CheckedReplay:
    """Association provider for system.assemble that replays another implementation's decisions.

    fetch(i, j, poses) returns that implementation's flat target index (or -1) per source pixel of
    the directed pair i -> j; check_poses(i, j), if defined, the 4x4 poses of i and j at which it
    took them (None: the poses the oracle passes).  The oracle checks them against its own
    association at those poses with check_replay (AssertionError on a disagreement outside the
    rounding bounds) and replays them at its own poses.  ``iteration`` is set by the Gauss-Newton
    loop before each assembly (its linearisation index; n_gn for the final energy).  Counts the
    valid pixels (of the oracle's association) and the differing decisions (flips)."""

    def __init__(self, fetch, W, H, eps=(EPS_PX, EPS_D, EPS_N)):
        self.fetch, self.W, self.H, self.eps = fetch, W, H, eps
        self.n_valid = 0
        self.n_flips = 0
        self.calls = 0
        self.iteration = 0

    def check_poses(self, i, j):
        return None

    def record(self, n_valid, n_flips, err, i, j):
        if err:
            raise AssertionError(f"evaluation {self.iteration}, pair {i}->{j}: {err}")
        self.n_valid += n_valid
        self.n_flips += n_flips
        self.calls += 1

    def __call__(self, i, j, poses, own):
        rep, nv, nf, err = check_replay(own, self.fetch(i, j, poses), self.W, self.H, self.eps)
        self.record(nv, nf, err, i, j)
        return rep
