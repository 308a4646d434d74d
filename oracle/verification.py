"""Dense verification of a frame pair and chunk validation (oracle, Sec. 4.1.1 and Sec. 4.2).

Test-infrastructure only: the CUDA library never imports this package.

Sec. 4.1.1 aligns frames f_i and f_j with a relative transform T_ij (camera i -> camera j),
re-projects every pixel of one frame into the other in both directions, and keeps a pixel
correspondence when its depth discrepancy, normal deviation and photoconsistency pass three
gates; the pair is rejected if the re-projection error of the kept correspondences is too
large or too few of them exist.  Sec. 4.2 applies the same test to every frame pair of a chunk
at its optimised local poses and discards the chunk if any pair's error is too large.

Readings (the paper states the gates and thresholds but not every detail):

* the correspondence of source pixel (x, y) is the nearest target pixel of pi(T_ij p) (the same
  projective association as the dense energy, Sec. 4.3, without its bilinear border), inside
  the image, with valid depth and normal on both sides;
* gates: ||T_ij p - q|| < tau_d, (R_ij n_i) . n_j > tau_n, |C_i(x, y) - C_j(target)| < tau_c,
  where C is the frame's intensity (the luminance given with the depth);
* the re-projection error of the pair is the mean distance over the kept correspondences of
  both directions, sum(E_ij + E_ji) / (n_ij + n_ji); the pair is valid iff that mean is at most
  e_max (0.075 m) and n_ij + n_ji >= frac_min * w * h (frac_min = 0.02);
* chunk validation: every pair of the chunk's frames at the optimised local poses; the chunk is
  invalid if some pair with kept correspondences has a mean error above 0.05 m.

The gate decisions are taken in IEEE FP32 in the same operation order as the association of
the dense energy (association.py) and as the GPU kernel; the distances are summed in FP64.
"""
import dataclasses

import numpy as np

from . import association

f32 = np.float32


def inverse_transform32(R, t):
    """FP32 rounding of T^-1 for an FP64 rigid transform (R^T, -R^T t summed left to right)."""
    Ri = np.array([[R[b, a] for b in range(3)] for a in range(3)])
    ti = np.array([-((R[0, a] * t[0] + R[1, a] * t[1]) + R[2, a] * t[2]) for a in range(3)])
    return Ri.astype(f32), ti.astype(f32)


def reproject(fi, fj, M32, intr, tau_d=0.15, tau_n=0.9, tau_c=0.1):
    """One direction i -> j under M32 = fl32(T_ij): the kept correspondences' count and the FP64
    sum of their distances ||T_ij p - q||, plus the per-pixel mask."""
    R, t = M32
    W, H = intr["W"], intr["H"]
    kx, ky = association.ray_tables(intr)
    fx, fy, cx, cy = f32(intr["fx"]), f32(intr["fy"]), f32(intr["cx"]), f32(intr["cy"])
    ys, xs = np.divmod(np.arange(W * H), W)
    z = fi.D32.ravel()
    n_i = fi.N32.reshape(-1, 3)
    ok = fi.valid.ravel() & fi.nvalid.ravel()
    dx = kx[xs] * z
    dy = ky[ys] * z
    dz = z
    Y = [((R[a, 0] * dx + R[a, 1] * dy) + R[a, 2] * dz) + t[a] for a in range(3)]
    ok &= Y[2] > f32(0)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        iz = f32(1) / np.where(ok, Y[2], f32(1))
        ux = fx * (Y[0] * iz) + cx
        uy = fy * (Y[1] * iz) + cy
    ux = np.where(ok, ux, f32(-100))
    uy = np.where(ok, uy, f32(-100))
    nxf = np.floor(ux + f32(0.5))
    nyf = np.floor(uy + f32(0.5))
    ok &= (nxf >= 0) & (nxf <= W - 1) & (nyf >= 0) & (nyf <= H - 1)
    nx = np.where(ok, nxf, 0).astype(np.int64)
    ny = np.where(ok, nyf, 0).astype(np.int64)
    tgt = ny * W + nx
    ok &= fj.valid.ravel()[tgt] & fj.nvalid.ravel()[tgt]
    Dj = fj.D32.ravel()[tgt]
    qx = kx[nx] * Dj
    qy = ky[ny] * Dj
    qz = Dj
    ex, ey, ez = Y[0] - qx, Y[1] - qy, Y[2] - qz
    dist2 = (ex * ex + ey * ey) + ez * ez
    ok &= dist2 < f32(tau_d * tau_d)
    m = [(R[a, 0] * n_i[:, 0] + R[a, 1] * n_i[:, 1]) + R[a, 2] * n_i[:, 2] for a in range(3)]
    n_j = fj.N32.reshape(-1, 3)[tgt]
    dot = (m[0] * n_j[:, 0] + m[1] * n_j[:, 1]) + m[2] * n_j[:, 2]
    ok &= dot > f32(tau_n)
    ok &= np.abs(fi.C32.ravel() - fj.C32.ravel()[tgt]) < f32(tau_c)
    # distances of the kept correspondences in FP64 (camera-j coordinates)
    Ty = np.stack([Y[0], Y[1], Y[2]], axis=1).astype(np.float64)
    q = np.stack([qx, qy, qz], axis=1).astype(np.float64)
    d = np.sqrt(np.sum((Ty - q) ** 2, axis=1))
    return int(ok.sum()), float(d[ok].sum()), ok


@dataclasses.dataclass
class PairCheck:
    n_ij: int
    n_ji: int
    e_ij: float
    e_ji: float

    @property
    def mean(self):
        n = self.n_ij + self.n_ji
        return (self.e_ij + self.e_ji) / n if n else float("inf")


def verify_pair(fi, fj, T_ij, intr, tau_d=0.15, tau_n=0.9, tau_c=0.1):
    """Two-sided check of frames i, j under the relative transform T_ij (4x4, camera i -> j)."""
    R, t = np.asarray(T_ij, dtype=np.float64)[:3, :3], np.asarray(T_ij, dtype=np.float64)[:3, 3]
    M_ij = (R.astype(f32), t.astype(f32))
    M_ji = inverse_transform32(R, t)
    n1, e1, _ = reproject(fi, fj, M_ij, intr, tau_d, tau_n, tau_c)
    n2, e2, _ = reproject(fj, fi, M_ji, intr, tau_d, tau_n, tau_c)
    return PairCheck(n1, n2, e1, e2)


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
    """T_j^-1 T_i in FP64 with the explicit sums of association.pair_transform32 (before rounding)."""
    Ri, ti, Rj, tj = Ti[:3, :3], Ti[:3, 3], Tj[:3, :3], Tj[:3, 3]
    R = np.zeros((3, 3))
    t = np.zeros(3)
    dt = [ti[0] - tj[0], ti[1] - tj[1], ti[2] - tj[2]]
    for a in range(3):
        for b in range(3):
            R[a, b] = (Rj[0, a] * Ri[0, b] + Rj[1, a] * Ri[1, b]) + Rj[2, a] * Ri[2, b]
        t[a] = (Rj[0, a] * dt[0] + Rj[1, a] * dt[1]) + Rj[2, a] * dt[2]
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, t
    return T
