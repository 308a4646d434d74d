"""TSDF integration and de-integration on sparse voxel blocks (oracle, Sec. 5.1-5.3).

Test-infrastructure only: the CUDA library never imports this package.

Sec. 5.2 updates every voxel v touched by a depth frame D_i with the weighted running average
D' = (D W + w_i d_i) / (W + w_i), W' = W + w_i, and removes a frame with the inverse formula
(minus signs), so that re-integrating a frame at a new pose is de-integrate + integrate.
Sec. 5.1 stores the field in 8x8x8-voxel blocks addressed by spatial hashing (4 mm voxels by
default).  Sec. 5.3 re-integrates the frames whose integrated and optimised poses differ most,
by the distance ||s * (t_int - t_opt)||, s = (2, 2, 2, 1, 1, 1), over Euler angles and
translations, N_fix = 10 frames per update.

Readings (the paper leaves these open):

* a voxel keeps the integer sums S = sum w d_q, W = sum w and SC = sum w c_q, with the truncated
  signed distance quantised to q = 2^-20 m (d_q = round(sdf / q)) and the intensity to
  c_q = round(65535 c); the paper's D is S q / W.  Integer sums make de-integration the exact
  inverse of integration in any order, which the paper asks for ("one inverts the other");
* w_i = 1 for every sample (the paper names a per-sample weight but gives none);
* d_i(v) = D_i(u) - z, z the voxel centre's depth in camera i, u the nearest pixel of its
  projection (inside the image, valid depth); voxels with d < -mu are left alone and the
  others get sdf = min(d, mu); truncation mu = 5 voxels;
* a frame touches the blocks that contain one of its band samples: for every valid pixel, the
  points of its ray at depths D + k h, h = half a voxel, k = -K..K with K h >= mu; the frame
  updates the voxels of those blocks only, and de-integrating at the same pose touches the
  same blocks;
* every floating-point step that decides an integer (a block coordinate, a pixel, a
  quantised value) is taken in IEEE FP32 in the operation order written below, the same as on
  the device, from the pose rounded to FP32;
* Euler angles of a rotation R = Rz(gamma) Ry(beta) Rx(alpha): alpha = atan2(R21, R22),
  beta = asin(-R20), gamma = atan2(R10, R00).
"""
import math

import numpy as np

f32 = np.float32
Q_SDF = 2.0 ** -20
C_SCALE = 65535.0


class Params:
    def __init__(self, voxel=0.004, trunc_voxels=5):
        self.voxel = voxel
        self.mu = f32(trunc_voxels * voxel)
        self.h = f32(0.5 * voxel)
        self.K = int(math.ceil(trunc_voxels * 2))  # K h >= mu with h = voxel / 2
        self.inv_block = f32(1.0 / (8.0 * voxel))
        self.vs = f32(voxel)
        self.inv_q = f32(1.0 / Q_SDF)


def ray_tables(intr):
    """kx[x] = fl32((x - cx) / fx), ky[y] = fl32((y - cy) / fy): each computed in FP64, rounded once."""
    W, H = intr["W"], intr["H"]
    kx = ((np.arange(W, dtype=np.float64) - intr["cx"]) / intr["fx"]).astype(f32)
    ky = ((np.arange(H, dtype=np.float64) - intr["cy"]) / intr["fy"]).astype(f32)
    return kx, ky


def pose32(T):
    T = np.asarray(T, dtype=np.float64)
    return T[:3, :3].astype(f32), T[:3, 3].astype(f32)


def band_blocks(depth, intr, T, prm: Params):
    """Block coordinates (set of (bx, by, bz)) containing a band sample of a frame at pose T."""
    R, t = pose32(T)
    kx, ky = ray_tables(intr)
    H, W = depth.shape
    ys, xs = np.divmod(np.arange(W * H), W)
    D = np.asarray(depth, dtype=f32).ravel()
    ok = D > f32(0)
    xs, ys, D = xs[ok], ys[ok], D[ok]
    out = set()
    for k in range(-prm.K, prm.K + 1):
        z = D + f32(k) * prm.h
        m = z > f32(0)
        zz = z[m]
        c = [kx[xs[m]] * zz, ky[ys[m]] * zz, zz]
        p = [((R[a, 0] * c[0] + R[a, 1] * c[1]) + R[a, 2] * c[2]) + t[a] for a in range(3)]
        b = [np.floor(p[a] * prm.inv_block).astype(np.int64) for a in range(3)]
        out.update(zip(b[0].tolist(), b[1].tolist(), b[2].tolist()))
    return out


def voxel_centres(key, prm: Params):
    """FP32 world centres of a block's 512 voxels, index i = ix + 8 iy + 64 iz."""
    bx, by, bz = key
    i = np.arange(512)
    ix, iy, iz = i % 8, (i // 8) % 8, i // 64
    cx = (np.float32(8 * bx) + ix.astype(f32) + f32(0.5)) * prm.vs
    cy = (np.float32(8 * by) + iy.astype(f32) + f32(0.5)) * prm.vs
    cz = (np.float32(8 * bz) + iz.astype(f32) + f32(0.5)) * prm.vs
    return cx.astype(f32), cy.astype(f32), cz.astype(f32)


def integrate(volume, depth, color, intr, T, prm: Params, sign=1):
    """Add (sign = +1) or remove (-1) one frame.  volume: dict key -> int64 array (3, 512) with
    rows S, W, SC; blocks are created on first touch and never dropped."""
    R, t = pose32(T)
    kx, ky = ray_tables(intr)
    fx, fy, cx, cy = f32(intr["fx"]), f32(intr["fy"]), f32(intr["cx"]), f32(intr["cy"])
    H, W = depth.shape
    D = np.asarray(depth, dtype=f32).ravel()
    C = np.asarray(color, dtype=f32).ravel()
    for key in sorted(band_blocks(depth, intr, T, prm)):
        blk = volume.setdefault(key, np.zeros((3, 512), dtype=np.int64))
        v = voxel_centres(key, prm)
        d = [v[a] - t[a] for a in range(3)]
        c = [(R[0, a] * d[0] + R[1, a] * d[1]) + R[2, a] * d[2] for a in range(3)]  # R^T (v - t)
        ok = c[2] > f32(0)
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            iz = f32(1) / np.where(ok, c[2], f32(1))
            ux = fx * (c[0] * iz) + cx
            uy = fy * (c[1] * iz) + cy
        ux = np.where(ok, ux, f32(-100))
        uy = np.where(ok, uy, f32(-100))
        px, py = np.floor(ux + f32(0.5)), np.floor(uy + f32(0.5))
        ok &= (px >= 0) & (px <= W - 1) & (py >= 0) & (py <= H - 1)
        pix = np.where(ok, py * W + px, 0).astype(np.int64)
        Dv = D[pix]
        ok &= Dv > f32(0)
        sd = Dv - c[2]
        ok &= sd >= -prm.mu
        sdf = np.minimum(sd, prm.mu)
        dq = np.rint(sdf * prm.inv_q).astype(np.int64)
        cq = np.rint(C[pix] * f32(C_SCALE)).astype(np.int64)
        blk[0] += sign * np.where(ok, dq, 0)
        blk[1] += sign * ok.astype(np.int64)
        blk[2] += sign * np.where(ok, cq, 0)
    return volume


def tsdf_value(blk):
    """The paper's D (metres) and W of a block's voxels (D = 0 where W = 0)."""
    S, Wt = blk[0].astype(np.float64), blk[1].astype(np.float64)
    return np.where(Wt > 0, S * Q_SDF / np.maximum(Wt, 1), 0.0), Wt


def euler(R):
    return np.array([math.atan2(R[2, 1], R[2, 2]), math.asin(max(-1.0, min(1.0, -R[2, 0]))),
                     math.atan2(R[1, 0], R[0, 0])])


def pose_distance(Ta, Tb):
    """Sec. 5.3: ||s * (t_a - t_b)|| over (Euler angles, translation), s = (2, 2, 2, 1, 1, 1)."""
    va = np.concatenate([euler(Ta[:3, :3]), Ta[:3, 3]])
    vb = np.concatenate([euler(Tb[:3, :3]), Tb[:3, 3]])
    s = np.array([2.0, 2.0, 2.0, 1.0, 1.0, 1.0])
    return float(np.linalg.norm(s * va - s * vb))


def reintegration_order(integrated, optimised, n_fix=10):
    """Frame ids to re-integrate: descending distance, the first n_fix with distance > 0 (ties:
    smaller id first)."""
    d = [(-pose_distance(integrated[f], optimised[f]), f) for f in integrated]
    return [f for nd, f in sorted(d) if nd < 0][:n_fix]
