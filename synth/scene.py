"""Seeded synthetic scenes, trajectories and correspondences.

Input generation only: nothing here evaluates the alignment energy, its
derivatives or the solver.  The oracle and the CUDA library both read what this
module produces; neither is imported here.

World frame: y points down (like the camera's y axis), so a camera with
identity rotation looks horizontally along +z.  Scenes are "box rooms": a room
shell plus random axis-aligned boxes standing on the floor, rendered by the
analytic ray caster in ``render.c``.
"""
from __future__ import annotations

import ctypes
import os
import pathlib

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_LIB = None
TEX_STRIDE = 16


def build_renderer(force: bool = False) -> pathlib.Path:
    """Compile render.c into synth/_render.so with gcc (deterministic flags)."""
    out = _HERE / "_render.so"
    src = _HERE / "render.c"
    if force or not out.exists() or out.stat().st_mtime < src.stat().st_mtime:
        cmd = (f"gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC "
               f"{src} -o {out}.tmp -lm && mv {out}.tmp {out}")
        if os.system(cmd) != 0:
            raise RuntimeError("failed to build the synthetic renderer: " + cmd)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        path = build_renderer()
        lib = ctypes.CDLL(str(path))
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.synth_render.argtypes = [i, i, i, d, d, d, d, p, i, p, p, p, p, p, p]
        lib.synth_render.restype = None
        _LIB = lib
    return _LIB


# ----------------------------------------------------------------------------
# small rigid-motion helpers (generator-local; the solver has its own)
# ----------------------------------------------------------------------------

def rot_axis_angle(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    n = np.linalg.norm(axis)
    if n == 0.0 or angle == 0.0:
        return np.eye(3)
    k = axis / n
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


def rot_from_vec(v):
    v = np.asarray(v, dtype=np.float64)
    a = np.linalg.norm(v)
    return rot_axis_angle(v, a) if a > 0 else np.eye(3)


def make_pose(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def yaw_pitch_roll(yaw, pitch, roll):
    """Camera orientation: yaw about world y (down), then pitch about x, roll about z."""
    return rot_axis_angle([0, 1, 0], yaw) @ rot_axis_angle([1, 0, 0], pitch) @ rot_axis_angle([0, 0, 1], roll)


# ----------------------------------------------------------------------------
# intrinsics
# ----------------------------------------------------------------------------

def intrinsics(W: int, H: int):
    """Kinect-like fx=fy=525 at 640x480, scaled; pixel centres at integers."""
    s = W / 640.0
    fx = fy = 525.0 * s
    cx = (W - 1) / 2.0
    cy = (H - 1) / 2.0
    return dict(W=W, H=H, fx=fx, fy=fy, cx=cx, cy=cy)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def _random_texture(rng):
    tp = np.zeros(TEX_STRIDE)
    tp[0] = rng.uniform(0.3, 0.7)
    for k in range(3):
        amp = rng.uniform(0.03, 0.15)
        f = rng.uniform(0.8, 6.0)
        ang = rng.uniform(0, 2 * np.pi)
        tp[1 + 4 * k: 5 + 4 * k] = [amp, f * np.cos(ang), f * np.sin(ang), rng.uniform(0, 2 * np.pi)]
    if rng.uniform() < 0.7:
        tp[13] = rng.uniform(0.15, 0.6)
        tp[14] = rng.uniform(0.1, 0.4)
        tp[15] = rng.uniform(0, 1)
    return tp


class Scene:
    """Axis-aligned boxes with per-face textures."""

    def __init__(self, lo, hi, kind, tex):
        self.lo = np.ascontiguousarray(lo, dtype=np.float64)
        self.hi = np.ascontiguousarray(hi, dtype=np.float64)
        self.kind = np.ascontiguousarray(kind, dtype=np.int32)
        self.tex = np.ascontiguousarray(tex, dtype=np.float64)

    @property
    def n_boxes(self):
        return len(self.kind)

    def free(self, p, margin=0.3):
        """True if point p is inside the room shell and outside every solid box (with margin)."""
        for lo, hi, k in zip(self.lo, self.hi, self.kind):
            inside = np.all(p > lo - margin) and np.all(p < hi + margin)
            inside_strict = np.all(p > lo + margin) and np.all(p < hi - margin)
            if k == 0 and not inside_strict:
                return False
            if k == 1 and inside:
                return False
        return True


def box_room(rng, size=(8.0, 2.8, 8.0), n_boxes=(20, 60), keep_clear=None, clear_radius=0.8):
    """Room shell centred at the origin (floor at +size_y/2) with random boxes on the floor.

    keep_clear: optional (k,3) array of points no box may come closer to (horizontally)
    than clear_radius, so camera paths stay in free space.
    """
    sx, sy, sz = size
    lo = [[-sx / 2, -sy / 2, -sz / 2]]
    hi = [[sx / 2, sy / 2, sz / 2]]
    kind = [0]
    nb = int(rng.integers(n_boxes[0], n_boxes[1] + 1))
    floor = sy / 2
    tries = 0
    while len(kind) < nb + 1 and tries < 2000:
        tries += 1
        w = rng.uniform(0.2, 1.2, size=3)
        w[1] = rng.uniform(0.2, 1.6)
        cx = rng.uniform(-sx / 2 + w[0] / 2, sx / 2 - w[0] / 2)
        cz = rng.uniform(-sz / 2 + w[2] / 2, sz / 2 - w[2] / 2)
        if rng.uniform() < 0.2:  # some boxes hang on walls / float (shelves)
            cy = rng.uniform(-sy / 2 + w[1] / 2, floor - w[1] / 2)
        else:
            cy = floor - w[1] / 2
        blo = np.array([cx - w[0] / 2, cy - w[1] / 2, cz - w[2] / 2])
        bhi = np.array([cx + w[0] / 2, cy + w[1] / 2, cz + w[2] / 2])
        if keep_clear is not None and len(keep_clear):
            # horizontal distance from each clear point to the box footprint
            dx = np.maximum(0, np.maximum(blo[0] - keep_clear[:, 0], keep_clear[:, 0] - bhi[0]))
            dz = np.maximum(0, np.maximum(blo[2] - keep_clear[:, 2], keep_clear[:, 2] - bhi[2]))
            if np.min(np.hypot(dx, dz)) < clear_radius:
                continue
        lo.append(blo)
        hi.append(bhi)
        kind.append(1)
    tex = np.stack([_random_texture(rng) for _ in range(len(kind) * 6)]).reshape(len(kind), 6, TEX_STRIDE)
    return Scene(np.array(lo), np.array(hi), np.array(kind), tex)


def ring_corridor(rng, outer=(22.0, 2.8, 14.0), inner=(16.0, 8.0), n_boxes=(40, 80), keep_clear=None,
                  clear_radius=0.7):
    """Rectangular ring corridor: a room shell with a solid central block, boxes along the walls."""
    sx, sy, sz = outer
    ix, iz = inner
    lo = [[-sx / 2, -sy / 2, -sz / 2], [-ix / 2, -sy / 2 - 0.1, -iz / 2]]
    hi = [[sx / 2, sy / 2, sz / 2], [ix / 2, sy / 2 + 0.1, iz / 2]]
    kind = [0, 1]
    nb = int(rng.integers(n_boxes[0], n_boxes[1] + 1))
    floor = sy / 2
    tries = 0
    while len(kind) < nb + 2 and tries < 5000:
        tries += 1
        w = rng.uniform(0.2, 1.0, size=3)
        w[1] = rng.uniform(0.2, 1.6)
        cx = rng.uniform(-sx / 2 + w[0] / 2, sx / 2 - w[0] / 2)
        cz = rng.uniform(-sz / 2 + w[2] / 2, sz / 2 - w[2] / 2)
        cy = floor - w[1] / 2 if rng.uniform() > 0.2 else rng.uniform(-sy / 2 + w[1] / 2, floor - w[1] / 2)
        blo = np.array([cx - w[0] / 2, cy - w[1] / 2, cz - w[2] / 2])
        bhi = np.array([cx + w[0] / 2, cy + w[1] / 2, cz + w[2] / 2])
        # must lie in the corridor (not overlapping the central block)
        if blo[0] < ix / 2 and bhi[0] > -ix / 2 and blo[2] < iz / 2 and bhi[2] > -iz / 2:
            continue
        if keep_clear is not None and len(keep_clear):
            dx = np.maximum(0, np.maximum(blo[0] - keep_clear[:, 0], keep_clear[:, 0] - bhi[0]))
            dz = np.maximum(0, np.maximum(blo[2] - keep_clear[:, 2], keep_clear[:, 2] - bhi[2]))
            if np.min(np.hypot(dx, dz)) < clear_radius:
                continue
        lo.append(blo)
        hi.append(bhi)
        kind.append(1)
    tex = np.stack([_random_texture(rng) for _ in range(len(kind) * 6)]).reshape(len(kind), 6, TEX_STRIDE)
    return Scene(np.array(lo), np.array(hi), np.array(kind), tex)


def planar_scene(normal_axis=2, offset=3.0, rng=None):
    """A single large textured wall (a huge room shell seen from inside): depth of a plane."""
    rng = rng or np.random.default_rng(0)
    big = 50.0
    lo = np.array([[-big, -big, -big]])
    hi = np.array([[big, big, big]])
    hi[0, normal_axis] = offset
    tex = np.stack([_random_texture(rng) for _ in range(6)]).reshape(1, 6, TEX_STRIDE)
    return Scene(lo, hi, np.array([0]), tex)


# ----------------------------------------------------------------------------
# rendering
# ----------------------------------------------------------------------------

def render(scene: Scene, poses, intr):
    """Render depth (camera z, 0 = no surface) and luminance for camera->world poses (n,4,4)."""
    poses = np.asarray(poses, dtype=np.float64)
    n = poses.shape[0]
    W, H = intr["W"], intr["H"]
    P = np.zeros((n, 12))
    P[:, :9] = poses[:, :3, :3].reshape(n, 9)
    P[:, 9:] = poses[:, :3, 3]
    P = np.ascontiguousarray(P)
    depth = np.zeros((n, H, W), dtype=np.float32)
    lum = np.zeros((n, H, W), dtype=np.float32)
    _lib().synth_render(n, W, H, intr["fx"], intr["fy"], intr["cx"], intr["cy"],
                        P.ctypes.data, scene.n_boxes, scene.lo.ctypes.data, scene.hi.ctypes.data,
                        scene.kind.ctypes.data, scene.tex.ctypes.data, depth.ctypes.data, lum.ctypes.data)
    return depth, lum


def render_culled(scene: Scene, poses, intr, max_range=4.5):
    """render(), one frame at a time with only the boxes whose bounds come within max_range of the
    camera centre (plus the room shell): depths below max_range are the same as with every box,
    and the per-frame work no longer grows with the size of the scene."""
    poses = np.asarray(poses, dtype=np.float64)
    n = poses.shape[0]
    depth = np.zeros((n, intr["H"], intr["W"]), dtype=np.float32)
    lum = np.zeros((n, intr["H"], intr["W"]), dtype=np.float32)
    for k in range(n):
        c = poses[k, :3, 3]
        gap = np.maximum(0.0, np.maximum(scene.lo - c, c - scene.hi))
        near = (np.linalg.norm(gap, axis=1) < max_range) | (scene.kind == 0)
        sub = Scene(scene.lo[near], scene.hi[near], scene.kind[near], scene.tex[near])
        d, l = render(sub, poses[k:k + 1], intr)
        depth[k], lum[k] = d[0], l[0]
    return depth, lum


def sensor_depth(rng, depth_gt, sigma=0.002, dmin=0.5, dmax=4.0):
    """Clip to [dmin, dmax] (outside -> 0 = invalid) and add N(0, sigma^2) noise to valid pixels."""
    d = depth_gt.astype(np.float64)
    valid = (d >= dmin) & (d <= dmax)
    noise = rng.normal(0.0, sigma, size=d.shape)
    out = np.where(valid, d + noise, 0.0)
    return out.astype(np.float32), valid


# ----------------------------------------------------------------------------
# trajectories
# ----------------------------------------------------------------------------

def smooth_walk(rng, n, start, max_rot_deg=5.0, max_trans=0.05, scene=None, smooth=0.7,
                rot_scale_deg=2.5, trans_scale=0.03):
    """Smoothed random walk of camera->world poses; per-frame motion <= max_rot_deg, <= max_trans."""
    poses = [np.array(start, dtype=np.float64)]
    w = np.zeros(3)
    v = np.zeros(3)
    for _ in range(n - 1):
        for _attempt in range(50):
            w_new = smooth * w + (1 - smooth) * rng.normal(0, np.deg2rad(rot_scale_deg), 3)
            v_new = smooth * v + (1 - smooth) * rng.normal(0, trans_scale, 3)
            wn = np.linalg.norm(w_new)
            if wn > np.deg2rad(max_rot_deg):
                w_new *= np.deg2rad(max_rot_deg) / wn
            vn = np.linalg.norm(v_new)
            if vn > max_trans:
                v_new *= max_trans / vn
            T = poses[-1]
            R = T[:3, :3] @ rot_from_vec(w_new)  # rotate about the camera's own axes
            t = T[:3, 3] + T[:3, :3] @ v_new
            if scene is None or scene.free(t, margin=0.4):
                break
            w, v = -w, -v  # bounce
        w, v = w_new, v_new
        poses.append(make_pose(R, t))
    return np.stack(poses)


def ring_loop(n, outer=(22.0, 14.0), inner=(16.0, 8.0), look_out_deg=55.0, wobble=None):
    """Camera centres on the mid-line of a rectangular ring corridor, one closed loop.

    Each camera looks along the direction of travel, turned towards the outer wall by
    look_out_deg, with an optional small (yaw, pitch, roll) wobble array (n,3) in radians.
    """
    ax, az = (outer[0] + inner[0]) / 4.0, (outer[1] + inner[1]) / 4.0  # mid-line half extents
    corners = np.array([[-ax, -az], [ax, -az], [ax, az], [-ax, az], [-ax, -az]])
    seg = np.linalg.norm(np.diff(corners, axis=0), axis=1)
    L = seg.sum()
    s = np.linspace(0, L, n, endpoint=False)
    poses = []
    for k, sk in enumerate(s):
        i = np.searchsorted(np.cumsum(seg), sk, side="right")
        i = min(i, 3)
        s0 = sk - (np.cumsum(seg)[i - 1] if i > 0 else 0.0)
        d = (corners[i + 1] - corners[i]) / seg[i]
        p = corners[i] + d * s0
        # travel direction d (x,z); outward normal for a counter-clockwise loop in (x,z)
        yaw_travel = np.arctan2(d[0], d[1])  # yaw about +y mapping +z to (x,z)=d
        yaw = yaw_travel - np.deg2rad(look_out_deg)
        dy = dp = dr = 0.0
        if wobble is not None:
            dy, dp, dr = wobble[k]
        R = yaw_pitch_roll(yaw + dy, dp, dr)
        poses.append(make_pose(R, np.array([p[0], 0.0, p[1]])))
    return np.stack(poses), L


def drift(rng, poses, step_trans=0.01, step_rot_deg=0.3):
    """Initial estimate: GT with an accumulated random-walk error (first pose unchanged)."""
    out = [poses[0].copy()]
    E = np.eye(4)
    for k in range(1, len(poses)):
        dR = rot_from_vec(rng.normal(0, np.deg2rad(step_rot_deg) / np.sqrt(3), 3))
        dt = rng.normal(0, step_trans / np.sqrt(3), 3)
        E = E @ make_pose(dR, dt)
        out.append(poses[0] @ E @ (np.linalg.inv(poses[0]) @ poses[k]))
    return np.stack(out)


# ----------------------------------------------------------------------------
# correspondences and overlap
# ----------------------------------------------------------------------------

def _backproject(intr, xs, ys, z):
    return np.stack([(xs - intr["cx"]) * z / intr["fx"], (ys - intr["cy"]) * z / intr["fy"], z], axis=-1)


def _project(intr, p):
    z = p[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = intr["fx"] * p[..., 0] / z + intr["cx"]
        v = intr["fy"] * p[..., 1] / z + intr["cy"]
    return u, v, z


def visible_mask(intr, depth_gt_i, depth_gt_j, Ti, Tj, tol=0.05, stride=1, dmin=0.5, dmax=4.0):
    """For pixels of i (subsampled by stride): valid in i and landing on a GT-consistent valid pixel of j."""
    H, W = depth_gt_i.shape
    ys, xs = np.mgrid[0:H:stride, 0:W:stride]
    z = depth_gt_i[ys, xs].astype(np.float64)
    vi = (z >= dmin) & (z <= dmax)
    p = _backproject(intr, xs, ys, z)
    Tji = np.linalg.inv(Tj) @ Ti
    q = p @ Tji[:3, :3].T + Tji[:3, 3]
    u, v, zq = _project(intr, q)
    ok = vi & (zq > 0.1)
    ui = np.floor(np.where(ok, u, -10) + 0.5).astype(np.int64)
    vi_ = np.floor(np.where(ok, v, -10) + 0.5).astype(np.int64)
    ok &= (ui >= 0) & (ui < W) & (vi_ >= 0) & (vi_ < H)
    dj = np.where(ok, depth_gt_j[np.clip(vi_, 0, H - 1), np.clip(ui, 0, W - 1)], 0.0)
    ok &= (dj >= dmin) & (dj <= dmax) & (np.abs(dj - zq) < tol)
    return ok, vi, xs, ys


def overlap(intr, depth_gt, poses, i, j, stride=2):
    ok, vi, _, _ = visible_mask(intr, depth_gt[i], depth_gt[j], poses[i], poses[j], stride=stride)
    nv = vi.sum()
    return float(ok.sum()) / nv if nv else 0.0


def sample_correspondences(rng, intr, depth_gt, depth_noisy, poses, i, j, n, sigma=0.01, outlier_frac=0.05):
    """n correspondences of pair (i,j): p_i in camera i (noisy depth), p_j = T_j^-1 T_i p_i + N(0, sigma^2 I).

    A fraction outlier_frac of p_j is replaced by the back-projection of a random valid pixel of j.
    Returns (p_i, p_j, is_outlier) as float32 / bool arrays, or None if nothing of i is visible in j.
    """
    stride = 1 if intr["W"] < 160 else 2  # candidates from every second pixel on large frames
    ok, _, xs, ys = visible_mask(intr, depth_gt[i], depth_gt[j], poses[i], poses[j], stride=stride)
    ok &= depth_noisy[i][ys, xs] > 0
    cand = np.flatnonzero(ok.ravel())
    if len(cand) == 0:
        return None
    pick = cand[rng.integers(0, len(cand), size=n)]
    px, py = xs.ravel()[pick], ys.ravel()[pick]
    p_i = _backproject(intr, px.astype(np.float64), py.astype(np.float64), depth_noisy[i][py, px].astype(np.float64))
    Tji = np.linalg.inv(poses[j]) @ poses[i]
    p_j = p_i @ Tji[:3, :3].T + Tji[:3, 3] + rng.normal(0, sigma, size=(n, 3))
    out = rng.uniform(size=n) < outlier_frac
    if out.any():
        vj = np.flatnonzero(depth_noisy[j].ravel() > 0)
        r = vj[rng.integers(0, len(vj), size=int(out.sum()))]
        oy, ox = np.divmod(r, intr["W"])
        p_j[out] = _backproject(intr, ox.astype(np.float64), oy.astype(np.float64),
                                depth_noisy[j].ravel()[r].astype(np.float64))
    return p_i.astype(np.float32), p_j.astype(np.float32), out
