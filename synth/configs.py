"""The workloads, as seeded synthetic problems.

Each builder returns a :class:`Problem`: frames (sensor depth with noise, luminance),
ground-truth camera->world poses, initial poses, and sparse correspondences per
unordered frame pair.  Shapes follow the paper's scans (Sec. 4.1: dense terms on
80x60 frames; Sec. 4.2: chunks of 11 frames; Sec. 7.3: roughly 150-250 features
per frame), rendered from box rooms since no dataset is available.

Seeds: master seed 1604; workload c uses seed 1604*100 + c.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

from . import scene as sc


@dataclasses.dataclass
class Problem:
    name: str
    intr: dict
    depth: np.ndarray          # (n,H,W) float32 sensor depth, 0 = invalid
    lum: np.ndarray            # (n,H,W) float32 luminance in [0,1]
    gt: np.ndarray             # (n,4,4) float64 camera->world
    init: np.ndarray           # (n,4,4) float64 initial camera->world
    pairs: np.ndarray          # (P,2) int32, i<j
    corr_off: np.ndarray       # (P+1,) int64 offsets into p_i/p_j
    p_i: np.ndarray            # (C,3) float32, camera coordinates of frame i
    p_j: np.ndarray            # (C,3) float32, camera coordinates of frame j
    outlier: np.ndarray        # (C,) bool (generator bookkeeping, not solver input)
    chunks: list | None = None  # list of int arrays (frame indices per chunk)
    solve: dict | None = None   # default solve parameters for this workload
    depth_gt: np.ndarray | None = None

    @property
    def n_frames(self):
        return self.depth.shape[0]

    @property
    def n_corr(self):
        return int(self.corr_off[-1])

    def pair_corr(self, k):
        a, b = self.corr_off[k], self.corr_off[k + 1]
        return self.p_i[a:b], self.p_j[a:b]


def seed_for(config_index: int) -> int:
    return 1604 * 100 + config_index


def _assemble(name, intr, depth, lum, gt, init, pair_list, corr, chunks=None, solve=None, depth_gt=None):
    pairs = np.array(pair_list, dtype=np.int32).reshape(-1, 2)
    counts = [len(c[0]) for c in corr]
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    if corr:
        p_i = np.concatenate([c[0] for c in corr]).astype(np.float32)
        p_j = np.concatenate([c[1] for c in corr]).astype(np.float32)
        out = np.concatenate([c[2] for c in corr])
    else:
        p_i = np.zeros((0, 3), np.float32)
        p_j = np.zeros((0, 3), np.float32)
        out = np.zeros(0, bool)
    return Problem(name, intr, depth, lum, gt, init, pairs, off, p_i, p_j, out, chunks, solve, depth_gt)


def _chunk_frames(rng, room, n, intr, start):
    gt = sc.smooth_walk(rng, n, start, scene=room)
    depth_gt, lum = sc.render(room, gt, intr)
    depth, _ = sc.sensor_depth(rng, depth_gt)
    return gt, depth_gt, depth, lum


def _chunk_start(rng, room_size):
    yaw = rng.uniform(-np.pi, np.pi)
    R = sc.yaw_pitch_roll(yaw, rng.uniform(-0.15, 0.15), rng.uniform(-0.05, 0.05))
    # back off from the wall we look at so that it sits ~2-3 m away
    fwd = R[:, 2]
    c = np.array([0.0, rng.uniform(-0.3, 0.3), 0.0]) - fwd * rng.uniform(0.3, 1.0)
    return sc.make_pose(R, c)


def chunk_problem(seed, n_frames=11, W=80, H=60, n_corr=(200, 200), sigma=0.01, outlier_frac=0.05,
                  room_size=(6.0, 2.8, 6.0), n_boxes=(20, 60), name="chunk"):
    """One chunk: consecutive frames on a smooth walk, every pair matched (Sec. 4.2)."""
    rng = np.random.default_rng(seed)
    intr = sc.intrinsics(W, H)
    start = _chunk_start(rng, room_size)
    room = sc.box_room(rng, room_size, n_boxes, keep_clear=start[None, :3, 3], clear_radius=1.0)
    gt, depth_gt, depth, lum = _chunk_frames(rng, room, n_frames, intr, start)
    pair_list, corr = [], []
    for i, j in itertools.combinations(range(n_frames), 2):
        n = int(rng.integers(n_corr[0], n_corr[1] + 1))
        c = sc.sample_correspondences(rng, intr, depth_gt, depth, gt, i, j, n, sigma, outlier_frac)
        if c is None:
            continue
        pair_list.append((i, j))
        corr.append(c)
    # local solve: poses relative to the chunk's first frame, initialised to identity
    rel = np.linalg.inv(gt[0]) @ gt
    init = np.tile(np.eye(4), (n_frames, 1, 1))
    return _assemble(name, intr, depth, lum, rel, init, pair_list, corr, depth_gt=depth_gt,
                     solve=dict(n_gn=4, n_pcg=10, w_sparse=1.0, w_dense=0.5, w_photo=0.1, w_geo=1.0))


def cfg1():
    """Single chunk: 11 frames at 80x60, all 55 pairs, 200 correspondences per pair, 4 GN x 10 PCG."""
    p = chunk_problem(seed_for(1), 11, 80, 60, (200, 200), 0.01, 0.05, name="chunk11_80x60")
    return p


def global_problem(seed, n_kf=300, W=80, H=60, n_corr=(64, 256), sigma=0.01, outlier_frac=0.05,
                   overlap_min=0.30, look_out_deg=90.0, outer=(24.0, 2.8, 16.0), inner=(14.0, 6.0),
                   name="global", max_pairs=None):
    """Keyframes along one loop of a ring corridor; pairs with GT overlap > overlap_min (Sec. 4.2)."""
    rng = np.random.default_rng(seed)
    intr = sc.intrinsics(W, H)
    wob = np.stack([rng.normal(0, 0.05, n_kf), rng.normal(0, 0.04, n_kf), rng.normal(0, 0.02, n_kf)], 1)
    gt, L = sc.ring_loop(n_kf, (outer[0], outer[2]), inner, look_out_deg, wob)
    gt[:, 1, 3] = rng.normal(0, 0.1, n_kf)
    centres = gt[:, :3, 3]
    room = sc.ring_corridor(rng, outer, inner, keep_clear=centres, clear_radius=0.5)
    depth_gt, lum = sc.render(room, gt, intr)
    depth, _ = sc.sensor_depth(rng, depth_gt)
    pair_list = []
    for i in range(n_kf):
        for j in range(i + 1, n_kf):
            if np.linalg.norm(centres[i] - centres[j]) > 5.0:
                continue
            if sc.overlap(intr, depth_gt, gt, i, j, stride=2) > overlap_min:
                pair_list.append((i, j))
    if max_pairs is not None and len(pair_list) > max_pairs:
        keep = np.sort(rng.choice(len(pair_list), max_pairs, replace=False))
        pair_list = [pair_list[k] for k in keep]
    corr, kept = [], []
    for (i, j) in pair_list:
        n = int(rng.integers(n_corr[0], n_corr[1] + 1))
        c = sc.sample_correspondences(rng, intr, depth_gt, depth, gt, i, j, n, sigma, outlier_frac)
        if c is None:
            continue
        kept.append((i, j))
        corr.append(c)
    init = sc.drift(rng, gt)
    return _assemble(name, intr, depth, lum, gt, init, kept, corr, depth_gt=depth_gt,
                     solve=dict(n_gn=8, n_pcg=20, w_sparse=1.0, w_dense=0.5, w_photo=0.1, w_geo=1.0))


def large_global_problem(seed, n_kf=2000, W=160, H=120, n_corr=(64, 136), sigma=0.01, outlier_frac=0.10,
                         overlap_min=0.30, max_pairs=25000, outer=(60.0, 2.8, 40.0), inner=(50.0, 30.0),
                         name="global2000_160x120"):
    """Large global solve: keyframes along one loop of a large ring corridor (about 180 m), cameras
    facing the outer wall; candidate pairs within 3 m, kept when their GT overlap exceeds
    overlap_min (stride-4 test), then subsampled to max_pairs; 10 % outliers."""
    rng = np.random.default_rng(seed)
    intr = sc.intrinsics(W, H)
    wob = np.stack([rng.normal(0, 0.05, n_kf), rng.normal(0, 0.04, n_kf), rng.normal(0, 0.02, n_kf)], 1)
    gt, L = sc.ring_loop(n_kf, (outer[0], outer[2]), inner, 90.0, wob)
    gt[:, 1, 3] = rng.normal(0, 0.1, n_kf)
    centres = gt[:, :3, 3]
    room = sc.ring_corridor(rng, outer, inner, n_boxes=(300, 400), keep_clear=centres, clear_radius=0.5)
    depth_gt, lum = sc.render_culled(room, gt, intr)
    depth, _ = sc.sensor_depth(rng, depth_gt)
    pair_list = []
    for i in range(n_kf):
        near = np.flatnonzero(np.linalg.norm(centres[i + 1:] - centres[i], axis=1) < 3.0) + i + 1
        for j in near:
            if sc.overlap(intr, depth_gt, gt, i, int(j), stride=4) > overlap_min:
                pair_list.append((i, int(j)))
    if len(pair_list) > max_pairs:
        keep = np.sort(rng.choice(len(pair_list), max_pairs, replace=False))
        pair_list = [pair_list[k] for k in keep]
    corr, kept = [], []
    for (i, j) in pair_list:
        n = int(rng.integers(n_corr[0], n_corr[1] + 1))
        c = sc.sample_correspondences(rng, intr, depth_gt, depth, gt, i, j, n, sigma, outlier_frac)
        if c is None:
            continue
        kept.append((i, j))
        corr.append(c)
    init = sc.drift(rng, gt)
    return _assemble(name, intr, depth, lum, gt, init, kept, corr, depth_gt=depth_gt,
                     solve=dict(n_gn=10, n_pcg=30, w_sparse=1.0, w_dense=0.5, w_photo=0.1, w_geo=1.0))


def cfg5():
    """Large global mixed-precision solve: 2000 keyframes at 160x120, ~25k pairs, ~2.5M
    correspondences with 10 % outliers, 10 GN x 30 PCG (BF16 frame storage in the benchmark)."""
    return large_global_problem(seed_for(5))


def cfg4_global():
    """The serving stream's global keyframe set: 2000 keyframes at 80x60 along one loop of the
    large ring corridor (pairs as in the large global workload, 64-256 correspondences per pair,
    5 % outliers), 8 GN x 20 PCG per solve.  A global request solves the first k keyframes, k
    growing from 100 to 2000 over a session."""
    p = large_global_problem(seed_for(4), 2000, 80, 60, n_corr=(64, 256), outlier_frac=0.05, name="global2000_80x60")
    p.solve = dict(n_gn=8, n_pcg=20, w_sparse=1.0, w_dense=0.5, w_photo=0.1, w_geo=1.0)
    return p


def cfg2():
    """Global solve: 300 keyframes at 80x60 along a ~60 m loop, overlap > 30 %, 8 GN x 20 PCG."""
    return global_problem(seed_for(2), 300, 80, 60, name="global300_80x60")


def chunk_batch(seed, n_chunks=256, W=320, H=240, length=(3, 11), n_corr=(100, 400), sigma=0.01,
                outlier_frac=0.05, name="chunks"):
    """Independent chunks of uneven length, each in its own room; frames concatenated."""
    rng = np.random.default_rng(seed)
    intr = sc.intrinsics(W, H)
    gts, depths, lums, chunks, pair_list, corr, dgts = [], [], [], [], [], [], []
    base = 0
    room_size = (6.0, 2.8, 6.0)
    for c in range(n_chunks):
        n = int(rng.integers(length[0], length[1] + 1))
        start = _chunk_start(rng, room_size)
        room = sc.box_room(rng, room_size, (20, 60), keep_clear=start[None, :3, 3], clear_radius=1.0)
        gt, depth_gt, depth, lum = _chunk_frames(rng, room, n, intr, start)
        for i, j in itertools.combinations(range(n), 2):
            k = int(rng.integers(n_corr[0], n_corr[1] + 1))
            cc = sc.sample_correspondences(rng, intr, depth_gt, depth, gt, i, j, k, sigma, outlier_frac)
            if cc is None:
                continue
            pair_list.append((base + i, base + j))
            corr.append(cc)
        gts.append(np.linalg.inv(gt[0]) @ gt)
        depths.append(depth)
        lums.append(lum)
        dgts.append(depth_gt)
        chunks.append(np.arange(base, base + n, dtype=np.int32))
        base += n
    gt = np.concatenate(gts)
    init = np.tile(np.eye(4), (base, 1, 1))
    return _assemble(name, intr, np.concatenate(depths), np.concatenate(lums), gt, init, pair_list, corr,
                     chunks=chunks, depth_gt=np.concatenate(dgts),
                     solve=dict(n_gn=6, n_pcg=10, w_sparse=1.0, w_dense=0.5, w_photo=0.1, w_geo=1.0))


def cfg3(n_chunks=256, W=320, H=240):
    """Batched chunk solves: 256 chunks of U{3..11} frames at 320x240, 100-400 corr./pair, 6 GN x 10 PCG."""
    return chunk_batch(seed_for(3), n_chunks, W, H, name=f"chunks{n_chunks}_{W}x{H}")
