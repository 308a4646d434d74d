"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties one part of the oracle to something other than itself: closed
forms, library routines, finite differences, invariants, brute force, or values
printed in the paper (tests/golden/paper_constants.json).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize
from scipy.spatial.transform import Rotation

import synth
from synth import scene as sc
from oracle import association, frames, keypoints, lie, residuals, solver, system, tsdf, verification
from oracle.system import SolveParams, SparsePair

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


# ------------------------------------------------------------------ helpers

def rand_pose(rng, rot_scale=0.3, trans_scale=0.5):
    R = Rotation.from_rotvec(rng.normal(0, rot_scale, 3)).as_matrix()
    return lie.to44(R, rng.normal(0, trans_scale, 3))


def consistent_corr(rng, Ti, Tj, n, sigma=0.0):
    """Points p in camera i and q = T_j^-1 T_i p (+ noise) in camera j, FP64."""
    p = rng.uniform([-1, -1, 1], [1, 1, 3], size=(n, 3))
    Tji = np.linalg.inv(Tj) @ Ti
    q = p @ Tji[:3, :3].T + Tji[:3, 3] + rng.normal(0, sigma, size=(n, 3)) if sigma else p @ Tji[:3, :3].T + Tji[:3, 3]
    return p, q


def render_pair(rng, intr, scene, poses, noise=0.0):
    depth_gt, lum = sc.render(scene, poses, intr)
    depth = np.where((depth_gt > 0.5) & (depth_gt < 4.0), depth_gt + (rng.normal(0, noise, depth_gt.shape) if noise else 0), 0)
    return depth.astype(np.float32), lum


@pytest.fixture(scope="module")
def room_frames():
    """Three noise-free 80x60 renderings of a box room from nearby poses (GT known)."""
    rng = np.random.default_rng(7)
    intr = sc.intrinsics(80, 60)
    start = lie.to44(sc.yaw_pitch_roll(0.3, 0.05, 0.0), np.array([0.0, 0.0, -0.5]))
    room = sc.box_room(rng, (6.0, 2.8, 6.0), (20, 30), keep_clear=start[None, :3, 3], clear_radius=1.0)
    poses = sc.smooth_walk(rng, 3, start, scene=room)
    depth, lum = render_pair(rng, intr, room, poses)
    fr = [frames.Frame(depth[k], lum[k], intr) for k in range(3)]
    return intr, poses, fr, depth, lum


# ------------------------------------------------------------- golden values

def test_golden_constants_match_defaults():
    g = json.load(open(GOLDEN))
    p = SolveParams()
    assert p.tau_dist == g["tau_d_m"]["value"]
    assert p.tau_normal == g["tau_n"]["value"]
    assert p.max_angle_deg == g["max_angle_deg"]["value"]
    assert synth.cfg1().n_frames == g["n_chunk"]["value"]


def test_fig11_variable_count():
    """Sec. 7 (Fig. 11): 101 keyframes give 600 variables, i.e. 6 per frame with the first fixed."""
    g = json.load(open(GOLDEN))
    n = g["fig11_keyframes"]["value"]
    S = system.System(n)
    assert S.A.shape == (g["fig11_variables"]["value"],) * 2
    assert 6 * (n - 1) == g["fig11_variables"]["value"]


# ------------------------------------------------------------------ lie.py

@pytest.mark.parametrize("scale", [1e-12, 1e-9, 1e-4, 0.3, 2.5])
def test_exp_matches_matrix_exponential(scale):
    rng = np.random.default_rng(1)
    for _ in range(5):
        w = rng.normal(size=3) * scale
        E = scipy.linalg.expm(np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]))
        np.testing.assert_allclose(lie.exp_so3(w), E, atol=1e-14, rtol=0)


def test_exp_is_rotation_and_skew_is_cross():
    rng = np.random.default_rng(2)
    w, u = rng.normal(size=3), rng.normal(size=3)
    R = lie.exp_so3(w)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1) < 1e-14
    np.testing.assert_allclose(lie.skew(w) @ u, np.cross(w, u), atol=1e-15)


# --------------------------------------------------------------- frames.py

def test_normals_of_a_plane_are_exact():
    """A noise-free plane: central-difference normals equal the plane normal, facing the camera."""
    intr = sc.intrinsics(80, 60)
    n_true = np.array([0.3, -0.2, -1.0])
    n_true /= np.linalg.norm(n_true)
    # plane n.X = -2.5 (camera at the origin on the side the normal points to)
    ys, xs = np.mgrid[0:60, 0:80].astype(np.float64)
    ray = np.stack([(xs - intr["cx"]) / intr["fx"], (ys - intr["cy"]) / intr["fy"], np.ones_like(xs)], -1)
    z = -2.5 / (ray @ n_true)
    f = frames.Frame(z, np.zeros((60, 80)), intr)
    assert f.nvalid[1:-1, 1:-1].all() and not f.nvalid[0].any() and not f.nvalid[:, -1].any()
    np.testing.assert_allclose(f.N[1:-1, 1:-1], np.broadcast_to(n_true, (58, 78, 3)), atol=1e-12)


def test_normal_invalid_next_to_invalid_depth():
    intr = sc.intrinsics(80, 60)
    D = np.full((60, 80), 2.0)
    D[30, 40] = 0.0
    f = frames.Frame(D, np.zeros((60, 80)), intr)
    for (y, x) in [(30, 40), (29, 40), (31, 40), (30, 39), (30, 41)]:
        assert not f.nvalid[y, x]
    assert f.nvalid[29, 39] and f.nvalid[32, 40]


def test_intensity_gradient_closed_forms():
    """L = c (x + y)^2: central differences are exact, |grad L| = 2 sqrt(2) c (x + y), grad I = 2 sqrt(2) c (1, 1)."""
    ys, xs = np.mgrid[0:60, 0:80].astype(np.float64)
    c = 1e-4
    I, Ix, Iy = frames.intensity_gradient(c * (xs + ys) ** 2)
    k = 2 * math.sqrt(2) * c
    np.testing.assert_allclose(I[1:-1, 1:-1], k * (xs + ys)[1:-1, 1:-1], rtol=1e-12)
    assert not I[0].any() and not I[:, 0].any()
    np.testing.assert_allclose(Ix[2:-2, 2:-2], k, rtol=1e-10)
    np.testing.assert_allclose(Iy[2:-2, 2:-2], k, rtol=1e-10)
    assert not Ix[1].any() and not Iy[:, 1].any()
    # a linear ramp has constant gradient magnitude and zero grad I
    I2, Ix2, Iy2 = frames.intensity_gradient(0.01 * xs - 0.02 * ys)
    np.testing.assert_allclose(I2[1:-1, 1:-1], math.hypot(0.01, 0.02), rtol=1e-12)
    assert np.abs(Ix2).max() < 1e-15 and np.abs(Iy2).max() < 1e-15


def test_depth_validity_range():
    D = np.array([[0.05, 0.1, 0.5, 9.99, 10.0, np.nan, np.inf]])
    np.testing.assert_array_equal(frames.valid_depth(D, 0.1, 10.0)[0], [False, False, True, True, False, False, False])


# ----------------------------------------------------------- sparse residuals

def test_sparse_zero_at_ground_truth():
    rng = np.random.default_rng(3)
    Ti, Tj = rand_pose(rng), rand_pose(rng)
    p, q = consistent_corr(rng, Ti, Tj, 50)
    r = residuals.sparse_residuals(Ti[:3, :3], Ti[:3, 3], Tj[:3, :3], Tj[:3, 3], p, q)
    assert np.abs(r).max() < 1e-14
    poses = np.stack([np.eye(4), np.linalg.inv(Ti) @ Tj])  # frame 0 = camera i as world
    S = system.assemble([None, None], None, poses, [SparsePair(0, 1, p, q)], [], SolveParams(dense_on=False), 0.0)
    assert S.e_sparse < 1e-26 and np.abs(S.b).max() < 1e-12


def fd_check(fun, poses, idx, J_analytic, h=1e-6):
    """Central differences of fun(poses) w.r.t. the 6 tangent coordinates of frame idx."""
    J = np.zeros((len(fun(poses)), 6))
    for c in range(6):
        e = np.zeros(6)
        e[c] = h
        Pp, Pm = poses.copy(), poses.copy()
        R, t = lie.apply_update(poses[idx][:3, :3], poses[idx][:3, 3], e)
        Pp[idx] = lie.to44(R, t)
        R, t = lie.apply_update(poses[idx][:3, :3], poses[idx][:3, 3], -e)
        Pm[idx] = lie.to44(R, t)
        J[:, c] = (fun(Pp) - fun(Pm)) / (2 * h)
    scale = np.abs(J_analytic).max()
    np.testing.assert_allclose(J, J_analytic, atol=2e-7 * scale, rtol=0)


def test_sparse_jacobian_finite_differences():
    rng = np.random.default_rng(4)
    poses = np.stack([rand_pose(rng), rand_pose(rng)])
    p = rng.normal(size=(20, 3))
    q = rng.normal(size=(20, 3))

    def f(P):
        return residuals.sparse_residuals(P[0][:3, :3], P[0][:3, 3], P[1][:3, :3], P[1][:3, 3], p, q).ravel()

    Ji, Jj = residuals.sparse_jacobians(poses[0][:3, :3], poses[0][:3, 3], poses[1][:3, :3], poses[1][:3, 3], p, q)
    fd_check(f, poses, 0, Ji.reshape(-1, 6))
    fd_check(f, poses, 1, Jj.reshape(-1, 6))


# ------------------------------------------------------------ dense residuals

def perturbed(poses, rng, rot=0.01, trans=0.01):
    out = poses.copy()
    for k in range(len(out)):
        R, t = lie.apply_update(out[k][:3, :3], out[k][:3, 3], np.r_[rng.normal(0, rot, 3), rng.normal(0, trans, 3)])
        out[k] = lie.to44(R, t)
    return out


def test_dense_geo_jacobian_finite_differences(room_frames):
    intr, poses, fr, _, _ = room_frames
    rng = np.random.default_rng(5)
    P0 = perturbed(poses, rng)
    M = association.relative_transform(P0[0][:3, :3], P0[0][:3, 3], P0[1][:3, :3], P0[1][:3, 3])
    asc = association.associate(fr[0], fr[1], M, intr)
    assert asc["valid"].sum() > 500
    d = residuals.dense_terms(fr[0], fr[1], P0[0][:3, :3], P0[0][:3, 3], P0[1][:3, :3], P0[1][:3, 3], asc)

    def f(P):
        return residuals.dense_residuals_only(fr[0], fr[1], P[0][:3, :3], P[0][:3, 3], P[1][:3, :3], P[1][:3, 3], asc)[0]

    fd_check(f, P0, 0, d["J_geo_i"])
    fd_check(f, P0, 1, d["J_geo_j"])


def test_dense_photo_jacobian_finite_differences(room_frames):
    """With L = c (x+y)^2 the intensity I is linear, so bilinear sampling and grad I are exact and
    finite differences of r_p must equal -grad I^T Jpi dy/dtheta."""
    intr, poses, fr, depth, _ = room_frames
    ys, xs = np.mgrid[0:60, 0:80].astype(np.float64)
    L = 1e-4 * (xs + ys) ** 2
    f0 = frames.Frame(depth[0], L, intr)
    f1 = frames.Frame(depth[1], L, intr)
    rng = np.random.default_rng(6)
    P0 = perturbed(poses, rng)
    M = association.relative_transform(P0[0][:3, :3], P0[0][:3, 3], P0[1][:3, :3], P0[1][:3, 3])
    asc = association.associate(f0, f1, M, intr)
    d = residuals.dense_terms(f0, f1, P0[0][:3, :3], P0[0][:3, 3], P0[1][:3, :3], P0[1][:3, 3], asc)

    def f(P):
        return residuals.dense_residuals_only(f0, f1, P[0][:3, :3], P[0][:3, 3], P[1][:3, :3], P[1][:3, 3], asc)[1]

    fd_check(f, P0, 0, d["J_photo_i"])
    fd_check(f, P0, 1, d["J_photo_j"])


def test_dense_duplicate_frame_zero_residual(room_frames):
    """Frame j = frame i at the identical pose: every associated pixel maps onto itself, r_g = r_p = 0."""
    intr, poses, fr, _, _ = room_frames
    P = np.stack([poses[1], poses[1]])
    M = association.relative_transform(P[0][:3, :3], P[0][:3, 3], P[1][:3, :3], P[1][:3, 3])
    asc = association.associate(fr[1], fr[1], M, intr)
    idx = np.flatnonzero(asc["valid"])
    ys, xs = np.divmod(idx, 80)
    np.testing.assert_array_equal(asc["nx"][idx], xs)
    np.testing.assert_array_equal(asc["ny"][idx], ys)
    d = residuals.dense_terms(fr[1], fr[1], P[0][:3, :3], P[0][:3, 3], P[1][:3, :3], P[1][:3, 3], asc)
    assert np.abs(d["r_geo"]).max() == 0.0
    assert np.abs(d["r_photo"]).max() < 1e-12
    # every pixel with valid depth + normal strictly inside the 3-pixel border is associated
    inner = fr[1].valid & fr[1].nvalid
    inner[:3] = inner[-3:] = False
    inner[:, :3] = inner[:, -3:] = False
    assert np.all(asc["valid"][inner.ravel()])


def test_dense_geo_vanishes_on_noise_free_surfaces_at_gt(room_frames):
    """Noise-free renderings at GT: point-to-plane residuals vanish except at rare edge pixels;
    a transposed relative transform or a sign error would break this."""
    intr, poses, fr, _, _ = room_frames
    M = association.relative_transform(poses[0][:3, :3], poses[0][:3, 3], poses[2][:3, :3], poses[2][:3, 3])
    asc = association.associate(fr[0], fr[2], M, intr)
    d = residuals.dense_terms(fr[0], fr[2], poses[0][:3, :3], poses[0][:3, 3], poses[2][:3, :3], poses[2][:3, 3], asc)
    assert len(d["r_geo"]) > 1500
    assert np.median(np.abs(d["r_geo"])) < 1e-5
    # shared mask: one photometric and one geometric residual per associated pixel (Sec. 4.4)
    assert len(d["r_geo"]) == len(d["r_photo"])
    M_bad = (M[0].T.copy(), M[1])
    asc_bad = association.associate(fr[0], fr[2], M_bad, intr)
    if asc_bad["valid"].sum() > 0:
        d_bad = residuals.dense_terms(fr[0], fr[2], poses[0][:3, :3], poses[0][:3, 3], poses[2][:3, :3],
                                      poses[2][:3, 3], asc_bad)
        assert asc_bad["valid"].sum() < 0.9 * asc["valid"].sum() or np.median(np.abs(d_bad["r_geo"])) > 1e-4


def test_plane_geo_residual_zero_for_any_pair():
    """A textured plane rendered noise-free from two poses: r_g = 0 at GT for every associated pixel."""
    rng = np.random.default_rng(8)
    intr = sc.intrinsics(80, 60)
    scene = sc.planar_scene(2, 3.0, rng)
    poses = np.stack([lie.to44(np.eye(3), np.zeros(3)),
                      lie.to44(Rotation.from_rotvec([0.02, -0.05, 0.01]).as_matrix(), np.array([0.1, -0.05, 0.2]))])
    depth, lum = render_pair(rng, intr, scene, poses)
    fr = [frames.Frame(depth[k], lum[k], intr) for k in range(2)]
    M = association.relative_transform(poses[0][:3, :3], poses[0][:3, 3], poses[1][:3, :3], poses[1][:3, 3])
    asc = association.associate(fr[0], fr[1], M, intr)
    d = residuals.dense_terms(fr[0], fr[1], poses[0][:3, :3], poses[0][:3, 3], poses[1][:3, :3], poses[1][:3, 3], asc)
    assert len(d["r_geo"]) > 3000
    assert np.abs(d["r_geo"]).max() < 2e-6  # float32 depth storage only


# -------------------------------------------------------------- the system

def stacked_residuals(fr, intr, poses, sparse_pairs, dense_assoc, params, wd):
    """Weighted residual vector sqrt(w) r with frozen dense associations (test-side stacking)."""
    out = []
    for sp in sparse_pairs:
        r = residuals.sparse_residuals(poses[sp.a][:3, :3], poses[sp.a][:3, 3], poses[sp.b][:3, :3],
                                       poses[sp.b][:3, 3], sp.p, sp.q)
        out.append(math.sqrt(params.w_sparse) * r.ravel())
    for (i, j), asc in dense_assoc.items():
        rg, rp = residuals.dense_residuals_only(fr[i], fr[j], poses[i][:3, :3], poses[i][:3, 3],
                                                poses[j][:3, :3], poses[j][:3, 3], asc)
        out.append(math.sqrt(wd * params.w_geo) * rg)
        out.append(math.sqrt(wd * params.w_photo) * rp)
    return np.concatenate(out)


def test_normal_equations_equal_fd_jacobian_products(room_frames):
    """A = J^T W J and b = -J^T W r with J from finite differences of the whole stacked
    residual vector (gauge frame excluded): pins block placement, weights and gauge."""
    intr, poses, fr, _, _ = room_frames
    rng = np.random.default_rng(9)
    P0 = perturbed(poses, rng, 0.005, 0.005)
    sp = []
    for (a, b) in [(0, 1), (0, 2), (1, 2)]:
        p, q = consistent_corr(rng, poses[a], poses[b], 30, sigma=0.01)
        sp.append(SparsePair(a, b, p, q))
    params = SolveParams(w_sparse=1.3, w_geo=0.8, w_photo=0.0)
    wd = 0.7
    dense_pairs = [(0, 1), (1, 2)]
    S = system.assemble(fr, intr, P0, sp, dense_pairs, params, wd)
    assoc = {}
    for (a, b) in dense_pairs:
        for (i, j) in ((a, b), (b, a)):
            M = association.relative_transform(P0[i][:3, :3], P0[i][:3, 3], P0[j][:3, :3], P0[j][:3, 3])
            assoc[(i, j)] = association.associate(fr[i], fr[j], M, intr)
    f = lambda P: stacked_residuals(fr, intr, P, sp, assoc, params, wd)  # noqa: E731
    r0 = f(P0)
    J = np.zeros((len(r0), 12))
    h = 1e-6
    for fidx in (1, 2):
        for c in range(6):
            e = np.zeros(6)
            e[c] = h
            Pp, Pm = P0.copy(), P0.copy()
            Pp[fidx] = lie.to44(*lie.apply_update(P0[fidx][:3, :3], P0[fidx][:3, 3], e))
            Pm[fidx] = lie.to44(*lie.apply_update(P0[fidx][:3, :3], P0[fidx][:3, 3], -e))
            J[:, 6 * (fidx - 1) + c] = (f(Pp) - f(Pm)) / (2 * h)
    A_fd = J.T @ J
    b_fd = -J.T @ r0
    np.testing.assert_allclose(S.A, A_fd, atol=1e-6 * np.abs(A_fd).max(), rtol=0)
    np.testing.assert_allclose(S.b, b_fd, atol=1e-6 * np.abs(b_fd).max(), rtol=0)
    assert abs(S.energy - r0 @ r0) < 1e-10 * (r0 @ r0)
    # residual count identity (Sec. 4.4): 3 per correspondence, 2 per associated pixel
    n_px = sum(a["valid"].sum() for a in assoc.values())
    assert S.n_sparse == 3 * sum(s.p.shape[0] for s in sp)
    assert len(r0) == S.n_sparse + 2 * n_px


def test_gauge_invariance_of_energy(room_frames):
    intr, poses, fr, _, _ = room_frames
    rng = np.random.default_rng(10)
    P0 = perturbed(poses, rng)
    sp = [SparsePair(0, 1, *consistent_corr(rng, poses[0], poses[1], 40, 0.01))]
    params = SolveParams()
    S = system.assemble(fr, intr, P0, sp, [(0, 1), (1, 2), (0, 2)], params, 0.5)
    G = rand_pose(rng, 0.5, 1.0)
    S2 = system.assemble(fr, intr, np.einsum("ab,kbc->kac", G, P0), sp, [(0, 1), (1, 2), (0, 2)], params, 0.5)
    assert S.n_dense == S2.n_dense
    assert abs(S.energy - S2.energy) < 1e-10 * S.energy


def sparse_problem(rng, n, n_corr=40, sigma=0.01, spread=0.3):
    gt = np.stack([np.eye(4)] + [rand_pose(rng, spread, spread) for _ in range(n - 1)])
    sp = []
    for a in range(n):
        for b in range(a + 1, n):
            p, q = consistent_corr(rng, gt[a], gt[b], n_corr, sigma)
            sp.append(SparsePair(a, b, p, q))
    return gt, sp


def test_gn_iterates_are_gauge_covariant():
    """Solving from G X0 gives G X_k for every Gauss-Newton iterate (block-Jacobi PCG)."""
    rng = np.random.default_rng(11)
    gt, sp = sparse_problem(rng, 4)
    X0 = perturbed(gt, rng, 0.05, 0.05)
    params = SolveParams(n_gn=3, n_pcg=5, dense_on=False)
    r1 = solver.gauss_newton([None] * 4, None, X0, sp, params)
    G = rand_pose(rng, 0.7, 2.0)
    r2 = solver.gauss_newton([None] * 4, None, np.einsum("ab,kbc->kac", G, X0), sp, params)
    for Pa, Pb in zip(r1.pose_history, r2.pose_history):
        np.testing.assert_allclose(np.einsum("ab,kbc->kac", G, Pa), Pb, atol=1e-10)
    np.testing.assert_allclose(r1.energy, r2.energy, rtol=1e-10)


def kabsch(P, Q):
    """Textbook Kabsch/Umeyama: R, t minimising sum ||P - (R Q + t)||^2."""
    mp, mq = P.mean(0), Q.mean(0)
    H = (Q - mq).T @ (P - mp)
    U, _, Vt = np.linalg.svd(H)
    D = np.diag([1, 1, np.sign(np.linalg.det(Vt.T @ U.T))])
    R = Vt.T @ D @ U.T
    return R, mp - R @ mq


def test_two_frame_sparse_converges_to_kabsch():
    """Sec. 4.1.1 cites Kabsch: with frame 0 fixed, the sparse-only optimum is the Kabsch fit."""
    rng = np.random.default_rng(12)
    gt, sp = sparse_problem(rng, 2, n_corr=100, sigma=0.02, spread=0.4)
    sp[0].q[:5] += rng.normal(0, 0.5, (5, 3))  # outliers: still the L2 optimum
    params = SolveParams(n_gn=12, n_pcg=6, dense_on=False)
    res = solver.gauss_newton([None] * 2, None, np.stack([np.eye(4)] * 2), sp, params)
    R, t = kabsch(sp[0].p, sp[0].q)
    np.testing.assert_allclose(res.poses[1][:3, :3], R, atol=1e-10)
    np.testing.assert_allclose(res.poses[1][:3, 3], t, atol=1e-10)


def test_noise_free_recovers_ground_truth():
    rng = np.random.default_rng(13)
    for n in (2, 3):
        gt, sp = sparse_problem(rng, n, sigma=0.0, spread=0.25)
        res = solver.gauss_newton([None] * n, None, np.stack([np.eye(4)] * n), sp,
                                  SolveParams(n_gn=10, n_pcg=6 * (n - 1), dense_on=False))
        for k in range(n):
            rot, tr = lie.pose_error(res.poses[k], gt[k])
            assert rot < 1e-9 and tr < 1e-9


def test_three_frame_noisy_matches_independent_least_squares():
    """Brute force: scipy least_squares with a rotation-vector parameterisation and numeric
    Jacobian reaches the same minimum as the oracle's Gauss-Newton."""
    rng = np.random.default_rng(14)
    gt, sp = sparse_problem(rng, 3, sigma=0.02, spread=0.2)

    def fun(x):
        T = [np.eye(4)]
        for k in range(2):
            T.append(lie.to44(Rotation.from_rotvec(x[6 * k:6 * k + 3]).as_matrix(), x[6 * k + 3:6 * k + 6]))
        out = []
        for s in sp:
            out.append(((s.p @ T[s.a][:3, :3].T + T[s.a][:3, 3]) - (s.q @ T[s.b][:3, :3].T + T[s.b][:3, 3])).ravel())
        return np.concatenate(out)

    best = None
    for trial in range(3):
        x0 = rng.normal(0, 0.1, 12)
        r = scipy.optimize.least_squares(fun, x0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15)
        if best is None or r.cost < best.cost:
            best = r
    res = solver.gauss_newton([None] * 3, None, np.stack([np.eye(4)] * 3), sp,
                              SolveParams(n_gn=15, n_pcg=12, dense_on=False))
    assert abs(res.energy[-1] - 2 * best.cost) < 1e-9 * res.energy[-1]
    for k in range(2):
        Rk = Rotation.from_rotvec(best.x[6 * k:6 * k + 3]).as_matrix()
        np.testing.assert_allclose(res.poses[k + 1][:3, :3], Rk, atol=1e-7)
        np.testing.assert_allclose(res.poses[k + 1][:3, 3], best.x[6 * k + 3:6 * k + 6], atol=1e-7)


# --------------------------------------------------------------------- PCG

@pytest.mark.parametrize("kind", ["block", "jacobi"])
def test_pcg_equals_direct_solve_after_n_iterations(kind):
    rng = np.random.default_rng(15)
    gt, sp = sparse_problem(rng, 5, sigma=0.01)
    S = system.assemble([None] * 5, None, perturbed(gt, rng), sp, [], SolveParams(dense_on=False), 0.0)
    Minv, flags = solver.block_jacobi_inverse(S.A, kind)
    assert all(f == "ok" for f in flags)
    x, it = solver.pcg(S.A, S.b, Minv, 6 * 4 * 3)
    xd = np.linalg.solve(S.A, S.b)
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-8 * np.abs(xd).max())


def test_block_jacobi_is_exact_inverse_of_diagonal_blocks():
    rng = np.random.default_rng(16)
    B = rng.normal(size=(12, 12))
    A = B @ B.T + 12 * np.eye(12)
    Minv, _ = solver.block_jacobi_inverse(A)
    for k in range(2):
        s = slice(6 * k, 6 * k + 6)
        np.testing.assert_allclose(Minv[s, s] @ A[s, s], np.eye(6), atol=1e-12)
    assert not Minv[:6, 6:].any()


def test_empty_block_stays_zero():
    """A frame with no constraints (Sec. 4.4.1: implicitly removed) gets a zero update."""
    rng = np.random.default_rng(17)
    gt, sp = sparse_problem(rng, 3, sigma=0.01)
    sp = [s for s in sp if 2 not in (s.a, s.b)]
    S = system.assemble([None] * 3, None, perturbed(gt, rng), sp, [], SolveParams(dense_on=False), 0.0)
    Minv, flags = solver.block_jacobi_inverse(S.A)
    assert flags == ["ok", "empty"]
    x, _ = solver.pcg(S.A, S.b, Minv, 10)
    assert not x[6:].any()


def test_dense_pair_angle_gate():
    """Sec. 4.3: dense pairs need camera angles within 60 degrees."""
    R59 = Rotation.from_rotvec([0, np.deg2rad(59.0), 0]).as_matrix()
    R61 = Rotation.from_rotvec([0, np.deg2rad(61.0), 0]).as_matrix()
    P = np.stack([np.eye(4), lie.to44(R59, np.zeros(3)), lie.to44(R61, np.zeros(3))])
    sp = [SparsePair(0, 1, np.zeros((3, 3)), np.zeros((3, 3))), SparsePair(0, 2, np.zeros((3, 3)), np.zeros((3, 3)))]
    assert system.dense_pair_set(P, sp, 60.0) == [(0, 1)]


def test_r_max_finds_the_worst_pair():
    rng = np.random.default_rng(18)
    gt, sp = sparse_problem(rng, 3, sigma=0.0)
    sp[2].q[7] += np.array([0.0, 0.3, 0.4])
    val, pair = solver.r_max(gt, sp)
    assert pair == (sp[2].a, sp[2].b)
    # the moved point is now 0.5 m away in camera b coordinates -> 0.5 m in world
    assert abs(val - 0.5) < 1e-12



# ------------------------------------------------------------------ Sec. 4.4.1 pruning
def false_loop_problem(rng, n=4, bad=(1, 3), offset=(0.0, 0.25, 0.2)):
    """Noise-free correspondences on every pair except `bad`, whose points in frame b are all
    shifted by one rigid offset (a false loop closure consistent with a wrong transform)."""
    gt, sp = sparse_problem(rng, n, sigma=0.0)
    for k, p in enumerate(sp):
        if (p.a, p.b) == bad:
            sp[k] = SparsePair(p.a, p.b, p.p, p.q + np.array(offset))
    return gt, sp


def test_pruning_removes_the_false_pair_and_equals_the_clean_solve():
    rng = np.random.default_rng(41)
    gt, sp = false_loop_problem(rng)
    X0 = perturbed(gt, rng, 0.02, 0.03)
    prm = SolveParams(n_gn=6, n_pcg=30, dense_on=False)
    first = solver.gauss_newton([None] * 4, None, X0, sp, prm)
    assert first.r_max > 0.05 and first.r_max_pair == (1, 3)
    out = solver.gauss_newton_pruned([None] * 4, None, X0, sp, prm, prune_rmax=0.05)
    assert out.pruned == [(1, 3)] and out.rounds == 2 and out.invalid == []
    clean = solver.gauss_newton([None] * 4, None, X0, [p for p in sp if (p.a, p.b) != (1, 3)], prm)
    np.testing.assert_array_equal(out.result.poses, clean.poses)  # re-solve restarts from X0
    assert out.result.r_max < 1e-6
    P = out.result.poses
    for k in range(4):  # noise-free remaining pairs: the ground truth up to the gauge (frame 0 fixed)
        np.testing.assert_allclose(np.linalg.inv(P[0]) @ P[k], np.linalg.inv(gt[0]) @ gt[k], atol=1e-8)


def test_pruning_marks_a_frame_without_pairs_invalid():
    """Frame 3 is tied to the others only through the false pair: once it is pruned the frame
    has no constraint left, is reported invalid and keeps its initial pose."""
    rng = np.random.default_rng(42)
    gt, sp = sparse_problem(rng, 4, sigma=0.0)
    sp = [p for p in sp if p.b != 3 or p.a == 2]
    k = next(i for i, p in enumerate(sp) if (p.a, p.b) == (2, 3))
    q = sp[k].q.copy()
    q[::2] += np.array([0.0, 0.3, 0.0])  # half the matches wrong: no rigid motion explains the pair
    sp[k] = SparsePair(2, 3, sp[k].p, q)
    X0 = perturbed(gt, rng, 0.02, 0.03)
    prm = SolveParams(n_gn=6, n_pcg=30, dense_on=False)
    out = solver.gauss_newton_pruned([None] * 4, None, X0, sp, prm, prune_rmax=0.05)
    assert out.pruned == [(2, 3)] and out.invalid == [3]
    np.testing.assert_array_equal(out.result.poses[3], X0[3])


def test_no_pruning_below_the_threshold():
    rng = np.random.default_rng(43)
    gt, sp = false_loop_problem(rng)
    X0 = perturbed(gt, rng, 0.02, 0.03)
    prm = SolveParams(n_gn=4, n_pcg=20, dense_on=False)
    plain = solver.gauss_newton([None] * 4, None, X0, sp, prm)
    out = solver.gauss_newton_pruned([None] * 4, None, X0, sp, prm, prune_rmax=plain.r_max + 1.0)
    assert out.pruned == [] and out.rounds == 1
    np.testing.assert_array_equal(out.result.poses, plain.poses)
    capped = solver.gauss_newton_pruned([None] * 4, None, X0, sp, prm, prune_rmax=1e-300, max_rounds=2)
    assert len(capped.pruned) == 2 and capped.rounds == 3


# ------------------------------------------------------------- Sec. 4.1.1 dense verification
def test_verification_of_a_frame_with_itself(room_frames):
    """Identity transform, the same frame on both sides: every pixel with valid depth and normal
    re-projects onto itself with distance exactly 0, in both directions."""
    intr, poses, fr, depth, lum = room_frames
    chk = verification.verify_pair(fr[0], fr[0], np.eye(4), intr)
    n_valid = int((fr[0].valid & fr[0].nvalid).sum())
    assert chk.n_ij == chk.n_ji == n_valid and chk.e_ij == 0.0 and chk.e_ji == 0.0
    assert verification.pair_valid(chk, intr)


def test_verification_gates(room_frames):
    """Each gate alone rejects everything when violated by construction."""
    intr, poses, fr, depth, lum = room_frames
    n_valid = int((fr[0].valid & fr[0].nvalid).sum())
    brighter = frames.Frame(depth[0], lum[0] + 0.2, intr)  # tau_c = 0.1
    assert verification.verify_pair(fr[0], brighter, np.eye(4), intr).n_ij == 0
    slightly = frames.Frame(depth[0], lum[0] + 0.05, intr)
    assert verification.verify_pair(fr[0], slightly, np.eye(4), intr).n_ij == n_valid
    deeper = frames.Frame(depth[0] + np.float32(0.2), lum[0], intr)  # 0.2 m along z: > tau_d = 0.15
    chk = verification.verify_pair(fr[0], deeper, np.eye(4), intr)
    assert chk.n_ij == 0 and chk.n_ji == 0
    assert verification.verify_pair(fr[0], fr[0], np.eye(4), intr, tau_n=1.01).n_ij == 0
    assert not verification.pair_valid(chk, intr)


def small_room_pair(seed=51, W=32, H=24):
    rng = np.random.default_rng(seed)
    intr = sc.intrinsics(W, H)
    start = lie.to44(sc.yaw_pitch_roll(0.2, 0.05, 0.0), np.array([0.0, 0.0, -0.5]))
    room = sc.box_room(rng, (6.0, 2.8, 6.0), (20, 30), keep_clear=start[None, :3, 3], clear_radius=1.0)
    poses = sc.smooth_walk(rng, 2, start, scene=room)
    depth, lum = render_pair(rng, intr, room, poses)
    return intr, poses, [frames.Frame(depth[k], lum[k], intr) for k in range(2)]


def test_verification_matches_a_per_pixel_loop():
    """Brute force on a small frame: a pure-Python loop over pixels (the Sec. 4.1.1 gates written
    out per pixel with Python floats) gives the same count and error sum as the vectorised oracle."""
    intr, poses, (fi, fj) = small_room_pair()
    T = np.linalg.inv(poses[1]) @ poses[0]
    n, e, _, _, _, _ = verification.reproject(fi, fj, T, intr)
    W, H = intr["W"], intr["H"]
    fx, fy, cx, cy = intr["fx"], intr["fy"], intr["cx"], intr["cy"]
    cnt, tot = 0, 0.0
    for y in range(H):
        for x in range(W):
            if not (fi.valid[y, x] and fi.nvalid[y, x]):
                continue
            z = float(fi.D[y, x])
            d = [(x - cx) * z / fx, (y - cy) * z / fy, z]
            Y = [sum(T[a, b] * d[b] for b in range(3)) + T[a, 3] for a in range(3)]
            if not Y[2] > 0:
                continue
            tx, ty = math.floor(fx * Y[0] / Y[2] + cx + 0.5), math.floor(fy * Y[1] / Y[2] + cy + 0.5)
            if not (0 <= tx < W and 0 <= ty < H) or not (fj.valid[ty, tx] and fj.nvalid[ty, tx]):
                continue
            zq = float(fj.D[ty, tx])
            q = [(tx - cx) * zq / fx, (ty - cy) * zq / fy, zq]
            dist = math.sqrt(sum((Y[a] - q[a]) ** 2 for a in range(3)))
            m = [sum(T[a, b] * fi.N[y, x, b] for b in range(3)) for a in range(3)]
            if not (dist < 0.15 and sum(m[a] * fj.N[ty, tx, a] for a in range(3)) > 0.9
                    and abs(fi.C[y, x] - fj.C[ty, tx]) < 0.1):
                continue
            cnt += 1
            tot += dist
    assert cnt > 100 and n == cnt
    assert abs(e - tot) <= 1e-12 * tot


def test_association_matches_a_per_pixel_loop():
    """Brute force on a small frame pair: a pure-Python loop over pixels (Sec. 4.3 dense matching
    written out per pixel with Python floats) takes the same decisions as the vectorised oracle."""
    intr, poses, (fi, fj) = small_room_pair(52, 40, 30)
    rng = np.random.default_rng(3)
    P = perturbed(poses, rng, 0.01, 0.02)
    M = association.relative_transform(P[0][:3, :3], P[0][:3, 3], P[1][:3, :3], P[1][:3, 3])
    asc = association.associate(fi, fj, M, intr)
    R, t = M
    W, H = intr["W"], intr["H"]
    fx, fy, cx, cy = intr["fx"], intr["fy"], intr["cx"], intr["cy"]
    n_valid = 0
    for y in range(H):
        for x in range(W):
            k = y * W + x
            keep = False
            if fi.valid[y, x] and fi.nvalid[y, x]:
                z = float(fi.D[y, x])
                d = [(x - cx) * z / fx, (y - cy) * z / fy, z]
                Y = [sum(R[a, b] * d[b] for b in range(3)) + t[a] for a in range(3)]
                if Y[2] > 0:
                    ux, uy = fx * Y[0] / Y[2] + cx, fy * Y[1] / Y[2] + cy
                    tx, ty = math.floor(ux + 0.5), math.floor(uy + 0.5)
                    bx, by = math.floor(ux), math.floor(uy)
                    if 3 <= tx <= W - 4 and 3 <= ty <= H - 4 and fj.valid[ty, tx] and fj.nvalid[ty, tx]:
                        assert 2 <= bx and bx + 1 <= W - 3 and 2 <= by and by + 1 <= H - 3
                        zq = float(fj.D[ty, tx])
                        q = [(tx - cx) * zq / fx, (ty - cy) * zq / fy, zq]
                        dist = math.sqrt(sum((Y[a] - q[a]) ** 2 for a in range(3)))
                        m = [sum(R[a, b] * fi.N[y, x, b] for b in range(3)) for a in range(3)]
                        keep = dist < 0.15 and sum(m[a] * fj.N[ty, tx, a] for a in range(3)) > 0.9
                        if keep:
                            assert (asc["nx"][k], asc["ny"][k], asc["bx"][k], asc["by"][k]) == (tx, ty, bx, by)
            assert bool(asc["valid"][k]) == keep, (x, y)
            n_valid += keep
    assert n_valid > 200


def fronto_parallel_pair(shift_x, shift_y, W=40, H=30, Z=2.0):
    """Two frames of the plane z = Z facing the camera; camera i sits at the origin, camera j is
    moved so that every point of i projects to u = (x + shift_x, y + shift_y) in j.  I_i = 0 and
    I_j(x, y) = x^2 + 0.5 y^2 (a quadratic: bilinear interpolation from the right four taps has a
    closed form, extrapolation from wrong ones does not)."""
    intr = sc.intrinsics(W, H)
    D = np.full((H, W), Z)
    fi = frames.Frame(D, np.zeros((H, W)), intr)
    fj = frames.Frame(D, np.zeros((H, W)), intr)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    fi.I = np.zeros((H, W))
    fj.I = xs ** 2 + 0.5 * ys ** 2
    # camera j at -shift * Z / f along x, y: a point X of camera i is X + (shift_x Z / fx, shift_y Z / fy, 0) in j
    Tj = lie.to44(np.eye(3), np.array([-shift_x * Z / intr["fx"], -shift_y * Z / intr["fy"], 0.0]))
    return intr, fi, fj, np.eye(4), Tj


@pytest.mark.parametrize("shift", [(0.7, 0.25), (0.3, 0.6), (-0.6, -0.35)])
def test_bilinear_taps_nearest_pixel_and_interior_closed_form(shift):
    """Sec. 4.3 dense matching on a fronto-parallel plane with a known sub-pixel shift u = x + s:
    the nearest target is floor(u + 1/2), the bilinear base tap floor(u), a pixel is kept exactly
    when its nearest pixel lies on the 3-pixel interior (so that the four taps lie on the 2-pixel
    one), and the photometric residual equals minus the closed-form bilinear interpolation of I_j;
    r_g = 0."""
    sx, sy = shift
    intr, fi, fj, Ti, Tj = fronto_parallel_pair(sx, sy)
    W, H = intr["W"], intr["H"]
    M = association.relative_transform(Ti[:3, :3], Ti[:3, 3], Tj[:3, :3], Tj[:3, 3])
    asc = association.associate(fi, fj, M, intr)
    ys, xs = np.divmod(np.arange(W * H), W)
    ux, uy = xs + sx, ys + sy
    np.testing.assert_allclose(asc["ux"][fi.nvalid.ravel()], ux[fi.nvalid.ravel()], atol=1e-12)
    bx, by = np.floor(ux), np.floor(uy)
    nx, ny = np.floor(ux + 0.5), np.floor(uy + 0.5)
    expect = fi.nvalid.ravel() & (nx >= 3) & (nx <= W - 4) & (ny >= 3) & (ny <= H - 4)
    np.testing.assert_array_equal(asc["valid"], expect)
    assert (bx[expect] >= 2).all() and (bx[expect] + 1 <= W - 3).all() and (by[expect] >= 2).all()
    v = asc["valid"]
    np.testing.assert_array_equal(asc["nx"][v], np.floor(ux + 0.5)[v])
    np.testing.assert_array_equal(asc["ny"][v], np.floor(uy + 0.5)[v])
    np.testing.assert_array_equal(asc["bx"][v], bx[v])
    d = residuals.dense_terms(fi, fj, Ti[:3, :3], Ti[:3, 3], Tj[:3, :3], Tj[:3, 3], asc)
    wx, wy = ux - bx, uy - by
    # linear interpolation of x^2 between bx and bx + 1: bx^2 + wx (2 bx + 1); same for 0.5 y^2
    closed = (bx ** 2 + wx * (2 * bx + 1)) + 0.5 * (by ** 2 + wy * (2 * by + 1))
    np.testing.assert_allclose(d["r_photo"], -closed[v], rtol=0, atol=1e-9)
    # the true quadratic differs from the interpolation, so a wrong tap choice cannot pass above
    assert np.abs((ux ** 2 + 0.5 * uy ** 2)[v] - closed[v]).min() > 0.01
    assert np.abs(d["r_geo"]).max() < 1e-12


def test_hierarchy_composes_a_closed_form_chain():
    """Sec. 4.2: chunks of 11 frames overlapping by one; local poses relative to the chunk's first
    frame (its keyframe).  On a trajectory of known rigid motions, each keyframe's world pose is the
    previous keyframe's composed with the local pose of the previous chunk's last frame (the shared
    frame), and every member's world pose is its keyframe's composed with its local pose."""
    from oracle import hierarchy

    def world(f):  # closed form: a screw motion, rotation 0.05 f about z then 0.02 f about x
        c, s = math.cos(0.05 * f), math.sin(0.05 * f)
        Rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
        c2, s2 = math.cos(0.02 * f), math.sin(0.02 * f)
        Rx = np.array([[1.0, 0.0, 0.0], [0.0, c2, -s2], [0.0, s2, c2]])
        return lie.to44(Rz @ Rx, np.array([0.1 * f, 0.5 * math.sin(0.3 * f), 0.02 * f * f]))

    def inv(T):
        return lie.to44(T[:3, :3].T, -T[:3, :3].T @ T[:3, 3])

    chunks = [list(range(10 * c, 10 * c + 11)) for c in range(4)]  # 0..10, 10..20, ...: one shared frame
    kf_world = world(0)
    for c, ids in enumerate(chunks):
        np.testing.assert_allclose(kf_world, world(ids[0]), atol=1e-12)
        local = {f: inv(world(ids[0])) @ world(f) for f in ids}
        np.testing.assert_allclose(local[ids[0]], np.eye(4), atol=1e-15)
        for f in ids:
            np.testing.assert_allclose(hierarchy.compose(kf_world, local[f]), world(f), atol=1e-12)
        kf_world = hierarchy.keyframe_init(kf_world, local[ids[-1]])
    # the composition order matters: local @ keyframe is a different pose on this trajectory
    assert np.abs(local[ids[-1]] @ world(ids[0]) - world(ids[-1])).max() > 1e-2


def test_checked_replay_accepts_ties_and_rejects_other_disagreements(room_frames):
    """The replay used by the GPU parity tests: another implementation's decisions are accepted
    where they differ from the oracle's only on ties, and rejected anywhere else."""
    intr, poses, fr, _, _ = room_frames
    W, H = intr["W"], intr["H"]
    rng = np.random.default_rng(12)
    P0 = perturbed(poses, rng)
    M = association.relative_transform(P0[0][:3, :3], P0[0][:3, 3], P0[1][:3, :3], P0[1][:3, 3])
    own = association.associate(fr[0], fr[1], M, intr)
    ref = association.targets(own, W)
    same = association.CheckedReplay(lambda i, j, p: ref, W, H)
    rep = same(0, 1, P0, own)
    np.testing.assert_array_equal(association.targets(rep, W), ref)
    np.testing.assert_array_equal(rep["bx"][rep["valid"]], own["bx"][own["valid"]])
    assert same.n_flips == 0 and same.n_valid == int((ref >= 0).sum())
    # flip one tie (widened bounds make the pixel with the smallest margin a tie) and one non-tie
    k_tie = int(np.argmin(np.where(own["valid"], own["margin_px"], np.inf)))
    flipped = ref.copy()
    flipped[k_tie] = -1
    eps = (own["margin_px"][k_tie] * 1.01, association.EPS_D, association.EPS_N)
    ok = association.CheckedReplay(lambda i, j, p: flipped, W, H, eps)
    assert association.targets(ok(0, 1, P0, own), W)[k_tie] == -1 and ok.n_flips == 1
    k_far = int(np.argmax(np.where(own["valid"], own["margin_px"], -1.0)))
    flipped[k_far] = -1
    with pytest.raises(AssertionError):
        association.CheckedReplay(lambda i, j, p: flipped, W, H, eps)(0, 1, P0, own)
    # a replayed system equals the oracle's own when the decisions are the same
    sp = [SparsePair(0, 1, *consistent_corr(rng, poses[0], poses[1], 20, 0.01))]
    prm = SolveParams()
    S = system.assemble(fr, intr, P0, sp, [(0, 1)], prm, 0.5)
    fetch = association.CheckedReplay(
        lambda i, j, p: association.targets(association.associate(
            fr[i], fr[j], association.relative_transform(p[i][:3, :3], p[i][:3, 3], p[j][:3, :3], p[j][:3, 3]),
            intr), W), W, H)
    S2 = system.assemble(fr, intr, P0, sp, [(0, 1)], prm, 0.5, assoc=fetch)
    np.testing.assert_array_equal(S.A, S2.A)
    assert S.energy == S2.energy and fetch.calls == 2
    # the same on a process pool: the workers check and replay, the sums stay in pair order
    with system.frame_pool(fr, 2) as pool:
        S3 = system.assemble([None] * len(fr), intr, P0, sp, [(0, 1)], prm, 0.5, assoc=fetch,
                             pmap=lambda f, tasks: pool.map(f, tasks))
        np.testing.assert_array_equal(S.A, S3.A)
        np.testing.assert_array_equal(S.b, S3.b)
        assert S.energy == S3.energy and fetch.calls == 4
        bad = association.CheckedReplay(lambda i, j, p: np.full(W * H, -1), W, H)
        with pytest.raises(AssertionError):
            system.assemble([None] * len(fr), intr, P0, sp, [(0, 1)], prm, 0.5, assoc=bad,
                            pmap=lambda f, tasks: pool.map(f, tasks))


def test_chunk_validation_flags_a_misaligned_frame(room_frames):
    """At the ground-truth poses every pair is consistent (mean error below 0.05 m); moving one
    frame's pose by 0.2 m makes its pairs fail and the chunk invalid.  (The tau_d gate keeps only
    correspondences closer than 0.15 m, so the mean error of a misaligned pair grows slowly: at
    0.1 m it is still below the 0.05 m threshold.)"""
    intr, poses, fr, depth, lum = room_frames
    local = np.einsum("ab,kbc->kac", np.linalg.inv(poses[0]), poses)
    ok, worst, arg, checks = verification.validate_chunk(fr, local, intr)
    assert ok and worst < 0.03  # nearest-pixel sampling at 80x60 leaves about 2 cm
    bad = local.copy()
    bad[2][:3, 3] += np.array([0.2, 0.0, 0.0])
    ok2, worst2, arg2, _ = verification.validate_chunk(fr, bad, intr)
    assert not ok2 and worst2 > 0.05 and 2 in arg2


# ------------------------------------------------------- Sec. 4.1.1 key-point filters
def spread_points(rng, n, scale=(1.0, 0.8, 0.5), centre=(0.0, 0.0, 2.0)):
    return rng.uniform(-1, 1, (n, 3)) * np.array(scale) + np.array(centre)


def test_kabsch_matches_an_independent_wahba_solver():
    """scipy's Rotation.align_vectors (Wahba's problem, a different algorithm) on the centred
    point sets gives the same rotation."""
    rng = np.random.default_rng(61)
    P = spread_points(rng, 40)
    R0 = Rotation.from_rotvec([0.2, -0.4, 0.3]).as_matrix()
    Q = P @ R0.T + np.array([0.3, -0.1, 0.5]) + rng.normal(0, 0.01, (40, 3))
    R, t = keypoints.kabsch(P, Q)
    Ra, _ = Rotation.align_vectors(Q - Q.mean(0), P - P.mean(0))
    np.testing.assert_allclose(R, Ra.as_matrix(), atol=1e-12)
    np.testing.assert_allclose(t, Q.mean(0) - R @ P.mean(0), atol=1e-12)


def test_keypoint_filter_drops_exactly_the_outliers():
    rng = np.random.default_rng(62)
    P = spread_points(rng, 30)
    R0 = Rotation.from_rotvec([0.1, 0.3, -0.2]).as_matrix()
    t0 = np.array([0.2, 0.0, -0.3])
    Q = P @ R0.T + t0
    bad = [4, 11, 12, 25]
    Q[bad] += rng.normal(0, 0.3, (len(bad), 3))  # gross mismatches, anywhere in the match order
    out = keypoints.filter_pair(P, Q)
    assert out.status == 0 and sorted(out.keep) == [k for k in range(30) if k not in bad]
    np.testing.assert_allclose(out.R, R0, atol=1e-10)
    np.testing.assert_allclose(out.t, t0, atol=1e-10)


def test_keypoint_filter_residual_threshold():
    """One correspondence off by 5 cm is removed, one off by 1 cm stays (its residual under the
    refit is below the 2 cm threshold)."""
    rng = np.random.default_rng(63)
    P = spread_points(rng, 20)
    Q = P.copy()
    Q[7] += np.array([0.05, 0.0, 0.0])
    assert 7 not in keypoints.filter_pair(P, Q).keep
    Q = P.copy()
    Q[7] += np.array([0.01, 0.0, 0.0])
    assert 7 in keypoints.filter_pair(P, Q).keep


def test_keypoint_filter_rejects_collinear_and_too_few():
    rng = np.random.default_rng(64)
    s = rng.uniform(-1, 1, 20)
    P = np.stack([s, 2 * s, 0.5 * s + 2], axis=1) + rng.normal(0, 1e-4, (20, 3))  # nearly a line
    assert keypoints.filter_pair(P, P + 0.1).status == 1
    P4 = spread_points(rng, 4)
    assert keypoints.filter_pair(P4, P4).status == 1  # fewer than N_min = 5


def test_surface_area_of_a_rectangle():
    """Points filling a 0.3 x 0.2 m rectangle (any rigid placement): area 0.06 m^2; 0.1 x 0.2: 0.02."""
    rng = np.random.default_rng(65)
    for a, b in ((0.3, 0.2), (0.1, 0.2)):
        grid = np.array([[x, y, 0.0] for x in np.linspace(0, a, 7) for y in np.linspace(0, b, 5)])
        R = Rotation.from_rotvec(rng.normal(size=3)).as_matrix()
        X = grid @ R.T + rng.normal(size=3)
        assert abs(keypoints.surface_area(X) - a * b) < 1e-12
    grid = np.array([[x, y, 0.0] for x in np.linspace(0, 0.1, 7) for y in np.linspace(0, 0.2, 5)]) + [0, 0, 2.0]
    assert keypoints.filter_pair(grid, grid).status == 2
    big = grid * np.array([3.0, 1.0, 1.0])
    assert keypoints.filter_pair(big, big).status == 0


# ------------------------------------------------------------- Sec. 5 TSDF integration
def plane_depth(intr, Z):
    return np.full((intr["H"], intr["W"]), Z, dtype=np.float32)


def test_tsdf_plane_closed_form():
    """A fronto-parallel plane at depth Z seen from the identity pose: every touched voxel in
    front of it within the truncation band holds Z - z, further in front mu, and nothing behind
    Z + mu is touched."""
    intr = sc.intrinsics(80, 60)
    prm = tsdf.Params()
    Z = 1.3
    vol = tsdf.integrate({}, plane_depth(intr, Z), np.full((60, 80), 0.25, np.float32), intr, np.eye(4), prm)
    assert len(vol) > 50
    mu = float(prm.mu)
    n_band = 0
    for key, blk in vol.items():
        D, Wt = tsdf.tsdf_value(blk)
        z = (8 * key[2] + np.arange(512) // 64 + 0.5) * 0.004
        hit = Wt > 0
        assert np.all(z[hit] <= Z + mu + 1e-6)  # nothing behind the band
        near = hit & (np.abs(Z - z) < mu - 1e-5)
        np.testing.assert_allclose(D[near], Z - z[near], atol=2e-6)
        np.testing.assert_allclose(D[hit & (Z - z > mu + 1e-5)], mu, atol=1e-6)
        assert np.all(blk[2][hit] == round(0.25 * 65535))  # one sample: the quantised intensity
        n_band += near.sum()
    assert n_band > 1000


def test_tsdf_running_average_and_exact_inverse():
    """Two planes (Z1, Z2) give the paper's running average D = (d1 + d2) / 2 with W = 2;
    removing one with the inverse update leaves exactly the other; the order of integration
    does not matter and integrate + de-integrate restores every sum to zero."""
    intr = sc.intrinsics(80, 60)
    prm = tsdf.Params()
    c = np.full((60, 80), 0.5, np.float32)
    d1, d2 = plane_depth(intr, 1.30), plane_depth(intr, 1.31)
    both = tsdf.integrate(tsdf.integrate({}, d1, c, intr, np.eye(4), prm), d2, c, intr, np.eye(4), prm)
    rev = tsdf.integrate(tsdf.integrate({}, d2, c, intr, np.eye(4), prm), d1, c, intr, np.eye(4), prm)
    assert both.keys() == rev.keys() and all(np.array_equal(both[k], rev[k]) for k in both)
    one = tsdf.integrate({}, d1, c, intr, np.eye(4), prm)
    for k, blk in both.items():
        D, Wt = tsdf.tsdf_value(blk)
        z = (8 * k[2] + np.arange(512) // 64 + 0.5) * 0.004
        two = Wt == 2
        sdf = lambda Z: np.minimum(Z - z, float(prm.mu))
        np.testing.assert_allclose(D[two], 0.5 * (sdf(1.30) + sdf(1.31))[two], atol=2e-6)
    back = tsdf.integrate({k: v.copy() for k, v in both.items()}, d2, c, intr, np.eye(4), prm, sign=-1)
    for k, blk in back.items():
        np.testing.assert_array_equal(blk, one.get(k, np.zeros((3, 512), np.int64)))
    zero = tsdf.integrate(back, d1, c, intr, np.eye(4), prm, sign=-1)
    assert all(not blk.any() for blk in zero.values())


def test_tsdf_pose_moves_the_surface():
    """Integrating the plane from a camera moved by +0.1 m along z at a pose that says so puts
    the same world surface in the same voxels as the original view."""
    intr = sc.intrinsics(80, 60)
    prm = tsdf.Params()
    c = np.full((60, 80), 0.5, np.float32)
    T = np.eye(4)
    T[2, 3] = 0.1  # camera 0.1 m further along +z: the plane at 1.3 is at depth 1.2
    a = tsdf.integrate({}, plane_depth(intr, 1.3), c, intr, np.eye(4), prm)
    b = tsdf.integrate({}, plane_depth(intr, 1.2), c, intr, T, prm)
    common = set(a) & set(b)
    assert len(common) > 20
    for k in common:
        Da, Wa = tsdf.tsdf_value(a[k])
        Db, Wb = tsdf.tsdf_value(b[k])
        both = (Wa > 0) & (Wb > 0)
        np.testing.assert_allclose(Da[both], Db[both], atol=1e-5)


def test_euler_angles_and_pose_distance():
    rng = np.random.default_rng(66)
    for _ in range(5):
        al, be, ga = rng.uniform(-1, 1, 3)
        R = Rotation.from_euler("ZYX", [ga, be, al]).as_matrix()  # Rz(ga) Ry(be) Rx(al)
        np.testing.assert_allclose(tsdf.euler(R), [al, be, ga], atol=1e-12)
    Ta, Tb = np.eye(4), np.eye(4)
    Tb[:3, :3] = Rotation.from_euler("ZYX", [0.0, 0.0, 0.1]).as_matrix()
    Tb[:3, 3] = [0.3, 0.0, 0.4]
    assert abs(tsdf.pose_distance(Ta, Tb) - math.sqrt(0.2 ** 2 + 0.3 ** 2 + 0.4 ** 2)) < 1e-12
    integ = {5: Ta, 7: Ta, 9: Ta}
    opt = {5: Tb, 7: Ta, 9: Tb}
    assert tsdf.reintegration_order(integ, opt, n_fix=10) == [5, 9]
    assert tsdf.reintegration_order(integ, opt, n_fix=1) == [5]

# ------------------------------------------------------------------ 16-bit frame storage
def _fp16_grid_values(rng, n):
    """FP64 values around FP16 numbers: exact grid points, midpoints (ties), near-midpoints,
    subnormals and values past the largest finite one."""
    bits = rng.integers(0, 0x7C00, size=n, dtype=np.uint16)  # finite, non-negative halves
    h = bits.view(np.float16).astype(np.float64)
    nxt = (bits + 1).view(np.float16).astype(np.float64)
    mid = 0.5 * (h + nxt)
    eps = np.abs(mid) * 2.0 ** -30
    x = np.concatenate([h, mid, mid + eps, mid - eps, rng.uniform(-70000, 70000, n)])
    return np.concatenate([x, -x])


def test_fp16_rounding_matches_ieee_half_conversion():
    """round_to_storage('fp16') is IEEE round-to-nearest-even: NumPy's double -> half cast."""
    x = _fp16_grid_values(np.random.default_rng(5), 4000)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    got = frames.round_to_storage(x, "fp16")
    np.testing.assert_array_equal(got, ref)


def test_bf16_rounding_is_nearest_with_ties_to_even():
    """Brute force: among the numbers with 8 significant bits around x, the result is a nearest
    one, and on a tie the one with an even last bit."""
    rng = np.random.default_rng(6)
    x = np.concatenate([rng.normal(size=3000) * 10.0 ** rng.integers(-30, 30, 3000),
                        1.0 + np.array([2.0 ** -8, 3 * 2.0 ** -8, 2.0 ** -9, 5 * 2.0 ** -9])])
    got = frames.round_to_storage(x, "bf16")
    for v, q in zip(x, got):
        e = math.frexp(v)[1]
        quantum = 2.0 ** (e - 8)
        k0 = math.floor(v / quantum)
        cands = [k * quantum for k in (k0 - 1, k0, k0 + 1, k0 + 2)]
        dist = [abs(c - v) for c in cands]
        best = min(dist)
        near = [k for k, dd in zip((k0 - 1, k0, k0 + 1, k0 + 2), dist) if dd == best]
        k = near[0] if len(near) == 1 else [k for k in near if k % 2 == 0][0]
        assert q == k * quantum, (v, q, k * quantum)
    # the closed-form ties above
    assert list(got[-4:]) == [1.0, 1.0 + 2.0 ** -6, 1.0, 1.0 + 2.0 ** -7]


def test_storage_rounding_of_a_frame():
    """16-bit storage rounds normals, I and grad I only; depth and validity are untouched, and
    every stored value is representable in the format (rounding it again changes nothing)."""
    prob = synth.cfg1()
    intr = prob.intr
    f64 = frames.Frame(prob.depth[0], prob.lum[0], intr)
    for kind in ("bf16", "fp16"):
        f = frames.Frame(prob.depth[0], prob.lum[0], intr, storage=kind)
        np.testing.assert_array_equal(f.D, f64.D)
        np.testing.assert_array_equal(f.nvalid, f64.nvalid)
        for a, b in ((f.N, f64.N), (f.I, f64.I), (f.Ix, f64.Ix), (f.Iy, f64.Iy)):
            np.testing.assert_array_equal(frames.round_to_storage(a, kind), a)
            bits = 8 if kind == "bf16" else 11
            np.testing.assert_array_less(np.abs(a - b), np.abs(b) * 2.0 ** -bits + 2.0 ** -24 + 1e-300)
        assert np.any(f.N != f64.N)
    f32 = frames.Frame(prob.depth[0], prob.lum[0], intr, storage="fp32")
    np.testing.assert_array_equal(f32.N, f64.N)


def test_global300_golden_is_the_oracles_output():
    """tests/golden/global300_oracle.json (the full-size reference of the GPU tests) is what the
    oracle computes today on the seeded workload: regenerate the first Gauss-Newton step and compare
    its energies and iterate X_1."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "global300_oracle.json")
    with open(path) as f:
        gold = json.load(f)
    prob = synth.cfg2()
    d = prob.solve
    fr = [frames.Frame(prob.depth[k], prob.lum[k], prob.intr) for k in range(prob.n_frames)]
    prm = SolveParams(n_gn=1, n_pcg=d["n_pcg"], w_sparse=d["w_sparse"], w_dense=d["w_dense"], w_photo=d["w_photo"],
                      w_geo=d["w_geo"])
    res = solver.gauss_newton(fr, prob.intr, prob.init, solver.sparse_pairs_for(prob, range(prob.n_frames)), prm)
    np.testing.assert_allclose(res.energy[0], gold["energy"][0], rtol=1e-12)
    np.testing.assert_allclose(np.stack([P[:3, :].ravel() for P in res.poses]), np.array(gold["iterates"]["1"]),
                               rtol=0, atol=1e-12)


# ------------------------------------------------------------- planted mistakes
class _CrossSwapped:
    """Stand-in for numpy inside residuals.py whose cross product takes its operands the wrong way
    round (everything else is numpy's)."""

    def __getattr__(self, name):
        return getattr(np, name)

    @staticmethod
    def cross(a, b, *args, **kw):
        return np.cross(b, a, *args, **kw)


def test_planted_mistakes_fail_the_pins(monkeypatch, room_frames):
    """Four plausible mistakes planted in the oracle, one at a time: each makes a pin fail."""
    # 1. wrong cross-product order in the residual Jacobians
    with monkeypatch.context() as m:
        m.setattr(residuals, "np", _CrossSwapped())
        with pytest.raises(AssertionError):
            test_dense_geo_jacobian_finite_differences(room_frames)
    # 2. a dropped Jacobian term: the photometric residual's dependence on frame j's rotation
    orig_terms = residuals.dense_terms

    def dropped(*a, **kw):
        d = orig_terms(*a, **kw)
        d["J_photo_j"][:, :3] = 0.0
        return d

    with monkeypatch.context() as m:
        m.setattr(residuals, "dense_terms", dropped)
        with pytest.raises(AssertionError):
            test_dense_photo_jacobian_finite_differences(room_frames)
    # 3. a transposed rotation in the pair transform (R_i^T R_j instead of R_j^T R_i)
    orig_rel = association.relative_transform

    def transposed(Ri, ti, Rj, tj):
        R, t = orig_rel(Ri, ti, Rj, tj)
        return R.T, t

    with monkeypatch.context() as m:
        m.setattr(association, "relative_transform", transposed)
        with pytest.raises(AssertionError):
            test_plane_geo_residual_zero_for_any_pair()
    # 4. a corrupted gradient magnitude (|gx| + |gy| instead of the Euclidean norm)
    orig_grad = frames.intensity_gradient

    def l1(L):
        I, Ix, Iy = orig_grad(L)
        L = np.asarray(L, dtype=np.float64)
        gx = 0.5 * (L[1:-1, 2:] - L[1:-1, :-2])
        gy = 0.5 * (L[2:, 1:-1] - L[:-2, 1:-1])
        I = I.copy()
        I[1:-1, 1:-1] = np.abs(gx) + np.abs(gy)
        return I, Ix, Iy

    with monkeypatch.context() as m:
        m.setattr(frames, "intensity_gradient", l1)
        with pytest.raises(AssertionError):
            test_intensity_gradient_closed_forms()
