"""Residuals and Jacobians of the alignment energy (oracle, FP64, world frame).

Sec. 4.3 writes E_align = w_sparse E_sparse + w_dense (w_photo E_photo + w_geo E_geo).
Each scalar residual r depends on two poses, T_i and T_j; its Jacobian row is
returned as two 6-vectors (d/d(dw_i, dt_i), d/d(dw_j, dt_j)) under the left
update R <- Exp(dw) R, t <- t + dt (lie.py).

Sparse term (Sec. 4.3, "Sparse Matching"): r = T_i p_ik - T_j p_jl, three rows per
correspondence:  d/d dw_i = -[R_i p]_x,  d/d dt_i = I,  d/d dw_j = +[R_j q]_x,
d/d dt_j = -I.

Geometric term (Sec. 4.3, E_geo): point-to-plane n_ik^T (d_ik - T_i^-1 T_j q) with q the
back-projected target pixel, rewritten exactly in world coordinates as
r_g = n_w . (P - Q), n_w = R_i n, P = T_i d, Q = T_j q, the association held fixed:
  d/d dw_i = n_w x (P - Q) + (R_i d) x n_w,   d/d dt_i = n_w,
  d/d dw_j = n_w x (R_j q),                   d/d dt_j = -n_w.

Photometric term (Sec. 4.3, E_photo): r_p = I_i(k) - I_j(pi(y)), y = T_j^-1 T_i d, with
I the gradient magnitude of the luminance and I_j sampled bilinearly:
  d r_p / d theta = -grad I_j(u)^T Jpi(y) dy/d theta,
  Jpi = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]],
  dy/d dw_i = -R_j^T [R_i d]_x,  dy/d dt_i = R_j^T,
  dy/d dw_j =  R_j^T [P - t_j]_x, dy/d dt_j = -R_j^T.
"""
import numpy as np

from .lie import skew


# ---------------------------------------------------------------- sparse term

def sparse_residuals(Ri, ti, Rj, tj, p, q):
    """r (N,3) = (R_i p + t_i) - (R_j q + t_j)."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    return (p @ Ri.T + ti) - (q @ Rj.T + tj)


def sparse_jacobians(Ri, ti, Rj, tj, p, q):
    """Jacobians (N,3,6) w.r.t. frame i and frame j of the three residual rows."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    N = p.shape[0]
    A = p @ Ri.T
    B = q @ Rj.T
    Ji = np.zeros((N, 3, 6))
    Jj = np.zeros((N, 3, 6))
    for k in range(N):
        Ji[k, :, :3] = -skew(A[k])
        Ji[k, :, 3:] = np.eye(3)
        Jj[k, :, :3] = skew(B[k])
        Jj[k, :, 3:] = -np.eye(3)
    return Ji, Jj


# ----------------------------------------------------------------- dense term

def _bilinear(img, bx, by, ux, uy):
    wx = ux - bx
    wy = uy - by
    H, W = img.shape
    f = img.ravel()
    i00 = by * W + bx
    return ((1 - wx) * (1 - wy) * f[i00] + wx * (1 - wy) * f[i00 + 1]
            + (1 - wx) * wy * f[i00 + W] + wx * wy * f[i00 + W + 1])


def dense_terms(fi, fj, Ri, ti, Rj, tj, assoc):
    """Geometric and photometric residuals and Jacobians over the associated pixels.

    assoc: output of association.associate (held fixed).  Returns a dict with
    idx (source pixel indices), r_geo, J_geo_i, J_geo_j, r_photo, J_photo_i, J_photo_j.
    """
    W = fi.W
    idx = np.flatnonzero(assoc["valid"])
    ys, xs = np.divmod(idx, W)
    z = fi.D.ravel()[idx]
    d = np.stack([(xs - fi.cx) * z / fi.fx, (ys - fi.cy) * z / fi.fy, z], axis=-1)
    n = fi.N.reshape(-1, 3)[idx]
    Rd = d @ Ri.T
    P = Rd + ti
    y = (P - tj) @ Rj           # R_j^T (P - t_j), row-vector form
    nx, ny = assoc["nx"][idx], assoc["ny"][idx]
    bx, by = assoc["bx"][idx], assoc["by"][idx]
    Dj = fj.D.ravel()[ny * W + nx]
    q = np.stack([(nx - fj.cx) * Dj / fj.fx, (ny - fj.cy) * Dj / fj.fy, Dj], axis=-1)
    Rq = q @ Rj.T
    Q = Rq + tj
    # geometric: point-to-plane
    n_w = n @ Ri.T
    Delta = P - Q
    r_g = np.sum(n_w * Delta, axis=1)
    Jg_i = np.concatenate([np.cross(n_w, Delta) + np.cross(Rd, n_w), n_w], axis=1)
    Jg_j = np.concatenate([np.cross(n_w, Rq), -n_w], axis=1)
    # photometric: gradient-magnitude image sampled at u = pi(y)
    zz = y[:, 2]
    ux = fj.fx * y[:, 0] / zz + fj.cx
    uy = fj.fy * y[:, 1] / zz + fj.cy
    Ij = _bilinear(fj.I, bx, by, ux, uy)
    gx = _bilinear(fj.Ix, bx, by, ux, uy)
    gy = _bilinear(fj.Iy, bx, by, ux, uy)
    r_p = fi.I.ravel()[idx] - Ij
    # g = d r_p / d y = -grad I^T Jpi(y)
    g = -np.stack([gx * fj.fx / zz, gy * fj.fy / zz,
                   -(gx * fj.fx * y[:, 0] + gy * fj.fy * y[:, 1]) / (zz * zz)], axis=-1)
    # d y = R_j^T (dw_i x R_i d + dt_i) for frame i; R_j^T ((P - t_j) x dw_j - dt_j) for frame j
    h = g @ Rj.T                # world-frame vector R_j g: d r_p = h . (world displacement)
    Jp_i = np.concatenate([np.cross(Rd, h), h], axis=1)
    Jp_j = np.concatenate([np.cross(h, P - tj), -h], axis=1)
    return dict(idx=idx, r_geo=r_g, J_geo_i=Jg_i, J_geo_j=Jg_j, r_photo=r_p, J_photo_i=Jp_i, J_photo_j=Jp_j)


def dense_residuals_only(fi, fj, Ri, ti, Rj, tj, assoc):
    """(r_geo, r_photo) at the given poses with a frozen association (for finite differences)."""
    t = dense_terms(fi, fj, Ri, ti, Rj, tj, assoc)
    return t["r_geo"], t["r_photo"]
