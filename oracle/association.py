"""Dense projective association for a directed frame pair i -> j (oracle).

Sec. 4.3 (dense matching) maps the 3D point d_ik of source pixel k into frame j
through T_j^-1 T_i, projects it with pi, reads D_j there, ignores projections
outside the frame, and prunes ICP-style by distance and normal after each step.
Readings used (the paper gives no numbers for this pruning):

* the association is recomputed once per Gauss-Newton iteration at the current
  poses and held fixed inside the linearisation (projective, "ICP-like");
* target pixel = nearest pixel (floor(u + 0.5) per axis), inside the image, with
  valid depth and a valid normal;
* the photometric term samples I_j and grad I_j bilinearly at u; all 4 taps must
  lie on the 2-pixel interior where grad I is defined;
* gates ||T_i d - T_j q|| < tau_d and (R_i n_i).(R_j n_j) > tau_n with the dense
  verification constants of Sec. 4.1.1 (tau_d = 0.15 m, tau_n = 0.9);
* the photometric and geometric residuals share one validity mask;
* the source pixel needs valid depth and a valid normal.

Every one of these decisions turns a floating-point value into an integer or a
boolean.  They are taken in IEEE FP32 in the fixed order written below: products, sums and
fused multiply-adds (one rounding of a*b + c, see fma32), and one correctly rounded
reciprocal 1/y_z for the projection; the same precision and order as the GPU kernel, so that
both sides take identical decisions on identical inputs.  The residual values themselves
(residuals.py) are FP64.

Per directed pair the relative transform M = T_j^-1 T_i is formed in FP64 with
explicit sums (R = R_j^T R_i, t = R_j^T (t_i - t_j)) and rounded once to FP32.
"""
import numpy as np

f32 = np.float32


def fma32(a, b, c):
    """IEEE FP32 fused multiply-add: a*b + c rounded once to nearest (ties to even).

    a, b, c are FP32.  In FP64 the product p = a*b is exact (24 + 24 significant bits);
    TwoSum gives p + c = s + e exactly with s = fl64(p + c).  Rounding s + e to FP64 "to odd"
    (s itself if e == 0 or s's last significand bit is odd, else the FP64 neighbour of s in
    the direction of e) and then to FP32 to nearest is the correctly rounded FP32 result,
    because FP64 carries at least two bits more than FP32 (Boldo and Melquiond, "Emulation of
    FMA and correctly rounded sums: proved algorithms using rounding to odd", IEEE TC 2008).
    """
    a64 = np.asarray(a, dtype=f32).astype(np.float64)
    b64 = np.asarray(b, dtype=f32).astype(np.float64)
    c64 = np.asarray(c, dtype=f32).astype(np.float64)
    p = a64 * b64
    s = p + c64
    bb = s - p
    e = (p - (s - bb)) + (c64 - bb)
    even = (np.asarray(s).view(np.int64) & 1) == 0
    with np.errstate(invalid="ignore"):
        toward = np.where(e > 0, np.inf, -np.inf)
        s_odd = np.where((e != 0) & even & np.isfinite(s), np.nextafter(s, toward), s)
    return s_odd.astype(f32)


def pair_transform32(Ri, ti, Rj, tj):
    """FP32 rounding of T_j^-1 T_i, each FP64 entry summed left to right."""
    R = np.zeros((3, 3))
    t = np.zeros(3)
    dt = [ti[0] - tj[0], ti[1] - tj[1], ti[2] - tj[2]]
    for a in range(3):
        for b in range(3):
            R[a, b] = (Rj[0, a] * Ri[0, b] + Rj[1, a] * Ri[1, b]) + Rj[2, a] * Ri[2, b]
        t[a] = (Rj[0, a] * dt[0] + Rj[1, a] * dt[1]) + Rj[2, a] * dt[2]
    return R.astype(f32), t.astype(f32)


def ray_tables(intr):
    """kx[x] = fl32((x - cx)/fx), ky[y] = fl32((y - cy)/fy), each computed in FP64 and rounded once."""
    W, H = intr["W"], intr["H"]
    kx = ((np.arange(W, dtype=np.float64) - intr["cx"]) / intr["fx"]).astype(f32)
    ky = ((np.arange(H, dtype=np.float64) - intr["cy"]) / intr["fy"]).astype(f32)
    return kx, ky


def associate(fi, fj, M32, intr, tau_d=0.15, tau_n=0.9):
    """Association of every source pixel of frame i into frame j.

    Returns a dict of flat arrays over the source pixels (row-major):
      valid (bool), nx, ny (nearest target pixel), bx, by (bilinear base tap).
    """
    R, t = M32
    W, H = intr["W"], intr["H"]
    kx, ky = ray_tables(intr)
    fx, fy, cx, cy = f32(intr["fx"]), f32(intr["fy"]), f32(intr["cx"]), f32(intr["cy"])
    ys, xs = np.divmod(np.arange(W * H), W)
    z = fi.D32.ravel()
    n_i = fi.N32.reshape(-1, 3)
    ok = fi.valid.ravel() & fi.nvalid.ravel()
    # camera-space source point (rounded products), then y = R d + t as fused multiply-adds
    # accumulated from t: y_a = fma(R_a2, d_z, fma(R_a1, d_y, fma(R_a0, d_x, t_a)))
    dx = kx[xs] * z
    dy = ky[ys] * z
    dz = z
    Y = [fma32(R[a, 2], dz, fma32(R[a, 1], dy, fma32(R[a, 0], dx, t[a]))) for a in range(3)]
    ok &= Y[2] > f32(0)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        iz = f32(1) / np.where(ok, Y[2], f32(1))
        ux = fma32(fx, Y[0] * iz, cx)
        uy = fma32(fy, Y[1] * iz, cy)
    ux = np.where(ok, ux, f32(-100))
    uy = np.where(ok, uy, f32(-100))
    nxf = np.floor(ux + f32(0.5))
    nyf = np.floor(uy + f32(0.5))
    ok &= (nxf >= 0) & (nxf <= W - 1) & (nyf >= 0) & (nyf <= H - 1)
    bxf = np.floor(ux)
    byf = np.floor(uy)
    ok &= (bxf >= 2) & (bxf + 1 <= W - 3) & (byf >= 2) & (byf + 1 <= H - 3)
    nx = np.where(ok, nxf, 0).astype(np.int64)
    ny = np.where(ok, nyf, 0).astype(np.int64)
    bx = np.where(ok, bxf, 0).astype(np.int64)
    by = np.where(ok, byf, 0).astype(np.int64)
    tgt = ny * W + nx
    ok &= fj.valid.ravel()[tgt] & fj.nvalid.ravel()[tgt]
    Dj = fj.D32.ravel()[tgt]
    qx = kx[nx] * Dj
    qy = ky[ny] * Dj
    qz = Dj
    ex, ey, ez = Y[0] - qx, Y[1] - qy, Y[2] - qz
    dist2 = fma32(ez, ez, fma32(ey, ey, ex * ex))
    ok &= dist2 < f32(tau_d * tau_d)
    m = [fma32(R[a, 2], n_i[:, 2], fma32(R[a, 1], n_i[:, 1], R[a, 0] * n_i[:, 0])) for a in range(3)]
    n_j = fj.N32.reshape(-1, 3)[tgt]
    dot = fma32(m[2], n_j[:, 2], fma32(m[1], n_j[:, 1], m[0] * n_j[:, 0]))
    ok &= dot > f32(tau_n)
    return dict(valid=ok, nx=nx, ny=ny, bx=bx, by=by)
