"""Per-frame preprocessing (oracle, FP64).

Sec. 4.1.1 caches, per frame, the low-resolution depth, the camera-space positions
P^low and normals N^low; Sec. 4.3 evaluates the photometric term on the gradient of
the luminance, I_i.  The paper gives no formulas for either, so this follows the
readings below (pixel centres at integer coordinates, pinhole intrinsics fx, fy,
cx, cy):

* depth D is valid iff finite and depth_min < D < depth_max; invalid depth -> 0;
* back-projection pi^-1(x, y, z) = ((x - cx) z / fx, (y - cy) z / fy, z);
* normal n = normalize((P(x,y+1) - P(x,y-1)) x (P(x+1,y) - P(x-1,y))), which faces the
  camera on every front-facing surface; invalid on the 1-pixel border, if the pixel or
  any of its 4 neighbours has invalid depth, or if the cross product's norm < 1e-12;
* I = ||grad L||_2 with central differences (f(x+1) - f(x-1)) / 2, defined on the
  1-pixel interior (0 elsewhere);
* grad I by central differences of I, defined on the 2-pixel interior (0 elsewhere).

16-bit frame storage (a B300 memory-layout option; the paper keeps its cached frames in
FP32): normals, I and grad I are rounded to BF16 or FP16 (round to nearest, ties to even)
and depth stays FP32.  The oracle rounds its own FP64 values, so it sees the same stored
images as the device up to the rare value whose FP32 and FP64 results straddle a 16-bit
rounding boundary.
"""
import numpy as np

# 16-bit storage formats: (significant bits incl. the implicit one, exponent of the smallest
# subnormal spacing, largest finite value)
STORAGE_FORMATS = {
    "bf16": (8, -133, float.fromhex("0x1.fep127")),
    "fp16": (11, -24, 65504.0),
}


def round_to_storage(x, kind):
    """Round FP64 values to the nearest BF16 / FP16 value, ties to even (IEEE 754 rounding).

    x = m 2^e with 0.5 <= |m| < 1 keeps p significant bits: the quantum is 2^(e - p), floored at
    the format's subnormal spacing; values past the largest finite one become +-inf."""
    if kind in (None, "fp32"):
        return np.asarray(x, dtype=np.float64)
    p, s_min, vmax = STORAGE_FORMATS[kind]
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)
    qexp = np.maximum(e - p, s_min)
    q = np.ldexp(np.round(np.ldexp(x, -qexp)), qexp)  # np.round: half to even
    return np.where(np.abs(q) > vmax, np.copysign(np.inf, x), q)


def valid_depth(D, depth_min, depth_max):
    D = np.asarray(D, dtype=np.float64)
    return np.isfinite(D) & (D > depth_min) & (D < depth_max)


def backproject(D, fx, fy, cx, cy):
    """Camera-space points P(x,y) = pi^-1(x, y, D(x,y)), shape (H,W,3), FP64."""
    H, W = D.shape
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    z = np.asarray(D, dtype=np.float64)
    return np.stack([(xs - cx) * z / fx, (ys - cy) * z / fy, z], axis=-1)


def normals(D, valid, fx, fy, cx, cy):
    """Per-pixel unit normals (H,W,3) and their validity mask (H,W)."""
    H, W = D.shape
    P = backproject(np.where(valid, D, 0.0), fx, fy, cx, cy)
    n = np.zeros((H, W, 3))
    ok = np.zeros((H, W), dtype=bool)
    c = (slice(1, H - 1), slice(1, W - 1))
    dy = P[2:, 1:-1] - P[:-2, 1:-1]
    dx = P[1:-1, 2:] - P[1:-1, :-2]
    cr = np.cross(dy, dx)
    nrm = np.sqrt(np.sum(cr * cr, axis=-1))
    nb = valid[c] & valid[2:, 1:-1] & valid[:-2, 1:-1] & valid[1:-1, 2:] & valid[1:-1, :-2]
    good = nb & (nrm >= 1e-12)
    inner = np.zeros_like(cr)
    inner[good] = cr[good] / nrm[good][:, None]
    n[c] = inner
    ok[c] = good
    return n, ok


def intensity_gradient(L):
    """I = ||grad L||_2 on the 1-pixel interior and grad I = (I_x, I_y) on the 2-pixel interior."""
    L = np.asarray(L, dtype=np.float64)
    H, W = L.shape
    I = np.zeros((H, W))
    gx = 0.5 * (L[1:-1, 2:] - L[1:-1, :-2])
    gy = 0.5 * (L[2:, 1:-1] - L[:-2, 1:-1])
    I[1:-1, 1:-1] = np.sqrt(gx * gx + gy * gy)
    Ix = np.zeros((H, W))
    Iy = np.zeros((H, W))
    Ix[2:-2, 2:-2] = 0.5 * (I[2:-2, 3:-1] - I[2:-2, 1:-3])
    Iy[2:-2, 2:-2] = 0.5 * (I[3:-1, 2:-2] - I[1:-3, 2:-2])
    return I, Ix, Iy


class Frame:
    """A preprocessed frame: depth, validity, normals, I and grad I (all FP64).

    storage "bf16" / "fp16" rounds N, I and grad I to that format after computing them in
    FP64 (depth stays exact); None or "fp32" keeps them as computed."""

    def __init__(self, depth, lum, intr, depth_min=0.1, depth_max=10.0, storage=None):
        self.W, self.H = intr["W"], intr["H"]
        self.fx, self.fy, self.cx, self.cy = intr["fx"], intr["fy"], intr["cx"], intr["cy"]
        D = np.asarray(depth, dtype=np.float64)
        self.valid = valid_depth(D, depth_min, depth_max)
        self.D = np.where(self.valid, D, 0.0)
        self.N, self.nvalid = normals(self.D, self.valid, self.fx, self.fy, self.cx, self.cy)
        self.I, self.Ix, self.Iy = intensity_gradient(lum)
        # the intensity itself, for the dense verification's photoconsistency test (Sec. 4.1.1)
        self.C = np.asarray(lum, dtype=np.float64)
        self.storage = storage
        if storage not in (None, "fp32"):
            self.N = round_to_storage(self.N, storage)
            self.I, self.Ix, self.Iy = (round_to_storage(v, storage) for v in (self.I, self.Ix, self.Iy))
            self.C = round_to_storage(self.C, storage)
        # FP32 depth and intensity: the inputs of the TSDF oracle (tsdf.py), which takes its
        # quantised decisions in FP32
        self.D32 = self.D.astype(np.float32)
        self.C32 = self.C.astype(np.float32)


class FrameCache:
    """Frames built on first use from raw depth / luminance arrays and kept (frame id -> Frame)."""

    def __init__(self, depth, lum, intr, depth_min=0.1, depth_max=10.0, storage=None):
        self.depth, self.lum, self.intr = depth, lum, intr
        self.args = (depth_min, depth_max, storage)
        self.cache = {}

    def __getitem__(self, k):
        k = int(k)
        if k not in self.cache:
            self.cache[k] = Frame(self.depth[k], self.lum[k], self.intr, *self.args)
        return self.cache[k]

    def __len__(self):
        return len(self.depth)


def preprocess(problem_depth, problem_lum, intr, depth_min=0.1, depth_max=10.0, storage=None):
    return [Frame(d, l, intr, depth_min, depth_max, storage) for d, l in zip(problem_depth, problem_lum)]
