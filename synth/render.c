/*
 * Analytic ray caster for the synthetic "box room" scenes.
 *
 * This is input generation only: it renders depth (camera z) and an albedo
 * luminance image for a set of axis-aligned boxes seen from pinhole cameras.
 * It knows nothing about the pose solver.  Both the FP64 oracle and the CUDA
 * library consume its output, so it must be deterministic: plain double
 * arithmetic, no FMA contraction (built with -ffp-contract=off), one pixel per
 * loop iteration with no cross-pixel state.
 *
 * Scene model:
 *   box k spans [lo_k, hi_k] (world, metres).  kind 0 = room shell (the camera
 *   is inside, the visible surface is where the ray leaves), kind 1 = solid box
 *   (visible surface is where the ray enters).
 *   Each (box, face) pair owns TEX_STRIDE texture parameters:
 *     base, 3 x (amp, freq_u, freq_v, phase), cell, contrast, patch_phase
 *   albedo(u,v) = base + sum_k amp_k sin(fu_k u + fv_k v + ph_k)
 *                 + contrast * (checker(u,v,cell) - 0.5), clipped to [0,1].
 *   (u,v) are the two world coordinates spanning the face.
 *
 * Camera: pose (R,t) maps camera -> world, row-major R then t (12 doubles).
 * Pixel (x,y) has its centre at integer coordinates; the ray direction in the
 * camera frame is ((x-cx)/fx, (y-cy)/fy, 1), so the hit parameter equals the
 * camera-frame depth z.
 */
#include <math.h>
#include <stdint.h>

#define TEX_STRIDE 16

static double albedo(const double *tp, double u, double v) {
  double a = tp[0];
  for (int k = 0; k < 3; ++k) {
    const double *s = tp + 1 + 4 * k;
    a += s[0] * sin(s[1] * u + s[2] * v + s[3]);
  }
  double cell = tp[13];
  if (cell > 0.0) {
    long cu = (long)floor(u / cell + tp[15]);
    long cv = (long)floor(v / cell + tp[15]);
    double chk = (double)(((cu + cv) % 2 + 2) % 2);
    a += tp[14] * (chk - 0.5);
  }
  if (a < 0.0) a = 0.0;
  if (a > 1.0) a = 1.0;
  return a;
}

/* Slab test. Returns 1 and the entry/exit parameters and axes if the ray
 * overlaps the box for some t. */
static int slab(const double o[3], const double d[3], const double lo[3],
                const double hi[3], double *t0, double *t1, int *ax0, int *ax1,
                int *side0, int *side1) {
  double tn = -1e300, tf = 1e300;
  int an = -1, af = -1, sn = 0, sf = 0;
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0) {
      if (o[a] < lo[a] || o[a] > hi[a]) return 0;
      continue;
    }
    double ta = (lo[a] - o[a]) / d[a];
    double tb = (hi[a] - o[a]) / d[a];
    int sa = 0, sb = 1; /* 0 = lo face, 1 = hi face */
    if (ta > tb) {
      double tmp = ta; ta = tb; tb = tmp;
      sa = 1; sb = 0;
    }
    if (ta > tn) { tn = ta; an = a; sn = sa; }
    if (tb < tf) { tf = tb; af = a; sf = sb; }
  }
  if (tn > tf) return 0;
  *t0 = tn; *t1 = tf; *ax0 = an; *ax1 = af; *side0 = sn; *side1 = sf;
  return 1;
}

/*
 * Render n_frames frames of W x H.
 *   poses:   n_frames x 12 doubles (R row-major, t)
 *   lo, hi:  n_boxes x 3 doubles; kind: n_boxes ints
 *   tex:     n_boxes x 6 faces x TEX_STRIDE doubles (face = 2*axis + side)
 *   depth:   n_frames x H x W floats, camera z of the first surface (0 if none)
 *   lum:     n_frames x H x W floats, albedo of that surface
 */
void synth_render(int n_frames, int W, int H, double fx, double fy, double cx,
                  double cy, const double *poses, int n_boxes, const double *lo,
                  const double *hi, const int *kind, const double *tex,
                  float *depth, float *lum) {
  long n_pix = (long)n_frames * W * H;
#pragma omp parallel for schedule(static)
  for (long idx = 0; idx < n_pix; ++idx) {
    long f = idx / ((long)W * H);
    long rem = idx - f * (long)W * H;
    int y = (int)(rem / W), x = (int)(rem - (long)y * W);
    const double *P = poses + 12 * f;
    double dc[3] = {((double)x - cx) / fx, ((double)y - cy) / fy, 1.0};
    double dw[3], o[3] = {P[9], P[10], P[11]};
    for (int r = 0; r < 3; ++r)
      dw[r] = P[3 * r + 0] * dc[0] + P[3 * r + 1] * dc[1] + P[3 * r + 2] * dc[2];
    double best = 1e300;
    int best_box = -1, best_ax = 0, best_side = 0;
    for (int b = 0; b < n_boxes; ++b) {
      double t0, t1;
      int a0, a1, s0, s1;
      if (!slab(o, dw, lo + 3 * b, hi + 3 * b, &t0, &t1, &a0, &a1, &s0, &s1))
        continue;
      if (kind[b] == 0) {
        if (t1 > 1e-9 && t1 < best) {
          best = t1; best_box = b; best_ax = a1; best_side = s1;
        }
      } else {
        if (t0 > 1e-9 && t0 < best) {
          best = t0; best_box = b; best_ax = a0; best_side = s0;
        }
      }
    }
    if (best_box < 0) {
      depth[idx] = 0.0f;
      lum[idx] = 0.0f;
      continue;
    }
    double hp[3];
    for (int r = 0; r < 3; ++r) hp[r] = o[r] + best * dw[r];
    int ua = (best_ax + 1) % 3, va = (best_ax + 2) % 3;
    const double *tp = tex + ((long)best_box * 6 + 2 * best_ax + best_side) * TEX_STRIDE;
    depth[idx] = (float)best;
    lum[idx] = (float)albedo(tp, hp[ua], hp[va]);
  }
}
