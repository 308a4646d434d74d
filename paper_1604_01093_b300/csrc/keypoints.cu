// Key-point correspondence filter and surface-area filter (Sec. 4.1.1), batched over frame pairs.
//
// One warp per frame pair.  The pair's matches arrive in order of match distance; the warp grows
// the set one match at a time.  After each addition it fits the rigid transform q ~ R p + t that
// minimises the RMSD over the set (Kabsch: SVD of the centred cross-covariance H), and the set
// fails when the largest residual exceeds max_residual or the fit is ambiguous: a condition
// number sigma_1 / sigma_2 above max_cond for the covariance of the set's p points, of its q
// points, or for H (nearly collinear points leave a rotation undetermined).  While it fails, the
// match with the largest residual (the earliest on a tie) leaves the set, until the set passes
// or fewer than 3 remain.  A pair keeps its matches if at least min_matches survive and the
// bounding rectangles of the kept p and q points in the planes of their two principal axes
// both cover at least min_area.
//
// Arithmetic is FP64 throughout (the keep/drop decisions compare fitted residuals and
// condition numbers with thresholds): lanes split the sums and residuals over the set, lanes
// 0-2 run the three symmetric 3x3 eigen-decompositions (cyclic Jacobi) side by side.  The
// membership of the set is a bit mask in shared memory; since matches join in index order, the
// set's order is index order.
#include "bf_internal.cuh"

namespace bf {

constexpr int KP_WARPS = 4;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (a00 a01 a02 a11 a12 a22).
// Eigenvalues w (descending) and eigenvectors V (column k = V[k], V[3 + k], V[6 + k]).
__device__ void jacobi3(const double *S, double *w, double *V) {
  double a[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
  double v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 16; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (!(off > 1e-36 * dia)) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        const double apq = a[p][q];
        if (apq == 0.0) continue;
        // rotation annihilating a[p][q]: theta = (a_qq - a_pp) / (2 a_pq), t = tan of the angle
        const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; ++k) {  // columns p, q of a
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // rows p, q
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
  }
  int o[3] = {0, 1, 2};  // sort descending
  for (int i = 0; i < 2; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (a[o[j]][o[j]] > a[o[i]][o[i]]) {
        const int tmp = o[i];
        o[i] = o[j];
        o[j] = tmp;
      }
  for (int k = 0; k < 3; ++k) {
    w[k] = a[o[k]][o[k]];
    for (int r = 0; r < 3; ++r) V[3 * r + k] = v[r][o[k]];
  }
}

__device__ __forceinline__ double ratio12(double s1, double s2) { return s2 > 0.0 ? s1 / s2 : INFINITY; }

struct KpPair {
  double R[9], t[3];
  int status;  // 0 kept, 1 too few, 2 area too small
  int pad;
};

template <int NMAX>
__global__ void __launch_bounds__(32 * KP_WARPS)
    k_keypoints(int n_pairs, const int *__restrict__ off, const float *__restrict__ P, const float *__restrict__ Q,
                double max_res, double max_cond, int min_matches, double min_area, unsigned char *__restrict__ keep,
                KpPair *__restrict__ res) {
  __shared__ unsigned mask_sh[KP_WARPS][NMAX / 32];
  __shared__ double fit_sh[KP_WARPS][16];  // R (9), t (3), stable flag
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int pr = blockIdx.x * KP_WARPS + w;
  if (pr >= n_pairs) return;  // whole warp
  unsigned *mask = mask_sh[w];
  double *fit = fit_sh[w];
  const int o0 = off[pr], n = off[pr + 1] - off[pr];
  const float *Pp = P + 3LL * o0, *Qp = Q + 3LL * o0;
  for (int k = lane; k < NMAX / 32; k += 32) mask[k] = 0u;
  __syncwarp();
  int size = 0;
  // sums over the set -> centroids, covariances, cross-covariance; lanes 0-2 decompose; lane 0
  // forms R, t.  Returns the stable flag (warp-uniform); R, t in fit[].
  auto fit_set = [&](int added) -> bool {
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int k = lane; k < added; k += 32)
      if (mask[k >> 5] >> (k & 31) & 1u) {
        s[0] += Pp[3 * k];
        s[1] += Pp[3 * k + 1];
        s[2] += Pp[3 * k + 2];
        s[3] += Qp[3 * k];
        s[4] += Qp[3 * k + 1];
        s[5] += Qp[3 * k + 2];
      }
    double c[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) c[i] = warp_sum_d(s[i]) / (double)size;
    double m[21];  // Cp (6), Cq (6), H (9) = sum pc qc^T
#pragma unroll
    for (int i = 0; i < 21; ++i) m[i] = 0.0;
    for (int k = lane; k < added; k += 32)
      if (mask[k >> 5] >> (k & 31) & 1u) {
        const double p0 = Pp[3 * k] - c[0], p1 = Pp[3 * k + 1] - c[1], p2 = Pp[3 * k + 2] - c[2];
        const double q0 = Qp[3 * k] - c[3], q1 = Qp[3 * k + 1] - c[4], q2 = Qp[3 * k + 2] - c[5];
        m[0] += p0 * p0; m[1] += p0 * p1; m[2] += p0 * p2; m[3] += p1 * p1; m[4] += p1 * p2; m[5] += p2 * p2;
        m[6] += q0 * q0; m[7] += q0 * q1; m[8] += q0 * q2; m[9] += q1 * q1; m[10] += q1 * q2; m[11] += q2 * q2;
        m[12] += p0 * q0; m[13] += p0 * q1; m[14] += p0 * q2;
        m[15] += p1 * q0; m[16] += p1 * q1; m[17] += p1 * q2;
        m[18] += p2 * q0; m[19] += p2 * q1; m[20] += p2 * q2;
      }
#pragma unroll
    for (int i = 0; i < 21; ++i) m[i] = warp_sum_d(m[i]);
    const double *H = m + 12;
    // lane 0: H^T H; lane 1: Cp; lane 2: Cq
    double S[6];
    if (lane == 0) {
      double HtH[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) HtH[a][b] = H[a] * H[b] + H[3 + a] * H[3 + b] + H[6 + a] * H[6 + b];
      S[0] = HtH[0][0]; S[1] = HtH[0][1]; S[2] = HtH[0][2]; S[3] = HtH[1][1]; S[4] = HtH[1][2]; S[5] = HtH[2][2];
    } else if (lane == 1) {
      for (int i = 0; i < 6; ++i) S[i] = m[i];
    } else {
      for (int i = 0; i < 6; ++i) S[i] = m[6 + i];
    }
    double ew[3] = {0, 0, 0}, V[9];
    if (lane < 3) jacobi3(S, ew, V);
    double cond = 0.0;
    if (lane == 0) cond = ratio12(sqrt(fmax(ew[0], 0.0)), sqrt(fmax(ew[1], 0.0)));
    else if (lane < 3) cond = ratio12(ew[0], ew[1]);
    const double c1 = __shfl_sync(0xffffffffu, cond, 1), c2 = __shfl_sync(0xffffffffu, cond, 2);
    if (lane == 0) {
      // H = U diag(sigma) V^T: u_i = H v_i / sigma_i (i = 1, 2), u_3 = +-(u_1 x u_2) on the side of
      // H v_3; R = V diag(1, 1, d) U^T with d = det(V U^T)
      double U[9];
      for (int i = 0; i < 2; ++i) {
        const double sg = sqrt(fmax(ew[i], 0.0));
        for (int r = 0; r < 3; ++r) {
          const double hv = H[3 * r] * V[i] + H[3 * r + 1] * V[3 + i] + H[3 * r + 2] * V[6 + i];
          U[3 * r + i] = sg > 0.0 ? hv / sg : 0.0;
        }
      }
      double u3[3] = {U[3] * U[7] - U[6] * U[4], U[6] * U[1] - U[0] * U[7], U[0] * U[4] - U[3] * U[1]};
      double hv3 = 0.0;
      for (int r = 0; r < 3; ++r)
        hv3 += (H[3 * r] * V[2] + H[3 * r + 1] * V[5] + H[3 * r + 2] * V[8]) * u3[r];
      const double sgn = hv3 < 0.0 ? -1.0 : 1.0;
      for (int r = 0; r < 3; ++r) U[3 * r + 2] = sgn * u3[r];
      double VU[9];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) VU[3 * a + b] = V[3 * a] * U[3 * b] + V[3 * a + 1] * U[3 * b + 1] + V[3 * a + 2] * U[3 * b + 2];
      const double det = VU[0] * (VU[4] * VU[8] - VU[5] * VU[7]) - VU[1] * (VU[3] * VU[8] - VU[5] * VU[6]) +
                         VU[2] * (VU[3] * VU[7] - VU[4] * VU[6]);
      const double d = det < 0.0 ? -1.0 : 1.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          fit[3 * a + b] = V[3 * a] * U[3 * b] + V[3 * a + 1] * U[3 * b + 1] + d * V[3 * a + 2] * U[3 * b + 2];
      for (int a = 0; a < 3; ++a)
        fit[9 + a] = c[3 + a] - (fit[3 * a] * c[0] + fit[3 * a + 1] * c[1] + fit[3 * a + 2] * c[2]);
      fit[12] = (cond <= max_cond && c1 <= max_cond && c2 <= max_cond) ? 1.0 : 0.0;
    }
    __syncwarp();
    return fit[12] != 0.0;
  };
  // largest residual over the set and its (lowest) index
  auto worst = [&](int added, double &rmax) -> int {
    double best = -1.0;
    int arg = 0x7fffffff;
    for (int k = lane; k < added; k += 32)
      if (mask[k >> 5] >> (k & 31) & 1u) {
        double e2 = 0.0;
        for (int a = 0; a < 3; ++a) {
          const double r = fit[3 * a] * Pp[3 * k] + fit[3 * a + 1] * Pp[3 * k + 1] + fit[3 * a + 2] * Pp[3 * k + 2] +
                           fit[9 + a] - Qp[3 * k + a];
          e2 += r * r;
        }
        const double e = sqrt(e2);
        if (e > best) {  // k ascends within a lane: the first of equals stays
          best = e;
          arg = k;
        }
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
      if (ob > best || (ob == best && oa < arg)) {
        best = ob;
        arg = oa;
      }
    }
    rmax = best;
    return arg;
  };
  for (int k = 0; k < n; ++k) {
    if (lane == 0) mask[k >> 5] |= 1u << (k & 31);
    __syncwarp();
    ++size;
    while (size >= 3) {
      const bool ok = fit_set(k + 1);
      double rmax;
      const int arg = worst(k + 1, rmax);
      if (rmax <= max_res && ok) break;
      if (lane == 0) mask[arg >> 5] &= ~(1u << (arg & 31));
      __syncwarp();
      --size;
    }
  }
  int status = 0;
  if (size < max(min_matches, 3)) {
    status = 1;
  } else {
    fit_set(n);
    // surface areas of the kept p and q points: lanes 1, 2 of the next decomposition give the
    // principal axes; project and take the extents
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int k = lane; k < n; k += 32)
      if (mask[k >> 5] >> (k & 31) & 1u)
        for (int i = 0; i < 3; ++i) {
          s[i] += Pp[3 * k + i];
          s[3 + i] += Qp[3 * k + i];
        }
    double c[6];
    for (int i = 0; i < 6; ++i) c[i] = warp_sum_d(s[i]) / (double)size;
    double cp[6] = {0, 0, 0, 0, 0, 0}, cq[6] = {0, 0, 0, 0, 0, 0};
    for (int k = lane; k < n; k += 32)
      if (mask[k >> 5] >> (k & 31) & 1u) {
        const double p0 = Pp[3 * k] - c[0], p1 = Pp[3 * k + 1] - c[1], p2 = Pp[3 * k + 2] - c[2];
        const double q0 = Qp[3 * k] - c[3], q1 = Qp[3 * k + 1] - c[4], q2 = Qp[3 * k + 2] - c[5];
        cp[0] += p0 * p0; cp[1] += p0 * p1; cp[2] += p0 * p2; cp[3] += p1 * p1; cp[4] += p1 * p2; cp[5] += p2 * p2;
        cq[0] += q0 * q0; cq[1] += q0 * q1; cq[2] += q0 * q2; cq[3] += q1 * q1; cq[4] += q1 * q2; cq[5] += q2 * q2;
      }
    for (int i = 0; i < 6; ++i) {
      cp[i] = warp_sum_d(cp[i]);
      cq[i] = warp_sum_d(cq[i]);
    }
    double ew[3], Vp[9], Vq[9];
    jacobi3(cp, ew, Vp);  // every lane decomposes (the axes are needed by all for the projection)
    jacobi3(cq, ew, Vq);
    double lo[4] = {INFINITY, INFINITY, INFINITY, INFINITY}, hi[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int k = lane; k < n; k += 32)
      if (mask[k >> 5] >> (k & 31) & 1u) {
        const double p0 = Pp[3 * k] - c[0], p1 = Pp[3 * k + 1] - c[1], p2 = Pp[3 * k + 2] - c[2];
        const double q0 = Qp[3 * k] - c[3], q1 = Qp[3 * k + 1] - c[4], q2 = Qp[3 * k + 2] - c[5];
        const double x[4] = {p0 * Vp[0] + p1 * Vp[3] + p2 * Vp[6], p0 * Vp[1] + p1 * Vp[4] + p2 * Vp[7],
                             q0 * Vq[0] + q1 * Vq[3] + q2 * Vq[6], q0 * Vq[1] + q1 * Vq[4] + q2 * Vq[7]};
        for (int i = 0; i < 4; ++i) {
          lo[i] = fmin(lo[i], x[i]);
          hi[i] = fmax(hi[i], x[i]);
        }
      }
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo[i] = fmin(lo[i], __shfl_xor_sync(0xffffffffu, lo[i], o));
        hi[i] = fmax(hi[i], __shfl_xor_sync(0xffffffffu, hi[i], o));
      }
    const double ap = (hi[0] - lo[0]) * (hi[1] - lo[1]), aq = (hi[2] - lo[2]) * (hi[3] - lo[3]);
    if (fmin(ap, aq) < min_area) status = 2;
  }
  for (int k = lane; k < n; k += 32)
    keep[o0 + k] = (status == 0 && (mask[k >> 5] >> (k & 31) & 1u)) ? 1 : 0;
  if (lane == 0) {
    KpPair &r = res[pr];
    r.status = status;
    r.pad = 0;
    for (int i = 0; i < 9; ++i) r.R[i] = status == 0 ? fit[i] : 0.0;
    for (int i = 0; i < 3; ++i) r.t[i] = status == 0 ? fit[9 + i] : 0.0;
  }
}

constexpr int KP_NMAX = 1024;

int keypoint_nmax() { return KP_NMAX; }

int launch_keypoints(int n_pairs, const int *off, const float *P, const float *Q, double max_res, double max_cond,
                     int min_matches, double min_area, unsigned char *keep, void *res, cudaStream_t st) {
  if (n_pairs <= 0) return 0;
  k_keypoints<KP_NMAX><<<(n_pairs + KP_WARPS - 1) / KP_WARPS, 32 * KP_WARPS, 0, st>>>(
      n_pairs, off, P, Q, max_res, max_cond, min_matches, min_area, keep, (KpPair *)res);
  return 1;
}

size_t keypoint_result_bytes() { return sizeof(KpPair); }

}  // namespace bf
