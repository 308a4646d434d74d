// Sparse feature term evaluation (one correspondence segment), shared by the sparse kernel of
// sparse.cu and the persistent batched solve of solve.cu; the design notes are at the top of
// sparse.cu.
#pragma once
#include "bf_internal.cuh"

namespace bf {


constexpr int SPARSE_BS = 128;  // threads of k_sparse: 4 warps, one segment each

// One correspondence segment s, evaluated by the calling warp: lanes stride the
// correspondences, a warp reduce-scatter sums the 57 partial sums (lane l writes sums 2l and
// 2l + 1), and in ENERGY mode a butterfly finds the largest distance (first index on ties).  No
// barrier.  CG: the pair transform is read through L2 (written by another CTA of a persistent
// launch).
template <int MODE, typename Part, bool CG = false>
__device__ __forceinline__ void sparse_seg(int s, const Tables &t, const float4 *__restrict__ P,
                                           const float4 *__restrict__ Q, const float *__restrict__ pairM,
                                           float w_sparse, Part *__restrict__ part, float *__restrict__ seg_rmax,
                                           int *__restrict__ seg_rarg) {
  const int lane = threadIdx.x & 31;
  const int pr = t.seg_pair[s];
  const int off = t.seg_off[s], cnt = t.seg_cnt[s];
  const bool swap = t.seg_swap[s] != 0;
  const float *M = pairM + pr * 24;  // T_b^-1 T_a
  float Mv[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) Mv[k] = CG ? __ldcg(M + k) : M[k];
  const float R00 = Mv[0], R01 = Mv[1], R02 = Mv[2], R10 = Mv[3], R11 = Mv[4], R12 = Mv[5];
  const float R20 = Mv[6], R21 = Mv[7], R22 = Mv[8], t0 = Mv[9], t1 = Mv[10], t2 = Mv[11];
  float acc[NPART];
#pragma unroll
  for (int k = 0; k < NPART; ++k) acc[k] = 0.f;
  float best = -1.f;
  int barg = 0x7fffffff;
  for (int k = lane; k < cnt; k += 32) {
    const float4 u = P[off + k], v = Q[off + k];
    // p in camera a, q in camera b (the pool stores the smaller frame id first)
    const float px = swap ? v.x : u.x, py = swap ? v.y : u.y, pz = swap ? v.z : u.z;
    const float qx = swap ? u.x : v.x, qy = swap ? u.y : v.y, qz = swap ? u.z : v.z;
    const float wc = u.w;
    const float A0 = R00 * px + R01 * py + R02 * pz;
    const float A1 = R10 * px + R11 * py + R12 * pz;
    const float A2 = R20 * px + R21 * py + R22 * pz;
    const float r0 = A0 + t0 - qx, r1 = A1 + t1 - qy, r2 = A2 + t2 - qz;
    const float d2 = r0 * r0 + r1 * r1 + r2 * r2;
    acc[P_E0] += wc * d2;
    acc[P_CNT] += 1.f;
    if (MODE == MODE_ENERGY) {
      const float dist = sqrtf(d2);
      if (dist > best) {
        best = dist;
        barg = k;
      }
    }
    if (MODE == MODE_ACCUM) {
      const float w = w_sparse * wc;
      // rows k = 0,1,2: a_k = A x e_k, v_k = e_k, c_k = e_k x q, written out per entry.
      // a_0 = (0, A2, -A1), a_1 = (-A2, 0, A0), a_2 = (A1, -A0, 0)
      // c_0 = (0, -qz, qy), c_1 = (qz, 0, -qx), c_2 = (-qy, qx, 0)
      // S_aa = sum_k a_k a_k^T = |A|^2 I - A A^T
      const float AA = A0 * A0 + A1 * A1 + A2 * A2;
      acc[P_AA + 0] += w * (AA - A0 * A0);
      acc[P_AA + 1] += w * (-A0 * A1);
      acc[P_AA + 2] += w * (-A0 * A2);
      acc[P_AA + 3] += w * (AA - A1 * A1);
      acc[P_AA + 4] += w * (-A1 * A2);
      acc[P_AA + 5] += w * (AA - A2 * A2);
      // S_av = sum_k a_k e_k^T = [a_0 a_1 a_2] as columns = [A]_x^T... entry (m, k) = (a_k)_m
      acc[P_AV + 0] += 0.f;       acc[P_AV + 1] += w * -A2;  acc[P_AV + 2] += w * A1;
      acc[P_AV + 3] += w * A2;    acc[P_AV + 4] += 0.f;      acc[P_AV + 5] += w * -A0;
      acc[P_AV + 6] += w * -A1;   acc[P_AV + 7] += w * A0;   acc[P_AV + 8] += 0.f;
      // S_vv = I
      acc[P_VV + 0] += w; acc[P_VV + 3] += w; acc[P_VV + 5] += w;
      // S_ac = sum_k a_k c_k^T ; S_vc = sum_k e_k c_k^T (row k = c_k) ; S_cc = |q|^2 I - q q^T
      {
        const float a[3][3] = {{0.f, A2, -A1}, {-A2, 0.f, A0}, {A1, -A0, 0.f}};
        const float c[3][3] = {{0.f, -qz, qy}, {qz, 0.f, -qx}, {-qy, qx, 0.f}};
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
          for (int n = 0; n < 3; ++n)
            acc[P_AC + 3 * m + n] += w * (a[0][m] * c[0][n] + a[1][m] * c[1][n] + a[2][m] * c[2][n]);
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
          for (int n = 0; n < 3; ++n) acc[P_VC + 3 * m + n] += w * c[m][n];
        const float qq = qx * qx + qy * qy + qz * qz;
        acc[P_CC + 0] += w * (qq - qx * qx);
        acc[P_CC + 1] += w * (-qx * qy);
        acc[P_CC + 2] += w * (-qx * qz);
        acc[P_CC + 3] += w * (qq - qy * qy);
        acc[P_CC + 4] += w * (-qy * qz);
        acc[P_CC + 5] += w * (qq - qz * qz);
        const float rr[3] = {r0, r1, r2};
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          acc[P_GA + m] += w * (a[0][m] * rr[0] + a[1][m] * rr[1] + a[2][m] * rr[2]);
          acc[P_GV + m] += w * rr[m];
          acc[P_GC + m] += w * (c[0][m] * rr[0] + c[1][m] * rr[1] + c[2][m] * rr[2]);
        }
      }
    }
  }
  float v[64];
#pragma unroll
  for (int k = 0; k < 64; ++k) v[k] = k < NPART ? acc[k] : 0.f;
  warp_reduce_scatter<64>(v);
  Part *out = part + (long long)s * NPART;
  if (2 * lane < NPART) out[2 * lane] = (Part)v[0];
  if (2 * lane + 1 < NPART) out[2 * lane + 1] = (Part)v[1];
  if (MODE == MODE_ENERGY) {
    // max and its first index over the segment (ties -> smallest index)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oa = __shfl_xor_sync(0xffffffffu, barg, o);
      if (ob > best || (ob == best && oa < barg)) {
        best = ob;
        barg = oa;
      }
    }
    if (lane == 0) {
      seg_rmax[s] = best;
      seg_rarg[s] = barg;
    }
  }
}

}  // namespace bf
