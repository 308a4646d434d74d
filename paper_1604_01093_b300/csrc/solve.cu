// Linear-system assembly, block-Jacobi PCG and the pose update (Sec. 4.4).
//
//   k_pair_xform   per pair: T_b^-1 T_a and T_a^-1 T_b, FP64 with explicit rounding, stored FP32
//   k_pair_merge   warp per pair: sum the pair's tile / segment partials (FP64 in mixed
//                  precision), rotate them from target-camera to world coordinates and expand the
//                  [a, v, c, -v] sums into the 6x6 blocks A_aa, A_ab, A_bb and rhs_a, rhs_b
//   k_assemble     warp per free frame: its diagonal block and rhs (sum over incident pairs in a
//                  fixed order) and the preconditioner: 6x6 Cholesky inverse (block-Jacobi) or the
//                  inverse diagonal (Jacobi, the paper's choice)
//   k_pcg          one CTA per problem (batches of small problems): exactly n_pcg PCG
//                  iterations from x = 0, stopping early only if p.Ap <= 0 or r.z == 0; a problem
//                  with at most 16 free frames keeps its whole system in shared memory
//   k_pcg_coop     one large problem over many CTAs (cooperative launch, all CTAs resident):
//                  warp per frame, two grid barriers per iteration, deterministic dot products
//   k_pcg_cluster  one large problem on a thread-block cluster (distributed shared memory)
// With the matrix-free sparse term (MatFree, Sec. 4.4's own scheme) k_pcg (general path) and
// k_pcg_coop evaluate J p and J^T (J p) over the correspondences in every iteration and read the
// dense term alone from the assembled blocks.
// Each PCG kernel also writes the problem's energy record of the linearisation it solves (the
// pairs' records summed in a fixed order) and, once the step is final, applies the exp-map pose
// update R <- Exp(dw) R, t <- t + dt (FP64) to its free frames; k_pcg then forms its pairs'
// transforms for the next linearisation.  A GN iteration of a batch of chunks is five launches:
// dense, sparse, merge, assemble, PCG.
//
// The paper's solver (Sec. 4.4) sums the PCG scalars with warp shuffles plus global atomics in a
// single kernel; here every dot product is reduced in a fixed order (warp tree, then CTA
// partials summed in index order by every CTA) so results do not depend on scheduling.
// Precision (mixed mode): vectors and their element-wise updates are FP32; a dot product's
// products are summed in FP32 within a warp (a 32-term tree) and everything above the warp,
// plus alpha and beta, in FP64.  B300 issues FP64 at 1/64 of the FP32 rate, so per-element
// FP64 arithmetic would dominate these latency-bound kernels.
#include <cooperative_groups.h>

#include <algorithm>

#include "bf_internal.cuh"

namespace cgx = cooperative_groups;

namespace bf {

// ------------------------------------------------------------------------------- pair xform
// Both transforms of every pair, M_ab = T_b^-1 T_a (source a) then M_ba, one thread per entry
// (24 per pair): each entry is a handful of FP64 operations, and spreading them over many warps
// keeps the slow FP64 pipe of each SM sub-partition short.  The per-problem PCG kernel refreshes
// its own pairs' transforms after the pose update; this kernel serves the first linearisation of
// a solve and the multi-CTA PCG variants.
__global__ void k_pair_xform(int n_pairs, const int *__restrict__ pa, const int *__restrict__ pb,
                             const double *__restrict__ pose, float *__restrict__ pairM) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 24 * n_pairs) return;
  const int p = k / 24, e = k % 24;
  const double *Ta = pose + 12 * pa[p];
  const double *Tb = pose + 12 * pb[p];
  pairM[k] = e < 12 ? pair_xform_entry(Ta, Tb, e) : pair_xform_entry(Tb, Ta, e - 12);
}

int launch_pair_xform(const Tables &t, const double *pose, float *pairM, cudaStream_t st) {
  if (t.n_pairs == 0) return 0;
  k_pair_xform<<<(24 * t.n_pairs + 127) / 128, 128, 0, st>>>(t.n_pairs, t.pair_a, t.pair_b, pose, pairM);
  return 1;
}

// ------------------------------------------------------------------------------- pair merge
// Rotated sums of one direction: 0..53 six 3x3 blocks (Saa, Sav, Svv, Sac, Svc, Scc, full
// row-major), 54..62 the vectors ga, gv, gc.
constexpr int NROT = 63;

__device__ __forceinline__ int part_index(int blk, int m, int n) {
  // position of element (m, n) of block blk in the NPART layout
  const int sym = (m == n) ? (m == 0 ? 0 : (m == 1 ? 3 : 5)) : (m + n == 1 ? 1 : (m + n == 2 ? 2 : 4));
  switch (blk) {
    case 0: return P_AA + sym;
    case 1: return P_AV + 3 * m + n;
    case 2: return P_VV + sym;
    case 3: return P_AC + 3 * m + n;
    case 4: return P_VC + 3 * m + n;
    default: return P_CC + sym;
  }
}

// For output slot s of a pair record and a direction whose source is frame a (src_is_a) or b,
// the rotated element feeding it and its sign (0 sign: no contribution).
__device__ __forceinline__ void slot_source(int s, bool src_is_a, int &idx, int &sign) {
  enum { SAA = 0, SAV = 9, SVV = 18, SAC = 27, SVC = 36, SCC = 45, GA = 54, GV = 57, GC = 60 };
  idx = 0;
  sign = 0;
  if (s < 108) {
    const int blk = s / 36, e = s % 36;
    int i = e / 6, j = e % 6;
    int role;  // 0: A_ss, 1: A_tt, 2: A_st, 3: A_st^T
    if (blk == 1) {
      role = src_is_a ? 2 : 3;
    } else {
      const bool is_src = (blk == 0) == src_is_a;
      role = is_src ? 0 : 1;
    }
    if (role == 3) {  // A_ab = A_st^T
      const int tmp = i;
      i = j;
      j = tmp;
      role = 2;
    }
    const bool ui = i < 3, uj = j < 3;
    const int i3 = ui ? i : i - 3, j3 = uj ? j : j - 3;
    if (role == 0) {  // [[Saa, Sav], [Sav^T, Svv]]
      if (ui && uj) { idx = SAA + 3 * i3 + j3; sign = 1; }
      else if (ui) { idx = SAV + 3 * i3 + j3; sign = 1; }
      else if (uj) { idx = SAV + 3 * j3 + i3; sign = 1; }
      else { idx = SVV + 3 * i3 + j3; sign = 1; }
    } else if (role == 1) {  // [[Scc, -Svc^T], [-Svc, Svv]]
      if (ui && uj) { idx = SCC + 3 * i3 + j3; sign = 1; }
      else if (ui) { idx = SVC + 3 * j3 + i3; sign = -1; }
      else if (uj) { idx = SVC + 3 * i3 + j3; sign = -1; }
      else { idx = SVV + 3 * i3 + j3; sign = 1; }
    } else {  // A_st = [[Sac, -Sav], [Svc, -Svv]]
      if (ui && uj) { idx = SAC + 3 * i3 + j3; sign = 1; }
      else if (ui) { idx = SAV + 3 * i3 + j3; sign = -1; }
      else if (uj) { idx = SVC + 3 * i3 + j3; sign = 1; }
      else { idx = SVV + 3 * i3 + j3; sign = -1; }
    }
  } else {
    const int r = s - 108;
    const bool is_a_rhs = r < 6;
    const int c = r % 6;
    const bool is_src = is_a_rhs == src_is_a;
    if (is_src) {  // -(ga, gv)
      idx = c < 3 ? GA + c : GV + c - 3;
      sign = -1;
    } else {  // -(gc, -gv)
      idx = c < 3 ? GC + c : GV + c - 3;
      sign = c < 3 ? -1 : 1;
    }
  }
}

constexpr int MERGE_WARPS = 1;  // one warp per CTA spreads the pairs over the SMs

// One warp per pair.  The pair's record combines up to three sources: the dense direction a -> b
// and the sparse segments (both evaluated in camera-b coordinates, source a), and the dense
// direction b -> a (camera a, source b).  Sources that share a target camera are summed in the
// NPART layout first and rotated to world coordinates once, R X R^T in two 3-FMA stages
// (X R^T, then R (X R^T)); B300 issues FP64 at 1/64 of the FP32 rate, so the merge is bound by
// its FP64 instruction count.
// Shared memory of one merging warp.
template <typename Acc>
struct MergeSmem {
  Acc S[NPART + 7];
  Acc T[54];
  Acc rot[NROT + 1];
  Acc R[9];
};

// Merge of pair p by the calling warp (all 32 lanes).  CG: partials and poses are read through
// L2 (written by other CTAs of a persistent launch).
template <typename Acc, typename Part, bool CG = false>
__device__ __forceinline__ void merge_pair(int p, const Tables &t, const double *__restrict__ pose,
                                           const Part *__restrict__ dpart, const Part *__restrict__ spart,
                                           Acc *__restrict__ pairblk, Acc *__restrict__ pairen,
                                           float *__restrict__ pairoff, MergeSmem<Acc> &sm) {
  const int lane = threadIdx.x & 31;
  Acc *S = sm.S;
  Acc *T = sm.T;
  Acc *rot = sm.rot;
  Acc *R = sm.R;
  Acc out[4] = {0, 0, 0, 0};  // slots lane, lane+32, lane+64, lane+96
  Acc en[4] = {0, 0, 0, 0};   // kept by lane 0: e_sparse, e_photo, e_geo, n_dense
  for (int half = 0; half < 2; ++half) {
    // half 0: target b (dense a -> b and the sparse segments); half 1: target a (dense b -> a)
    const int d = t.pair_dp[2 * p + half];
    const bool has_sparse = spart != nullptr && half == 0 && t.pair_seg1[p] > t.pair_seg0[p];
    if (d < 0 && !has_sparse) continue;
    const int tgt = half == 1 ? t.pair_a[p] : t.pair_b[p];
    const int srcf = half == 1 ? t.pair_b[p] : t.pair_a[p];
    if (lane < 9) R[lane] = (Acc)ldx<CG>(pose + 12 * tgt + lane);
    for (int k = lane; k < NPART; k += 32) S[k] = 0;
    __syncwarp();
    if (d >= 0) {
      // dense: sum the tiles' v / c sums (fixed order), then rebuild the a-sums with
      // a = T v - c, T v = v x t, t = t_ji = R_j^T (t_i - t_j)
      const int k0 = t.dp_tile0[d], k1 = t.dp_tile1[d];
      Acc *Sd = rot;  // scratch for the NPD sums
      for (int k = lane; k < NPD; k += 32) {
        Acc s = 0;
        for (int it = k0; it < k1; ++it) s += (Acc)ldx<CG>(dpart + (long long)it * NPD + k);
        Sd[k] = s;
      }
      __syncwarp();
      Acc tt[3];
      {
        const double *Ti = pose + 12 * srcf, *Tj = pose + 12 * tgt;
        const double d0 = ldx<CG>(Ti + 9) - ldx<CG>(Tj + 9), d1 = ldx<CG>(Ti + 10) - ldx<CG>(Tj + 10),
                     d2 = ldx<CG>(Ti + 11) - ldx<CG>(Tj + 11);
#pragma unroll
        for (int m = 0; m < 3; ++m)
          tt[m] = (Acc)(ldx<CG>(Tj + m) * d0 + ldx<CG>(Tj + 3 + m) * d1 + ldx<CG>(Tj + 6 + m) * d2);
      }
      const Acc T3[3][3] = {{0, tt[2], -tt[1]}, {-tt[2], 0, tt[0]}, {tt[1], -tt[0], 0}};
      for (int k = lane; k < 6; k += 32) {
        S[P_VV + k] = Sd[D_VV + k];
        S[P_CC + k] = Sd[D_CC + k];
      }
      for (int k = lane; k < 9; k += 32) S[P_VC + k] = Sd[D_VC + k];
      if (lane < 3) {
        S[P_GV + lane] = Sd[D_GV + lane];
        S[P_GC + lane] = Sd[D_GC + lane];
      }
      if (lane == 0) {
        en[2] += Sd[D_E0];
        en[1] += Sd[D_E1];
        en[3] += Sd[D_CNT];
      }
      __syncwarp();
      // S_av = T S_vv - S_vc^T ; S_ac = T S_vc - S_cc ; g_a = T g_v - g_c
      if (lane < 9) {
        const int i = lane / 3, j = lane % 3;
        Acc av = -S[P_VC + 3 * j + i], ac = -S[part_index(5, i, j)];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          av += T3[i][k] * S[part_index(2, k, j)];
          ac += T3[i][k] * S[P_VC + 3 * k + j];
        }
        S[P_AV + lane] = av;
        S[P_AC + lane] = ac;
      } else if (lane < 12) {
        const int i = lane - 9;
        S[P_GA + i] = T3[i][0] * S[P_GV] + T3[i][1] * S[P_GV + 1] + T3[i][2] * S[P_GV + 2] - S[P_GC + i];
      }
      __syncwarp();
      // S_aa = S_av T^T - S_ac (symmetric; upper triangle)
      if (lane < 6) {
        const int i = lane < 3 ? 0 : (lane < 5 ? 1 : 2);
        const int j = lane < 3 ? lane : (lane < 5 ? lane - 2 : 2);
        Acc aa = -S[P_AC + 3 * i + j];
#pragma unroll
        for (int k = 0; k < 3; ++k) aa += S[P_AV + 3 * i + k] * T3[j][k];
        S[P_AA + lane] = aa;
      }
      __syncwarp();
    }
    if (has_sparse) {
      // sparse: full NPART sums per segment (fixed order), added to the dense ones
      const int k0 = t.pair_seg0[p], k1 = t.pair_seg1[p];
      for (int k = lane; k < NPART; k += 32) {
        Acc s = 0;
        for (int it = k0; it < k1; ++it) s += (Acc)ldx<CG>(spart + (long long)it * NPART + k);
        if (k == P_E0) S[NPART] = s;  // the sparse energy, read by lane 0 below
        S[k] += s;
      }
      __syncwarp();
      if (lane == 0) en[0] += S[NPART];
    }
    // rotate to world: T_blk = X_blk R^T, then R T_blk; vectors R g
    for (int e = lane; e < 54; e += 32) {
      const int blk = e / 9, m = (e % 9) / 3, j = e % 3;
      T[e] = S[part_index(blk, m, 0)] * R[3 * j] + S[part_index(blk, m, 1)] * R[3 * j + 1] +
             S[part_index(blk, m, 2)] * R[3 * j + 2];
    }
    __syncwarp();
    for (int e = lane; e < NROT; e += 32) {
      Acc v;
      if (e < 54) {
        const int blk = e / 9, i = (e % 9) / 3, j = e % 3;
        v = R[3 * i] * T[9 * blk + j] + R[3 * i + 1] * T[9 * blk + 3 + j] + R[3 * i + 2] * T[9 * blk + 6 + j];
      } else {
        const int vec = (e - 54) / 3, i = (e - 54) % 3;
        const int off = vec == 0 ? P_GA : (vec == 1 ? P_GV : P_GC);
        v = R[3 * i] * S[off] + R[3 * i + 1] * S[off + 1] + R[3 * i + 2] * S[off + 2];
      }
      rot[e] = v;
    }
    __syncwarp();
    const bool src_is_a = half == 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int sl = lane + 32 * q;
      if (sl < PAIRBLK) {
        int idx, sign;
        slot_source(sl, src_is_a, idx, sign);
        if (sign > 0) out[q] += rot[idx];
        else if (sign < 0) out[q] -= rot[idx];
      }
    }
    __syncwarp();
  }
  Acc *o = pairblk + (long long)p * PAIRBLK;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int sl = lane + 32 * q;
    if (sl < PAIRBLK) {
      o[sl] = out[q];
      if (sl >= PB_AB && sl < PB_AB + 36) pairoff[(long long)p * 36 + sl - PB_AB] = (float)out[q];
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < PAIREN; ++k) pairen[(long long)p * PAIREN + k] = en[k];
  }
}

template <typename Acc, typename Part>
__global__ void __launch_bounds__(32 * MERGE_WARPS)
    k_pair_merge(Tables t, const double *__restrict__ pose, const Part *__restrict__ dpart,
                 const Part *__restrict__ spart, Acc *__restrict__ pairblk, Acc *__restrict__ pairen,
                 float *__restrict__ pairoff) {
  __shared__ MergeSmem<Acc> sm[MERGE_WARPS];
  const int w = threadIdx.x >> 5;
  const int p = blockIdx.x * MERGE_WARPS + w;
  if (p >= t.n_pairs) return;  // whole warp exits together
  merge_pair<Acc, Part>(p, t, pose, dpart, spart, pairblk, pairen, pairoff, sm[w]);
}

template <typename Acc, typename Part>
int launch_pair_merge(const Tables &t, const double *pose, const Part *dpart, const Part *spart, Acc *pairblk,
                      Acc *pairen, float *pairoff, cudaStream_t st) {
  if (t.n_pairs == 0) return 0;
  k_pair_merge<Acc, Part><<<(t.n_pairs + MERGE_WARPS - 1) / MERGE_WARPS, 32 * MERGE_WARPS, 0, st>>>(
      t, pose, dpart, spart, pairblk, pairen, pairoff);
  return 1;
}
template int launch_pair_merge<double, double>(const Tables &, const double *, const double *, const double *,
                                               double *, double *, float *, cudaStream_t);
template int launch_pair_merge<float, float>(const Tables &, const double *, const float *, const float *, float *,
                                             float *, float *, cudaStream_t);

// --------------------------------------------------------------------------------- assemble
// Block-Jacobi preconditioner block: the inverse of the 6x6 diagonal block D (FP64 sums) formed
// in FP32.  D is first scaled symmetrically to unit diagonal (Dh = S D S, S = diag(D_ii^-1/2)),
// then Dh = L L^T (Cholesky), Dh^-1 = L^-T L^-1 and D^-1 = S Dh^-1 S.  The preconditioner only
// steers the PCG iterates, and B300 issues FP64 at 1/64 of the FP32 rate: one FP64 Cholesky
// inverse in a single lane costs tens of microseconds there.  Returns false if the block is not
// positive definite.
__device__ bool chol_inverse6(const double *D, float *Mi) {
  float sc[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float d = (float)D[7 * i];
    if (!(d > 0.f)) return false;
    sc[i] = 1.f / sqrtf(d);
  }
  float L[36];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) L[6 * i + j] = j <= i ? (float)D[6 * i + j] * sc[i] * sc[j] : 0.f;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float d = L[7 * j];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > 0.f)) return false;
    const float ljj = sqrtf(d), inv = 1.f / ljj;
    L[7 * j] = ljj;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      float u = L[6 * i + j];
#pragma unroll
      for (int k = 0; k < j; ++k) u -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = u * inv;
    }
  }
  float Li[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) Li[k] = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float inv = 1.f / L[7 * i];
    Li[7 * i] = inv;
#pragma unroll
    for (int j = 0; j < i; ++j) {
      float s = 0.f;
#pragma unroll
      for (int k = j; k < i; ++k) s -= L[6 * i + k] * Li[6 * k + j];
      Li[6 * i + j] = s * inv;
    }
  }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float s = 0.f;
#pragma unroll
      for (int k = (i > j ? i : j); k < 6; ++k) s += Li[6 * k + i] * Li[6 * k + j];
      Mi[6 * i + j] = sc[i] * s * sc[j];
    }
  return true;
}

constexpr int ASM_WARPS = 1;  // one warp per CTA spreads the frames over the SMs

// Shared memory of one assembling warp.
struct AsmSmem {
  double D[36];
  float M[36];
};

// Diagonal block, rhs and preconditioner block of free frame v, by the calling warp.
template <typename Acc>
__device__ __forceinline__ void assemble_var(int v, const Tables &t, const Acc *__restrict__ pairblk, int precond,
                                             Acc *__restrict__ Dd, Acc *__restrict__ rhs, float *__restrict__ Df,
                                             float *__restrict__ Minv, int *__restrict__ vflags, AsmSmem &sm) {
  const int lane = threadIdx.x & 31;
  double *Dshw = sm.D;
  float *Mshw = sm.M;
  const int e0 = t.inc_off[v], e1 = t.inc_off[v + 1];
  // lane handles entries lane and lane + 32 of [D (36) | rhs (6)]; the incidences are read 8 at
  // a time (all loads in flight together) and summed in incidence order
  for (int k = lane; k < 42; k += 32) {
    Acc s = 0;
    for (int e = e0; e < e1; e += 8) {
      Acc v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        v[u] = 0;
        if (e + u < e1) {
          const int ent = t.inc[e + u];
          const int p = ent >> 1, side = ent & 1;
          const Acc *b = pairblk + (long long)p * PAIRBLK;
          v[u] = k < 36 ? b[(side == 0 ? PB_AA : PB_BB) + k] : b[(side == 0 ? PB_RA : PB_RB) + k - 36];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e + u < e1) s += v[u];
    }
    if (k < 36) {
      Dd[(long long)v * 36 + k] = s;
      Df[(long long)v * 36 + k] = (float)s;
      Dshw[k] = (double)s;
    } else {
      rhs[(long long)v * 6 + k - 36] = s;
    }
  }
  __syncwarp();
  if (lane == 0) {
    int flag = 0;
    bool empty = true;
    // integer test for +-0 (an FP64 compare would occupy the slow FP64 pipe 36 times)
    for (int k = 0; k < 36; ++k) empty = empty && ((__double_as_longlong(Dshw[k]) << 1) == 0);
    for (int k = 0; k < 36; ++k) Mshw[k] = 0.f;
    if (empty) {
      flag = 2;  // BF_FLAG_EMPTY_FRAME: zero inverse, the frame's update stays 0
    } else {
      bool ok = false;
      if (precond == 0) {
        ok = chol_inverse6(Dshw, Mshw);
        if (!ok) flag = 1;  // BF_FLAG_SINGULAR_BLOCK: fall back to the diagonal
      }
      if (!ok) {
        for (int k = 0; k < 36; ++k) Mshw[k] = 0.f;
        for (int k = 0; k < 6; ++k) {
          const float d = (float)Dshw[7 * k];
          Mshw[7 * k] = d > 0.f ? 1.f / d : 0.f;
        }
      }
    }
    vflags[v] = flag;
  }
  __syncwarp();
  for (int k = lane; k < 36; k += 32) Minv[(long long)v * 36 + k] = Mshw[k];
}

template <typename Acc>
__global__ void __launch_bounds__(32 * ASM_WARPS)
    k_assemble(Tables t, const Acc *__restrict__ pairblk, int precond, Acc *__restrict__ Dd, Acc *__restrict__ rhs,
               float *__restrict__ Df, float *__restrict__ Minv, int *__restrict__ vflags) {
  __shared__ AsmSmem sm[ASM_WARPS];
  const int w = threadIdx.x >> 5;
  const int v = blockIdx.x * ASM_WARPS + w;
  if (v >= t.n_vars) return;
  assemble_var<Acc>(v, t, pairblk, precond, Dd, rhs, Df, Minv, vflags, sm[w]);
}

template <typename Acc>
int launch_assemble(const Tables &t, const Acc *pairblk, int precond, Acc *Dd, Acc *rhs, float *Df, float *Minv,
                    int *vflags, cudaStream_t st) {
  if (t.n_vars == 0) return 0;
  k_assemble<Acc><<<(t.n_vars + ASM_WARPS - 1) / ASM_WARPS, 32 * ASM_WARPS, 0, st>>>(t, pairblk, precond, Dd, rhs,
                                                                                      Df, Minv, vflags);
  return 1;
}
template int launch_assemble<double>(const Tables &, const double *, int, double *, double *, float *, float *, int *,
                                     cudaStream_t);
template int launch_assemble<float>(const Tables &, const float *, int, float *, float *, float *, float *, int *,
                                    cudaStream_t);

// ------------------------------------------------------------------------- energy reduce
constexpr int EN_BS = 256;

// Energy record of problem `prob`: the sum of its pairs' records, formed by the first EN_BS threads
// of the calling block in a fixed order (strided partial sums, warp butterflies, warps in order),
// so every kernel that calls it produces the same bits.  Every thread of the block must call it.
template <typename Acc>
__device__ void problem_energy(const Tables &t, const Acc *__restrict__ pairen, int prob, double *__restrict__ out,
                               Acc (*sh)[PAIREN]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // warps past the problem's pair count hold zeros: left out (same result, less FP64 work)
  const int np = t.prob_pair1[prob] - t.prob_pair0[prob];
  const int nw = min(EN_BS / 32, (np + 31) / 32);
  if (warp < nw) {
    Acc s[PAIREN] = {0, 0, 0, 0};
    for (int p = t.prob_pair0[prob] + threadIdx.x; p < t.prob_pair1[prob]; p += EN_BS)
#pragma unroll
      for (int k = 0; k < PAIREN; ++k) s[k] += pairen[(long long)p * PAIREN + k];
#pragma unroll
    for (int k = 0; k < PAIREN; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
      if (lane == 0) sh[warp][k] = s[k];
    }
  }
  __syncthreads();
  if (threadIdx.x < PAIREN) {
    Acc v = 0;
    for (int w = 0; w < nw; ++w) v += sh[w][threadIdx.x];
    out[prob * PAIREN + threadIdx.x] = (double)v;
  }
  __syncthreads();
}

template <typename Acc>
__global__ void __launch_bounds__(EN_BS) k_energy_reduce(Tables t, const Acc *__restrict__ pairen,
                                                         double *__restrict__ out) {
  __shared__ Acc sh[EN_BS / 32][PAIREN];
  problem_energy<Acc>(t, pairen, blockIdx.x, out, sh);
}

template <typename Acc>
int launch_energy_reduce(const Tables &t, const Acc *pairen, double *out, cudaStream_t st) {
  if (t.n_prob == 0) return 0;
  k_energy_reduce<Acc><<<t.n_prob, EN_BS, 0, st>>>(t, pairen, out);
  return 1;
}
template int launch_energy_reduce<double>(const Tables &, const double *, double *, cudaStream_t);
template int launch_energy_reduce<float>(const Tables &, const float *, double *, cudaStream_t);

// ------------------------------------------------------------------------ PCG, one CTA/problem
constexpr int PCG_BS = 256;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum, valid in thread 0 only: FP32 warp trees, then the warps' sums in Acc in
// warp order.  The scalar recurrences (alpha, beta, the stop test) run in thread 0 alone and reach
// the block through shared memory: B300 issues FP64 at 1/64 of the FP32 rate, so FP64 work
// repeated by every thread would dominate the iteration.  The caller synchronises before wsum is
// written again.
// Warps at or beyond nw hold only zeros and are left out of the sum (the result is the same).
template <typename Acc, int BS>
__device__ __forceinline__ Acc block_sum0(float v, float *wsum, int nw = BS / 32) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  Acc s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) s += (Acc)wsum[w];
  return s;
}

// Scalars thread 0 hands to the block each half-iteration.
struct PcgScal {
  float fa, fb;
  int stop;
};

// z_v = Minv_v r_v for the row u = 6 v + c
__device__ __forceinline__ float precond_row(const float *__restrict__ Minv, const float *__restrict__ r, int v,
                                             int c) {
  const float *Mr = Minv + (long long)v * 36 + 6 * c;
  const float *rv = r + 6LL * v;
  return Mr[0] * rv[0] + Mr[1] * rv[1] + Mr[2] * rv[2] + Mr[3] * rv[3] + Mr[4] * rv[4] + Mr[5] * rv[5];
}

// Thread 0, after p.Ap: stop on breakdown, else alpha = rz / pq.  Returns the flag bits to add.
// alpha and beta feed FP32 vector updates, so they are FP32 quotients of the rounded sums (within
// 1.5 ulp of the rounded FP64 quotient; an FP64 division is a long FP64 instruction sequence).
template <typename Acc>
__device__ __forceinline__ int pcg_alpha(Acc rz, Acc pq, PcgScal &S) {
  if (!(pq > (Acc)0)) {
    S.stop = 1;
    return 4;  // BF_FLAG_PCG_BREAKDOWN
  }
  S.fa = __fdiv_rn((float)rz, (float)pq);
  return 0;
}

// Thread 0, after r.z: beta = rz_new / rz, stop once r.z reaches zero.
template <typename Acc>
__device__ __forceinline__ void pcg_beta(Acc &rz, Acc rz_new, PcgScal &S) {
  S.fb = __fdiv_rn((float)rz_new, (float)rz);
  rz = rz_new;
  S.stop = rz == (Acc)0;
}

// Matrix-free sparse product of one pair (Sec. 4.4: J p, then J^T (J p), the sparse residuals
// never assembled).  Correspondence k of the pair (a, b) has the world-frame residual
// r_k = T_a p_k - T_b q_k with Jacobian [-[P]x, I, [Q]x, -I] over (dw_a, dt_a, dw_b, dt_b),
// P = R_a p_k, Q = R_b q_k (rotations of the linearisation point).  For the direction d:
//   y_k = w_sparse w_k (dw_a x P + dt_a - dw_b x Q - dt_b)          (J p, three rows)
//   J^T y_k = (P x y_k, y_k) for frame a, (-(Q x y_k), -y_k) for frame b.
// The calling warp walks the pair's segments with lane-strided correspondences; the 12 sums
// (frame a's six, then frame b's) reach every lane through a butterfly.  da / db are the two
// frames' direction blocks (zero for a gauge frame).
__device__ void mf_pair(const Tables &t, const MatFree &mf, int pr, const float (&da)[6], const float (&db)[6],
                        float (&out)[12]) {
  const int lane = threadIdx.x & 31;
  const double *Ta = mf.pose + 12 * t.pair_a[pr], *Tb = mf.pose + 12 * t.pair_b[pr];
  float Ra[9], Rb[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Ra[k] = (float)Ta[k];
    Rb[k] = (float)Tb[k];
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = 0.f;
  for (int s = t.pair_seg0[pr]; s < t.pair_seg1[pr]; ++s) {
    const int off = t.seg_off[s], cnt = t.seg_cnt[s];
    const bool swap = t.seg_swap[s] != 0;
    for (int k = lane; k < cnt; k += 32) {
      const float4 u = mf.P[off + k], v = mf.Q[off + k];
      const float px = swap ? v.x : u.x, py = swap ? v.y : u.y, pz = swap ? v.z : u.z;
      const float qx = swap ? u.x : v.x, qy = swap ? u.y : v.y, qz = swap ? u.z : v.z;
      const float w = mf.w_sparse * u.w;
      const float P0 = Ra[0] * px + Ra[1] * py + Ra[2] * pz;
      const float P1 = Ra[3] * px + Ra[4] * py + Ra[5] * pz;
      const float P2 = Ra[6] * px + Ra[7] * py + Ra[8] * pz;
      const float Q0 = Rb[0] * qx + Rb[1] * qy + Rb[2] * qz;
      const float Q1 = Rb[3] * qx + Rb[4] * qy + Rb[5] * qz;
      const float Q2 = Rb[6] * qx + Rb[7] * qy + Rb[8] * qz;
      const float y0 = w * ((da[1] * P2 - da[2] * P1) + da[3] - (db[1] * Q2 - db[2] * Q1) - db[3]);
      const float y1 = w * ((da[2] * P0 - da[0] * P2) + da[4] - (db[2] * Q0 - db[0] * Q2) - db[4]);
      const float y2 = w * ((da[0] * P1 - da[1] * P0) + da[5] - (db[0] * Q1 - db[1] * Q0) - db[5]);
      out[0] += P1 * y2 - P2 * y1;
      out[1] += P2 * y0 - P0 * y2;
      out[2] += P0 * y1 - P1 * y0;
      out[3] += y0;
      out[4] += y1;
      out[5] += y2;
      out[6] -= Q1 * y2 - Q2 * y1;
      out[7] -= Q2 * y0 - Q0 * y2;
      out[8] -= Q0 * y1 - Q1 * y0;
      out[9] -= y0;
      out[10] -= y1;
      out[11] -= y2;
    }
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = warp_sum(out[k]);
}

// Problems with at most PCG_SMALL_N unknowns (16 free frames) are solved from a dense copy of
// their system in shared memory, one thread per unknown with its x, r, z, p in registers: no
// global-memory round trip inside the iteration.  The choice depends on the problem alone, so a
// problem solved in a batch gives the same bits as solved alone.
constexpr int PCG_SMALL_N = 96;

template <typename Acc>
__device__ int pcg_small(const Tables &t, const float *__restrict__ Df, const float *__restrict__ pairoff,
                         const float *__restrict__ Minv, const Acc *__restrict__ rhs, float *__restrict__ x,
                         int n_pcg, int v0, int v1, float *wsum, PcgScal &S, float *AT, float *sp, float *sr) {
  // AT: column-major dense system, AT[k * n + u] = A[u][k]; sp, sr: p and r of the iteration
  const int n = 6 * (v1 - v0);
  const int u = threadIdx.x;
  const bool own = u < n;
  for (int k = u; k < n * n; k += PCG_BS) AT[k] = 0.f;
  __syncthreads();
  float Mr[6] = {0, 0, 0, 0, 0, 0};
  float xu = 0.f, ru = 0.f, zu = 0.f, pu = 0.f;
  const int lv = u / 6, c = u % 6;
  if (own) {
    const int v = v0 + lv;
    const float *Dr = Df + (long long)v * 36 + 6 * c;
#pragma unroll
    for (int j = 0; j < 6; ++j) AT[(6 * lv + j) * n + u] = Dr[j];
    for (int e = t.inc_off[v]; e < t.inc_off[v + 1]; ++e) {
      const int ov = t.inc_ov[e];
      if (ov < 0) continue;
      const int ent = t.inc[e];
      const float *O = pairoff + (long long)(ent >> 1) * 36;
      float *col = AT + 6 * (ov - v0) * n + u;
      if ((ent & 1) == 0) {  // row c of A_ab
#pragma unroll
        for (int j = 0; j < 6; ++j) col[j * n] += O[6 * c + j];
      } else {  // row c of A_ba = A_ab^T
#pragma unroll
        for (int j = 0; j < 6; ++j) col[j * n] += O[6 * j + c];
      }
    }
    const float *M = Minv + (long long)v * 36 + 6 * c;
#pragma unroll
    for (int j = 0; j < 6; ++j) Mr[j] = M[j];
    ru = (float)rhs[6 * v0 + u];
    sr[u] = ru;
  }
  __syncthreads();
  if (own) {
    const float *rv = sr + 6 * lv;
    zu = Mr[0] * rv[0] + Mr[1] * rv[1] + Mr[2] * rv[2] + Mr[3] * rv[3] + Mr[4] * rv[4] + Mr[5] * rv[5];
    pu = zu;
    sp[u] = pu;
  }
  const int nw = (n + 31) / 32;  // warps holding unknowns
  Acc rz = block_sum0<Acc, PCG_BS>(own ? ru * zu : 0.f, wsum, nw);
  if (u == 0) S.stop = rz == (Acc)0;
  int flag = 0;
  __syncthreads();
  for (int it = 0; it < n_pcg; ++it) {
    if (S.stop) break;
    float qu = 0.f;
    if (own)
      for (int k = 0; k < n; ++k) qu += AT[k * n + u] * sp[k];
    const Acc pq = block_sum0<Acc, PCG_BS>(own ? pu * qu : 0.f, wsum, nw);
    if (u == 0) flag |= pcg_alpha(rz, pq, S);
    __syncthreads();
    if (S.stop) break;
    const float fa = S.fa;
    if (own) {
      xu += fa * pu;
      ru -= fa * qu;
      sr[u] = ru;
    }
    __syncthreads();
    if (own) {
      const float *rv = sr + 6 * lv;
      zu = Mr[0] * rv[0] + Mr[1] * rv[1] + Mr[2] * rv[2] + Mr[3] * rv[3] + Mr[4] * rv[4] + Mr[5] * rv[5];
    }
    const Acc rz_new = block_sum0<Acc, PCG_BS>(own ? ru * zu : 0.f, wsum, nw);
    if (u == 0) pcg_beta(rz, rz_new, S);
    __syncthreads();
    if (own) {
      pu = zu + S.fb * pu;
      sp[u] = pu;
    }
    __syncthreads();
  }
  if (own) x[6 * v0 + u] = xu;
  return flag;
}

// After the solve: pose update of the problem's free frames, then its pairs' transforms at the
// new poses (both need the whole block's x, respectively poses, written first).
template <bool CG = false>
__device__ void pcg_finish(const Tables &t, const float *x, int prob, int v0, int v1, const PcgOut &po) {
  __syncthreads();
  if (!po.pose) return;
  for (int v = v0 + threadIdx.x; v < v1; v += PCG_BS) update_pose<CG>(po.pose + 12 * t.var_frame[v], x + 6 * v);
  if (!po.pairM) return;
  __syncthreads();
  // one thread per transform entry (24 per pair): the FP64 work spreads over all warps
  const int p0 = t.prob_pair0[prob], n = 24 * (t.prob_pair1[prob] - p0);
  for (int k = threadIdx.x; k < n; k += PCG_BS) {
    const int p = p0 + k / 24, e = k % 24;
    const double *Ta = po.pose + 12 * t.pair_a[p];
    const double *Tb = po.pose + 12 * t.pair_b[p];
    po.pairM[24 * p + e] = e < 12 ? pair_xform_entry(Ta, Tb, e) : pair_xform_entry(Tb, Ta, e - 12);
  }
}

// Shared memory of one problem's PCG.
template <typename Acc>
struct PcgSmem {
  float AT[PCG_SMALL_N * PCG_SMALL_N];
  float sp[PCG_SMALL_N], sr[PCG_SMALL_N];
  float wsum[PCG_BS / 32];
  PcgScal S;
  Acc esh[EN_BS / 32][PAIREN];
};

// The PCG of problem `prob` by a CTA of PCG_BS threads: energy record, exactly n_pcg iterations
// (shared-memory dense path for small problems), pose update and pair transforms.  CG: the poses
// are read through L2 (written by other CTAs of a persistent launch).
template <typename Acc, bool CG = false>
__device__ void pcg_problem(int prob, const Tables &t, const float *__restrict__ Df,
                            const float *__restrict__ pairoff, const float *__restrict__ Minv,
                            const Acc *__restrict__ rhs, float *__restrict__ x, float *__restrict__ r,
                            float *__restrict__ z, float *__restrict__ p, float *__restrict__ q, int n_pcg,
                            int *__restrict__ pflags, const Acc *__restrict__ pairen, const PcgOut &po,
                            const MatFree &mf, PcgSmem<Acc> &sm) {
  float *wsum = sm.wsum;
  PcgScal &S = sm.S;
  if (po.energy) problem_energy<Acc>(t, pairen, prob, po.energy, sm.esh);
  const int v0 = t.prob_var0[prob], v1 = t.prob_var1[prob];
  const int u0 = 6 * v0, u1 = 6 * v1;
  if (u1 - u0 <= PCG_SMALL_N && !mf.P) {
    const int flag = pcg_small<Acc>(t, Df, pairoff, Minv, rhs, x, n_pcg, v0, v1, wsum, S, sm.AT, sm.sp, sm.sr);
    if (threadIdx.x == 0 && pflags) pflags[prob] |= flag;
    pcg_finish<CG>(t, x, prob, v0, v1, po);
    return;
  }
  for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
    x[u] = 0.f;
    r[u] = (float)rhs[u];
  }
  __syncthreads();
  float loc = 0.f;
  for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
    const float zu = precond_row(Minv, r, u / 6, u % 6);
    z[u] = zu;
    p[u] = zu;
    loc += r[u] * zu;
  }
  Acc rz = block_sum0<Acc, PCG_BS>(loc, wsum);
  if (threadIdx.x == 0) S.stop = rz == (Acc)0;
  int flag = 0;
  __syncthreads();
  for (int it = 0; it < n_pcg; ++it) {
    if (S.stop) break;
    if (mf.P) {
      // matrix-free sparse term: every pair's J^T W J p (warps over the problem's pairs), added
      // below by the pair's two frames
      const int lane = threadIdx.x & 31;
      for (int pr = t.prob_pair0[prob] + (threadIdx.x >> 5); pr < t.prob_pair1[prob]; pr += PCG_BS / 32) {
        float da[6], db[6], y[12];
        const int va = t.frame_var[t.pair_a[pr]], vb = t.frame_var[t.pair_b[pr]];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          da[k] = va >= 0 ? p[6 * va + k] : 0.f;
          db[k] = vb >= 0 ? p[6 * vb + k] : 0.f;
        }
        mf_pair(t, mf, pr, da, db, y);
#pragma unroll
        for (int k = 0; k < 12; ++k)
          if (lane == k) mf.mfy[12 * pr + k] = y[k];
      }
      __syncthreads();
    }
    loc = 0.f;
    for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
      const int v = u / 6, c = u % 6;
      const float *Drow = Df + (long long)v * 36 + 6 * c;
      const float *pv = p + 6LL * v;
      float s = Drow[0] * pv[0] + Drow[1] * pv[1] + Drow[2] * pv[2] + Drow[3] * pv[3] + Drow[4] * pv[4] +
                Drow[5] * pv[5];
      for (int e = t.inc_off[v]; e < t.inc_off[v + 1]; ++e) {
        const int ov = t.inc_ov[e];
        if (mf.P) s += mf.mfy[12 * (t.inc[e] >> 1) + 6 * (t.inc[e] & 1) + c];
        if (ov < 0) continue;
        const int ent = t.inc[e];
        const int pr = ent >> 1, side = ent & 1;
        const float *O = pairoff + (long long)pr * 36;
        const float *pw = p + 6LL * ov;
        if (side == 0) {  // row of A_ab
          s += O[6 * c] * pw[0] + O[6 * c + 1] * pw[1] + O[6 * c + 2] * pw[2] + O[6 * c + 3] * pw[3] +
               O[6 * c + 4] * pw[4] + O[6 * c + 5] * pw[5];
        } else {  // row of A_ba = A_ab^T
          s += O[c] * pw[0] + O[6 + c] * pw[1] + O[12 + c] * pw[2] + O[18 + c] * pw[3] + O[24 + c] * pw[4] +
               O[30 + c] * pw[5];
        }
      }
      q[u] = s;
      loc += p[u] * s;
    }
    const Acc pq = block_sum0<Acc, PCG_BS>(loc, wsum);
    if (threadIdx.x == 0) flag |= pcg_alpha(rz, pq, S);
    __syncthreads();
    if (S.stop) break;
    const float fa = S.fa;
    for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
      x[u] += fa * p[u];
      r[u] -= fa * q[u];
    }
    __syncthreads();
    loc = 0.f;
    for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
      const float zu = precond_row(Minv, r, u / 6, u % 6);
      z[u] = zu;
      loc += r[u] * zu;
    }
    const Acc rz_new = block_sum0<Acc, PCG_BS>(loc, wsum);
    if (threadIdx.x == 0) pcg_beta(rz, rz_new, S);
    __syncthreads();
    const float fb = S.fb;
    for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) p[u] = z[u] + fb * p[u];
    __syncthreads();
  }
  if (threadIdx.x == 0 && pflags) pflags[prob] |= flag;
  pcg_finish<CG>(t, x, prob, v0, v1, po);
}

template <typename Acc>
__global__ void __launch_bounds__(PCG_BS)
    k_pcg(Tables t, const float *__restrict__ Df, const float *__restrict__ pairoff, const float *__restrict__ Minv,
          const Acc *__restrict__ rhs, float *__restrict__ x, float *__restrict__ r, float *__restrict__ z,
          float *__restrict__ p, float *__restrict__ q, int n_pcg, int *__restrict__ pflags,
          const Acc *__restrict__ pairen, PcgOut po, MatFree mf) {
  __shared__ PcgSmem<Acc> sm;
  pcg_problem<Acc>(blockIdx.x, t, Df, pairoff, Minv, rhs, x, r, z, p, q, n_pcg, pflags, pairen, po, mf, sm);
}

template <typename Acc>
int launch_pcg(const Tables &t, const float *Df, const float *pairoff, const float *Minv, const Acc *rhs, float *x,
               float *r, float *z, float *p, float *q, int n_pcg, int *pflags, const Acc *pairen, PcgOut po,
               const MatFree &mf, cudaStream_t st) {
  if (t.n_prob == 0) return 0;
  k_pcg<Acc><<<t.n_prob, PCG_BS, 0, st>>>(t, Df, pairoff, Minv, rhs, x, r, z, p, q, n_pcg, pflags, pairen, po, mf);
  return 1;
}
template int launch_pcg<double>(const Tables &, const float *, const float *, const float *, const double *, float *,
                                float *, float *, float *, float *, int, int *, const double *, PcgOut,
                                const MatFree &, cudaStream_t);
template int launch_pcg<float>(const Tables &, const float *, const float *, const float *, const float *, float *,
                               float *, float *, float *, float *, int, int *, const float *, PcgOut, const MatFree &,
                               cudaStream_t);

// ------------------------------------------------------------- PCG, one problem over the grid
constexpr int COOP_BS = 256;
constexpr int COOP_WARPS = COOP_BS / 32;
// Spin limit of the grid barrier: 2^24 polls, the first 2^12 without back-off, the rest with a
// 64 ns back-off: about a second in all.
constexpr long long BARRIER_SPIN_LIMIT = 1LL << 24;
constexpr long long BARRIER_SPIN_FAST = 1LL << 12;

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  count/gen live in global
// memory and start at 0.  A CTA whose wait exceeds the spin limit sets *err and returns false;
// a CTA that sees *err set while waiting returns false too, so no CTA waits forever.
__device__ bool grid_barrier(unsigned *count, volatile unsigned *gen, unsigned nblocks, volatile int *err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd((unsigned *)gen, 1u);
    } else if (!wait_change(gen, g, err, BARRIER_SPIN_LIMIT, BARRIER_SPIN_FAST)) {
      *err = 1;  // timed out here, or another CTA already gave up
      ok = 0;
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

struct CoopState {
  unsigned *count;
  unsigned *gen;
  int *err;
  void *part_pq;  // [gridDim.x] Acc
  void *part_rz;  // [gridDim.x] Acc
};

// Sum of the per-CTA partials in a fixed order: lane l sums entries l, l+32, ... then a
// butterfly over the warp; called by warp 0 of each CTA, every such warp gets the same value.
template <typename Acc>
__device__ __forceinline__ Acc grid_total(const Acc *part, int n) {
  const int lane = threadIdx.x & 31;
  Acc s = 0;
  for (int k = lane; k < n; k += 32) s += __ldcg(part + k);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// This CTA's partial of a dot product into part[blockIdx.x]: FP32 warp trees, the warps' sums in
// Acc in warp order (thread 0).
template <typename Acc>
__device__ __forceinline__ void cta_partial(float v, float *wsum, Acc *part) {
  const Acc s = block_sum0<Acc, COOP_BS>(v, wsum);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename Acc>
__global__ void __launch_bounds__(COOP_BS)
    k_pcg_coop(Tables t, const float *__restrict__ Df, const float *__restrict__ pairoff,
               const float *__restrict__ Minv, const Acc *__restrict__ rhs, float *x, float *r, float *z, float *p0,
               float *p1, float *q, int n_pcg, int *__restrict__ pflags, CoopState cs,
               const Acc *__restrict__ pairen, PcgOut po, MatFree mf) {
  __shared__ float wsum[COOP_WARPS];
  __shared__ PcgScal S;
  __shared__ Acc esh[EN_BS / 32][PAIREN];
  if (blockIdx.x == 0 && po.energy) problem_energy<Acc>(t, pairen, 0, po.energy, esh);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * COOP_WARPS + warp, nw = gridDim.x * COOP_WARPS;
  const int v0 = t.prob_var0[0], v1 = t.prob_var1[0];
  Acc *ppq = (Acc *)cs.part_pq, *prz = (Acc *)cs.part_rz;
  volatile int *err = cs.err;
  // init: x = 0, r = b, z = M^-1 r, p_old = 0 (the first direction is z)
  float loc = 0.f;
  for (int v = v0 + gw; v < v1; v += nw) {
    if (lane < 6) {
      float rr[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) rr[k] = (float)rhs[6 * v + k];
      const float *M = Minv + (long long)v * 36 + 6 * lane;
      const float zl = M[0] * rr[0] + M[1] * rr[1] + M[2] * rr[2] + M[3] * rr[3] + M[4] * rr[4] + M[5] * rr[5];
      x[6 * v + lane] = 0.f;
      r[6 * v + lane] = rr[lane];
      z[6 * v + lane] = zl;
      p0[6 * v + lane] = 0.f;
      loc += rr[lane] * zl;
    }
  }
  cta_partial<Acc>(loc, wsum, prz);
  if (!grid_barrier(cs.count, cs.gen, gridDim.x, err)) return;
  Acc rz = 0;  // meaningful in thread 0
  if (warp == 0) {
    const Acc tot = grid_total(prz, gridDim.x);
    if (lane == 0) {
      rz = tot;
      S.stop = rz == (Acc)0;
      S.fb = 0.f;
    }
  }
  __syncthreads();
  int flag = 0;
  float *pold = p0, *pnew = p1;
  for (int it = 0; it < n_pcg; ++it) {
    if (S.stop) break;
    // Phase A: p_new = z + beta p_old (own frames); q = A p_new with the neighbours' p_new formed
    // on the fly from z and p_old (both final since the last barrier)
    const float fb = S.fb;
    if (mf.P) {
      // Phase A0 (matrix-free sparse term): every pair's J^T W J p_new, p_new of both frames formed
      // on the fly like the neighbours' below; the frames add their pairs' shares in phase A
      for (int pr = gw; pr < t.n_pairs; pr += nw) {
        float da[6], db[6], y[12];
        const int va = t.frame_var[t.pair_a[pr]], vb = t.frame_var[t.pair_b[pr]];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          da[k] = va >= 0 ? __ldcg(z + 6 * va + k) + fb * __ldcg(pold + 6 * va + k) : 0.f;
          db[k] = vb >= 0 ? __ldcg(z + 6 * vb + k) + fb * __ldcg(pold + 6 * vb + k) : 0.f;
        }
        mf_pair(t, mf, pr, da, db, y);
#pragma unroll
        for (int k = 0; k < 12; ++k)
          if (lane == k) mf.mfy[12 * pr + k] = y[k];
      }
      if (!grid_barrier(cs.count, cs.gen, gridDim.x, err)) return;
    }
    float lpq = 0.f;
    for (int v = v0 + gw; v < v1; v += nw) {
      float pn[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) pn[k] = __ldcg(z + 6 * v + k) + fb * __ldcg(pold + 6 * v + k);
      float acc[6] = {0, 0, 0, 0, 0, 0};
      for (int e = t.inc_off[v] + lane; e < t.inc_off[v + 1]; e += 32) {
        const int ov = t.inc_ov[e];
        if (mf.P) {
          const float *y = mf.mfy + 12 * (t.inc[e] >> 1) + 6 * (t.inc[e] & 1);
#pragma unroll
          for (int c = 0; c < 6; ++c) acc[c] += __ldcg(y + c);
        }
        if (ov < 0) continue;
        const int ent = t.inc[e];
        const int pr = ent >> 1, side = ent & 1;
        float pw[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) pw[k] = __ldcg(z + 6 * ov + k) + fb * __ldcg(pold + 6 * ov + k);
        const float *O = pairoff + (long long)pr * 36;
        if (side == 0) {
#pragma unroll
          for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[c] += O[6 * c + k] * pw[k];
        } else {
#pragma unroll
          for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[c] += O[6 * k + c] * pw[k];
        }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) acc[c] = warp_sum(acc[c]);
      float qmine = 0.f, pmine = 0.f;
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const float *Drow = Df + (long long)v * 36 + 6 * c;
        if (lane == c) {
          qmine = acc[c] + Drow[0] * pn[0] + Drow[1] * pn[1] + Drow[2] * pn[2] + Drow[3] * pn[3] +
                  Drow[4] * pn[4] + Drow[5] * pn[5];
          pmine = pn[c];
        }
      }
      if (lane < 6) {
        q[6 * v + lane] = qmine;
        pnew[6 * v + lane] = pmine;
        lpq += pmine * qmine;
      }
    }
    cta_partial<Acc>(lpq, wsum, ppq);
    if (!grid_barrier(cs.count, cs.gen, gridDim.x, err)) return;
    if (warp == 0) {
      const Acc pq = grid_total(ppq, gridDim.x);
      if (lane == 0) flag |= pcg_alpha(rz, pq, S);
    }
    __syncthreads();
    if (S.stop) break;
    const float fa = S.fa;
    // Phase B: x += alpha p_new, r -= alpha q, z = M^-1 r (own frames only, written by this warp)
    float lrz = 0.f;
    for (int v = v0 + gw; v < v1; v += nw) {
      const float rn_own = lane < 6 ? r[6 * v + lane] - fa * q[6 * v + lane] : 0.f;
      float rn[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) rn[k] = __shfl_sync(0xffffffffu, rn_own, k);
      if (lane < 6) {
        const float *M = Minv + (long long)v * 36 + 6 * lane;
        const float zl = M[0] * rn[0] + M[1] * rn[1] + M[2] * rn[2] + M[3] * rn[3] + M[4] * rn[4] + M[5] * rn[5];
        x[6 * v + lane] += fa * pnew[6 * v + lane];
        r[6 * v + lane] = rn_own;
        z[6 * v + lane] = zl;
        lrz += rn_own * zl;
      }
    }
    cta_partial<Acc>(lrz, wsum, prz);
    if (!grid_barrier(cs.count, cs.gen, gridDim.x, err)) return;
    if (warp == 0) {
      const Acc rz_new = grid_total(prz, gridDim.x);
      if (lane == 0) pcg_beta(rz, rz_new, S);
    }
    __syncthreads();
    float *tmp = pold;
    pold = pnew;
    pnew = tmp;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && pflags) pflags[0] |= flag;
  // a frame's step was written by lanes 0..5 of the warp that owns it
  if (po.pose)
    for (int v = v0 + gw; v < v1; v += nw) {
      __syncwarp();
      if (lane == 0) update_pose(po.pose + 12 * t.var_frame[v], x + 6 * v);
    }
}

int coop_max_grid() {
  static int max_blocks = -1;
  if (max_blocks < 0) {
    int dev = 0, sms = 0, per_sm = 0, per_sm_f = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_coop<double>, COOP_BS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, k_pcg_coop<float>, COOP_BS, 0);
    per_sm = per_sm < per_sm_f ? per_sm : per_sm_f;
    max_blocks = sms * (per_sm < 1 ? 1 : per_sm);
  }
  return max_blocks;
}

int coop_grid_size(int n_vars) {
  const int mx = coop_max_grid();
  int want = (n_vars + COOP_WARPS - 1) / COOP_WARPS;
  if (want < 1) want = 1;
  return want < mx ? want : mx;
}

size_t coop_mem_bytes(int grid) { return 256 + 2 * 8 * (size_t)grid; }

template <typename Acc>
int launch_pcg_coop(const Tables &t, const float *Df, const float *pairoff, const float *Minv, const Acc *rhs,
                    float *x, float *r, float *z, float *p0, float *p1, float *q, int n_pcg, int *pflags,
                    void *coop_mem, int grid, const Acc *pairen, PcgOut po, const MatFree &mf,
                    cudaStream_t st) {
  if (t.n_vars == 0) return 0;
  CoopState cs;
  char *m = (char *)coop_mem;
  cs.count = (unsigned *)m;
  cs.gen = (unsigned *)(m + 4);
  cs.err = (int *)(m + 8);
  cs.part_pq = m + 256;
  cs.part_rz = m + 256 + 8 * (size_t)grid;
  if (cudaMemsetAsync(m, 0, 16, st) != cudaSuccess) return -1;
  Tables tt = t;
  MatFree mff = mf;
  void *args[] = {&tt, &Df, &pairoff, &Minv, &rhs, &x, &r, &z, &p0, &p1, &q, &n_pcg, &pflags, &cs, &pairen, &po, &mff};
  if (cudaLaunchCooperativeKernel((const void *)k_pcg_coop<Acc>, dim3(grid), dim3(COOP_BS), args, 0, st) !=
      cudaSuccess)
    return -1;
  return 1;
}
template int launch_pcg_coop<double>(const Tables &, const float *, const float *, const float *, const double *,
                                     float *, float *, float *, float *, float *, float *, int, int *, void *, int,
                                     const double *, PcgOut, const MatFree &, cudaStream_t);
template int launch_pcg_coop<float>(const Tables &, const float *, const float *, const float *, const float *,
                                    float *, float *, float *, float *, float *, float *, int, int *, void *, int,
                                    const float *, PcgOut, const MatFree &, cudaStream_t);

// ------------------------------------------------------ PCG, one problem on a thread-block cluster
// One cluster of CL CTAs (up to 16, one per SM) solves one problem.  Every CTA keeps replicas of
// the full z and p vectors in its shared memory; a CTA owns a contiguous range of frames and
// broadcasts its frames' new z and p into every replica through distributed shared memory.
// Two hardware cluster barriers per iteration separate the phases, and the per-CTA dot-product
// partials are read from the other CTAs' shared memory and summed in rank order.
constexpr int CL_BS = 512;
constexpr int CL_WARPS = CL_BS / 32;
constexpr int CL_G = 16;  // lanes per frame in the matvec

// Sum of the CL per-CTA partials (slot k of each CTA's part array), read lane-parallel from the
// cluster's shared memory and combined by a butterfly: identical in every lane of every CTA.
template <typename Acc>
__device__ __forceinline__ Acc cluster_total(cgx::cluster_group &cluster, Acc *part, int k, int CL) {
  const int lane = threadIdx.x & 31;
  Acc s = lane < CL ? cluster.map_shared_rank(part, lane)[k] : (Acc)0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Fixed-order CTA sum of one FP32 value per warp (lane 0 holds it) into part[k]: a butterfly
// over the CL_WARPS values in warp 0 (FP32), then one conversion; FP64 starts at the sum over
// the cluster's CTAs.
template <typename Acc>
__device__ __forceinline__ void cluster_partial(float v, float *wsum, Acc *part, int k) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    float s = lane < CL_WARPS ? wsum[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[k] = (Acc)s;
  }
}

// Shared-memory layout of one CTA (floats unless noted), per = frames owned per CTA:
//   zp[per][12]              owned frames' z and p (interleaved: 3 float4 per frame); the other
//                            CTAs read them remotely through distributed shared memory
//   ox, orr, oq, opn [6 per] owned frames' x, r, q, p_new
//   part (2 Acc)             pq, rz partials
//   cache (optional):  sD[per][36] sM[per][36] sB[n_inc][36] sov[n_inc] (int: owner << 16 | index)
//     sB = the pair's off-diagonal block as seen from the owned frame (A_ab, or A_ab^T)
struct ClusterLayout {
  int per, max_inc;
  bool cache;
};

__host__ __device__ inline size_t cluster_bytes(int n_vars, int per, int max_inc, bool cache) {
  (void)n_vars;
  size_t b = (size_t)per * 12 * 4 + 4 * 6 * (size_t)per * 4;
  b = (b + 15) & ~(size_t)15;
  b += 2 * sizeof(double);
  if (cache) b += (size_t)per * 72 * 4 + (size_t)max_inc * 37 * 4;
  return b + 16;
}

template <typename Acc>
__global__ void __launch_bounds__(CL_BS, 1)
    k_pcg_cluster(Tables t, const float *__restrict__ Df, const float *__restrict__ pairoff,
                  const float *__restrict__ Minv, const Acc *__restrict__ rhs, float *__restrict__ xg, int n_pcg,
                  int *__restrict__ pflags, ClusterLayout L, const Acc *__restrict__ pairen, PcgOut po) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ const float4 *zp_rank[16];
  __shared__ Acc esh[CL_WARPS][PAIREN];
  __shared__ Acc eslice[PAIREN];
  cgx::cluster_group cluster = cgx::this_cluster();
  const int rank = (int)cluster.block_rank(), CL = (int)cluster.num_blocks();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (po.energy) {
    // this CTA's slice of the energy record: its share of the pairs, strided over threads, warp
    // trees, warps in order; rank 0 adds the slices in rank order after the first barrier
    const int p0 = t.prob_pair0[0], np = t.prob_pair1[0] - p0, chunk = (np + CL - 1) / CL;
    const int pa = p0 + min(np, rank * chunk), pb = p0 + min(np, (rank + 1) * chunk);
    Acc es[PAIREN] = {0, 0, 0, 0};
    for (int q = pa + threadIdx.x; q < pb; q += CL_BS)
#pragma unroll
      for (int c = 0; c < PAIREN; ++c) es[c] += pairen[(long long)q * PAIREN + c];
#pragma unroll
    for (int c = 0; c < PAIREN; ++c) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) es[c] += __shfl_xor_sync(0xffffffffu, es[c], o);
      if (lane == 0) esh[warp][c] = es[c];
    }
    __syncthreads();
    if (threadIdx.x < PAIREN) {
      Acc v = 0;
      for (int w = 0; w < CL_WARPS; ++w) v += esh[w][threadIdx.x];
      eslice[threadIdx.x] = v;
    }
  }
  const int v0 = t.prob_var0[0], v1 = t.prob_var1[0];
  const int nv = v1 - v0;
  const int per = L.per;
  const int o0 = min(nv, rank * per), o1 = min(nv, o0 + per);  // owned local var range
  const int no = o1 - o0;
  float *zp = (float *)smem_raw;
  float *ox = zp + 12 * per;
  float *orr = ox + 6 * per;
  float *oq = orr + 6 * per;
  float *opn = oq + 6 * per;
  Acc *part = (Acc *)(((uintptr_t)(opn + 6 * per) + 15) & ~(uintptr_t)15);
  float *sD = (float *)(part + 2);
  float *sM = sD + 36 * per;
  float *sB = sM + 36 * per;
  int *sov = (int *)(sB + 36 * (size_t)L.max_inc);
  __shared__ float wsum[CL_WARPS];
  const int e_base = t.inc_off[v0 + o0];
  if (threadIdx.x < CL) zp_rank[threadIdx.x] = (const float4 *)cluster.map_shared_rank(zp, (int)threadIdx.x);
  if (L.cache) {
    for (int u = threadIdx.x; u < 36 * no; u += CL_BS) {
      sD[u] = Df[(long long)(v0 + o0) * 36 + u];
      sM[u] = Minv[(long long)(v0 + o0) * 36 + u];
    }
    // one thread per incidence: its block as 9 independent 16-byte loads, stored pre-transposed
    const int n_inc = t.inc_off[v0 + o1] - e_base;
    for (int e = threadIdx.x; e < n_inc; e += CL_BS) {
      const int ent = t.inc[e_base + e];
      const int ov = t.inc_ov[e_base + e];
      const float4 *O4 = (const float4 *)(pairoff + (long long)(ent >> 1) * 36);
      float o[36];
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const float4 v4 = O4[q];
        o[4 * q] = v4.x;
        o[4 * q + 1] = v4.y;
        o[4 * q + 2] = v4.z;
        o[4 * q + 3] = v4.w;
      }
      float *dst = sB + 36 * e;
      if ((ent & 1) == 0) {
#pragma unroll
        for (int q = 0; q < 36; ++q) dst[q] = o[q];
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
          for (int j = 0; j < 6; ++j) dst[6 * c + j] = o[6 * j + c];
      }
      const int lo = ov - v0;
      sov[e] = ov < 0 ? -1 : (((lo / per) << 16) | (lo % per));
    }
    __syncthreads();  // the init below reads sM rows that other threads of the CTA filled
  }
  // Frames are processed by CL_G-lane groups: group g of a warp owns frame base + g; within a
  // group lane gl walks the frame's incidences gl, gl + CL_G, ... and lanes gl < 6 own the
  // frame's 6 rows.
  constexpr int GPW = 32 / CL_G;  // groups per warp
  const int g = lane / CL_G, gl = lane % CL_G, gbase = lane & ~(CL_G - 1);
  // init: x = 0, r = b, z = M^-1 r, p = 0 for owned frames
  float loc = 0.f;
  for (int base = o0 + GPW * warp; base < o1; base += GPW * CL_WARPS) {
    const int lv = base + g;
    const bool valid = lv < o1;
    const int v = v0 + lv, k = lv - o0;
    const float rown = (valid && gl < 6) ? (float)rhs[6 * v + gl] : 0.f;
    float rr[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) rr[c] = __shfl_sync(0xffffffffu, rown, gbase + c);
    if (valid && gl < 6) {
      const float *M = L.cache ? sM + 36 * k + 6 * gl : Minv + (long long)v * 36 + 6 * gl;
      const float zl = M[0] * rr[0] + M[1] * rr[1] + M[2] * rr[2] + M[3] * rr[3] + M[4] * rr[4] + M[5] * rr[5];
      ox[6 * k + gl] = 0.f;
      orr[6 * k + gl] = rr[gl];
      zp[12 * k + gl] = zl;
      zp[12 * k + 6 + gl] = 0.f;
      loc += rr[gl] * zl;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
  cluster_partial<Acc>(loc, wsum, part, 1);
  cluster.sync();  // all CTAs running, owned z / p initialised, energy slices ready
  if (po.energy && rank == 0 && threadIdx.x < PAIREN) {
    Acc v = 0;
    for (int r = 0; r < CL; ++r) v += cluster.map_shared_rank(eslice, r)[threadIdx.x];
    po.energy[threadIdx.x] = (double)v;
  }
  __shared__ PcgScal S;
  Acc rz = 0;  // meaningful in thread 0, which runs the scalar recurrences
  if (warp == 0) {
    const Acc tot = cluster_total(cluster, part, 1, CL);
    if (lane == 0) {
      rz = tot;
      S.stop = rz == (Acc)0;
      S.fb = 0.f;
    }
  }
  __syncthreads();
  int flag = 0;
  for (int it = 0; it < n_pcg; ++it) {
    if (S.stop) break;
    const float fb = S.fb;
    // Phase A: p_new = z + beta p (owned, kept in opn); q = A p_new, neighbours read remotely
    float lpq = 0.f;
    for (int base = o0 + GPW * warp; base < o1; base += GPW * CL_WARPS) {
      const int lv = base + g;
      const bool valid = lv < o1;
      const int v = v0 + lv, k = lv - o0;
      float acc[6] = {0, 0, 0, 0, 0, 0};
      if (valid) {
        const int e0 = t.inc_off[v], e1 = t.inc_off[v + 1];
        for (int e = e0 + gl; e < e1; e += CL_G) {
          int owner, idx;
          const float *B;
          bool trans = false;
          if (L.cache) {
            const int so = sov[e - e_base];
            if (so < 0) continue;
            owner = so >> 16;
            idx = so & 0xffff;
            B = sB + 36 * (e - e_base);
          } else {
            const int ov = t.inc_ov[e];
            if (ov < 0) continue;
            const int lo = ov - v0;
            owner = lo / per;
            idx = lo - owner * per;
            const int ent = t.inc[e];
            B = pairoff + (long long)(ent >> 1) * 36;
            trans = (ent & 1) != 0;
          }
          const float4 *src = zp_rank[owner] + 3 * idx;
          const float4 q0 = src[0], q1 = src[1], q2 = src[2];  // z0..z5 p0..p5
          float po[6];
          po[0] = q0.x + fb * q1.z;
          po[1] = q0.y + fb * q1.w;
          po[2] = q0.z + fb * q2.x;
          po[3] = q0.w + fb * q2.y;
          po[4] = q1.x + fb * q2.z;
          po[5] = q1.y + fb * q2.w;
          if (!trans) {
#pragma unroll
            for (int c = 0; c < 6; ++c)
#pragma unroll
              for (int j = 0; j < 6; ++j) acc[c] += B[6 * c + j] * po[j];
          } else {
#pragma unroll
            for (int c = 0; c < 6; ++c)
#pragma unroll
              for (int j = 0; j < 6; ++j) acc[c] += B[6 * j + c] * po[j];
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) {
#pragma unroll
        for (int o = CL_G / 2; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
      }
      if (valid && gl < 6) {
        float mine = acc[0];
#pragma unroll
        for (int c = 1; c < 6; ++c) mine = (gl == c) ? acc[c] : mine;
        float pn[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) pn[c] = zp[12 * k + c] + fb * zp[12 * k + 6 + c];
        const float *Drow = L.cache ? sD + 36 * k + 6 * gl : Df + (long long)v * 36 + 6 * gl;
        const float qc = mine + Drow[0] * pn[0] + Drow[1] * pn[1] + Drow[2] * pn[2] + Drow[3] * pn[3] +
                         Drow[4] * pn[4] + Drow[5] * pn[5];
        float pmine = pn[0];
#pragma unroll
        for (int c = 1; c < 6; ++c) pmine = (gl == c) ? pn[c] : pmine;
        oq[6 * k + gl] = qc;
        opn[6 * k + gl] = pmine;
        lpq += pmine * qc;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lpq += __shfl_xor_sync(0xffffffffu, lpq, o);
    cluster_partial<Acc>(lpq, wsum, part, 0);
    cluster.sync();  // every CTA has finished reading the old z / p
    if (warp == 0) {
      const Acc pq = cluster_total(cluster, part, 0, CL);
      if (lane == 0) flag |= pcg_alpha(rz, pq, S);
    }
    __syncthreads();
    if (S.stop) break;
    const float fa = S.fa;
    // Phase B (local): x += alpha p_new, r -= alpha q, z = M^-1 r, p = p_new
    float lrz = 0.f;
    for (int base = o0 + GPW * warp; base < o1; base += GPW * CL_WARPS) {
      const int lv = base + g;
      const bool valid = lv < o1;
      const int v = v0 + lv, k = lv - o0;
      const float rn_own = (valid && gl < 6) ? orr[6 * k + gl] - fa * oq[6 * k + gl] : 0.f;
      float rn[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) rn[c] = __shfl_sync(0xffffffffu, rn_own, gbase + c);
      if (valid && gl < 6) {
        const float *M = L.cache ? sM + 36 * k + 6 * gl : Minv + (long long)v * 36 + 6 * gl;
        const float zl = M[0] * rn[0] + M[1] * rn[1] + M[2] * rn[2] + M[3] * rn[3] + M[4] * rn[4] + M[5] * rn[5];
        const float pl = opn[6 * k + gl];
        ox[6 * k + gl] += fa * pl;
        orr[6 * k + gl] = rn_own;
        zp[12 * k + gl] = zl;
        zp[12 * k + 6 + gl] = pl;
        lrz += rn_own * zl;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lrz += __shfl_xor_sync(0xffffffffu, lrz, o);
    cluster_partial<Acc>(lrz, wsum, part, 1);
    cluster.sync();  // the new z / p are visible cluster-wide
    if (warp == 0) {
      const Acc rz_new = cluster_total(cluster, part, 1, CL);
      if (lane == 0) pcg_beta(rz, rz_new, S);
    }
    __syncthreads();
  }
  // write the owned part of the solution
  __syncthreads();
  for (int u = threadIdx.x; u < 6 * no; u += CL_BS) xg[6 * (v0 + o0) + u] = ox[u];
  if (po.pose)
    for (int k = threadIdx.x; k < no; k += CL_BS) update_pose(po.pose + 12 * t.var_frame[v0 + o0 + k], ox + 6 * k);
  if (rank == 0 && threadIdx.x == 0 && pflags) pflags[0] |= flag;
  cluster.sync();  // keep every CTA's shared memory alive until remote reads are done
}

// Largest supported cluster (16 if the device allows non-portable sizes, else 8).
static int g_cluster_max = -1;
void cluster_size_override(int cl) { g_cluster_max = cl; }
int cluster_size_max() {
  int &cl = g_cluster_max;
  if (cl < 0) {
    cl = 0;
    if (cudaFuncSetAttribute(k_pcg_cluster<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_pcg_cluster<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess)
      cl = 16;
    else
      cl = 8;
    cudaGetLastError();
  }
  return cl;
}

constexpr size_t CLUSTER_SMEM_LIMIT = 220 * 1024;

// Shared-memory plan for n_vars frames on cl CTAs; inc_off is the host copy of the incidence
// offsets (nullptr: no cache).  Returns 0 if even the replicas do not fit.
static ClusterLayout cluster_layout(int n_vars, int cl, const int *inc_off, size_t *bytes) {
  ClusterLayout L;
  L.per = (n_vars + cl - 1) / cl;
  L.max_inc = 0;
  L.cache = false;
  if (inc_off) {
    for (int r = 0; r < cl; ++r) {
      const int a = std::min(n_vars, r * L.per), b = std::min(n_vars, a + L.per);
      L.max_inc = std::max(L.max_inc, inc_off[b] - inc_off[a]);
    }
    L.cache = cluster_bytes(n_vars, L.per, L.max_inc, true) <= CLUSTER_SMEM_LIMIT;
  }
  *bytes = cluster_bytes(n_vars, L.per, L.max_inc, L.cache);
  return L;
}

size_t cluster_smem_bytes(int n_vars, int cl) {
  size_t b;
  cluster_layout(n_vars, cl, nullptr, &b);
  return b;
}

template <typename Acc>
int launch_pcg_cluster(const Tables &t, const float *Df, const float *pairoff, const float *Minv, const Acc *rhs,
                       float *x, int n_pcg, int *pflags, int cl, const int *inc_off_host, const Acc *pairen,
                       PcgOut po, cudaStream_t st) {
  if (t.n_vars == 0) return 0;
  size_t smem = 0;
  const ClusterLayout L = cluster_layout(t.n_vars, cl, inc_off_host, &smem);
  static size_t smem_set[2] = {0, 0};
  size_t &cur = smem_set[sizeof(Acc) == 8 ? 1 : 0];
  if (smem > cur) {
    if (cudaFuncSetAttribute(k_pcg_cluster<Acc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CLUSTER_SMEM_LIMIT) !=
        cudaSuccess)
      return -1;
    cur = CLUSTER_SMEM_LIMIT;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(CL_BS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_pcg_cluster<Acc>, t, Df, pairoff, Minv, rhs, x, n_pcg, pflags, L, pairen, po) !=
      cudaSuccess) {
    cudaGetLastError();
    if (cl <= 8) return -1;
    // the device refused the non-portable size: use the portable maximum from now on
    cluster_size_override(8);
    return launch_pcg_cluster<Acc>(t, Df, pairoff, Minv, rhs, x, n_pcg, pflags, 8, inc_off_host, pairen, po, st);
  }
  return 1;
}
template int launch_pcg_cluster<double>(const Tables &, const float *, const float *, const float *, const double *,
                                        float *, int, int *, int, const int *, const double *, PcgOut, cudaStream_t);
template int launch_pcg_cluster<float>(const Tables &, const float *, const float *, const float *, const float *,
                                       float *, int, int *, int, const int *, const float *, PcgOut, cudaStream_t);

}  // namespace bf
