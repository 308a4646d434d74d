// Device code of the linear-system assembly and the PCG (Sec. 4.4) shared by the kernels of
// solve.cu and the persistent batched solve of batch.cu: the pair merge, the frame assembly with
// the block-Jacobi inverse, the energy record, and the per-problem PCG with its pose update.  The
// design notes are at the top of solve.cu.
#pragma once
#include "bf_internal.cuh"

namespace bf {

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
        // lanes 0-2 form one component each (B300 runs FP64 at 1/64 rate: a warp FP64
        // instruction costs the same with 3 lanes active as with 32), then broadcast
        const double *Ti = pose + 12 * srcf, *Tj = pose + 12 * tgt;
        const int m = lane < 3 ? lane : 0;
        const double dm = ldx<CG>(Ti + 9 + m) - ldx<CG>(Tj + 9 + m);
        const double d0 = __shfl_sync(0xffffffffu, dm, 0), d1 = __shfl_sync(0xffffffffu, dm, 1),
                     d2 = __shfl_sync(0xffffffffu, dm, 2);
        const Acc tm = (Acc)(ldx<CG>(Tj + m) * d0 + ldx<CG>(Tj + 3 + m) * d1 + ldx<CG>(Tj + 6 + m) * d2);
#pragma unroll
        for (int k = 0; k < 3; ++k) tt[k] = __shfl_sync(0xffffffffu, tm, k);
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

// --------------------------------------------------------------------------------- assemble
// Block-Jacobi preconditioner block: the inverse of the 6x6 diagonal block D (FP64 sums) formed
// in FP32.  D is first scaled symmetrically to unit diagonal (Dh = S D S, S = diag(D_ii^-1/2)),
// then Dh = L L^T (Cholesky), Dh^-1 = L^-T L^-1 and D^-1 = S Dh^-1 S.  The preconditioner only
// steers the PCG iterates, and B300 issues FP64 at 1/64 of the FP32 rate: one FP64 Cholesky
// inverse in a single lane costs tens of microseconds there.  Returns false if the block is not
// positive definite.
__device__ inline bool chol_inverse6(const double *D, float *Mi) {
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
  // lane handles entries lane and lane + 32 of [D (36) | rhs (6)] in one pass over the incidences,
  // read 8 at a time (all loads in flight together) and summed in incidence order
  const int k2 = lane + 32;
  const bool has2 = k2 < 42;
  Acc s1 = 0, s2 = 0;
  for (int e = e0; e < e1; e += 8) {
    Acc v1[8], v2[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      v1[u] = 0;
      v2[u] = 0;
      if (e + u < e1) {
        const int ent = t.inc[e + u];
        const int p = ent >> 1, side = ent & 1;
        const Acc *b = pairblk + (long long)p * PAIRBLK;
        v1[u] = b[(side == 0 ? PB_AA : PB_BB) + lane];
        if (has2) v2[u] = k2 < 36 ? b[(side == 0 ? PB_AA : PB_BB) + k2] : b[(side == 0 ? PB_RA : PB_RB) + k2 - 36];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (e + u < e1) {
        s1 += v1[u];
        s2 += v2[u];
      }
  }
  Dd[(long long)v * 36 + lane] = s1;
  Df[(long long)v * 36 + lane] = (float)s1;
  Dshw[lane] = (double)s1;
  if (has2) {
    if (k2 < 36) {
      Dd[(long long)v * 36 + k2] = s2;
      Df[(long long)v * 36 + k2] = (float)s2;
      Dshw[k2] = (double)s2;
    } else {
      rhs[(long long)v * 6 + k2 - 36] = s2;
    }
  }
  // an all-zero block (integer test for +-0: an FP64 compare would occupy the slow FP64 pipe)
  const bool nz = ((__double_as_longlong((double)s1) << 1) != 0) ||
                  (k2 < 36 && ((__double_as_longlong((double)s2) << 1) != 0));
  const bool empty = __ballot_sync(0xffffffffu, nz) == 0u;
  for (int k = lane; k < 36; k += 32) Mshw[k] = 0.f;
  __syncwarp();
  if (lane == 0) {
    int flag = 0;
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

// Float-float sums for the cross-CTA reductions of the mixed-precision PCG.  B300 issues FP64 at
// 1/64 of the FP32 rate, so every FP64 step of a reduction chain (convert, add, compare) holds
// the chain for at least 64 cycles; an unevaluated sum hi + lo of two FP32 values, added with
// Knuth's TwoSum and renormalised (Dekker's FastTwoSum), keeps about 48 significant bits on the
// FP32 pipe.  ff_add is commutative (the low parts are added to each other first), so a butterfly
// leaves every lane with the same value.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_from(float x) { return FF{x, 0.f}; }
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));  // a.hi + b.hi - s, exactly
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, e);
  return FF{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
__device__ __forceinline__ FF ff_shfl_xor(FF a, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
// FP32 rounding of hi + lo (hi alone after renormalisation, but for the halfway cases)
__device__ __forceinline__ float ff_f32(FF a) { return __fadd_rn(a.hi, a.lo); }

// The PCG scalars from float-float sums (same decisions as the FP64 forms below).
__device__ __forceinline__ int pcg_alpha(FF rz, FF pq, PcgScal &S) {
  if (!(pq.hi > 0.f)) {
    S.stop = 1;
    return 4;  // BF_FLAG_PCG_BREAKDOWN
  }
  S.fa = __fdiv_rn(ff_f32(rz), ff_f32(pq));
  return 0;
}
__device__ __forceinline__ void pcg_beta(FF &rz, FF rz_new, PcgScal &S) {
  S.fb = __fdiv_rn(ff_f32(rz_new), ff_f32(rz));
  rz = rz_new;
  S.stop = rz.hi == 0.f;
}

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
__device__ inline void mf_pair(const Tables &t, const MatFree &mf, int pr, const float (&da)[6], const float (&db)[6],
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
__device__ inline void pcg_finish(const Tables &t, const float *x, int prob, int v0, int v1, const PcgOut &po) {
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

}  // namespace bf
