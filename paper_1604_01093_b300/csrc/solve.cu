// Linear-system assembly, block-Jacobi PCG and the pose update (Sec. 4.4).
//
//   k_pair_xform   per pair: T_b^-1 T_a and T_a^-1 T_b, FP64 with explicit rounding, stored FP32
//   k_pair_merge   per pair: sum the pair's tile / segment partials (FP64 in mixed precision),
//                  rotate them from target-camera to world coordinates and expand the
//                  [a, v, c, -v] sums into the 6x6 blocks A_aa, A_ab, A_bb and rhs_a, rhs_b
//   k_assemble     per free frame: its diagonal block and rhs (sum over incident pairs, fixed
//                  order) and the preconditioner: 6x6 Cholesky inverse (block-Jacobi) or the
//                  inverse diagonal (Jacobi, the paper's choice)
//   k_pcg          per problem, one CTA: exactly n_pcg PCG iterations from x = 0, stopping early
//                  only if p.Ap <= 0 or r.z == 0; block-sparse matvec over the pair blocks
//   k_update       per free frame: R <- Exp(dw) R, t <- t + dt (FP64)
#include "bf_internal.cuh"

namespace bf {

// ------------------------------------------------------------------------------- pair xform
__global__ void k_pair_xform(int n_pairs, const int *__restrict__ pa, const int *__restrict__ pb,
                             const double *__restrict__ pose, float *__restrict__ pairM) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  const double *Ta = pose + 12 * pa[p];
  const double *Tb = pose + 12 * pb[p];
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    const double *Ti = dir == 0 ? Ta : Tb;  // source
    const double *Tj = dir == 0 ? Tb : Ta;  // target
    float *M = pairM + p * 24 + dir * 12;
    const double d0 = __dsub_rn(Ti[9], Tj[9]), d1 = __dsub_rn(Ti[10], Tj[10]), d2 = __dsub_rn(Ti[11], Tj[11]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        // R[a][b] = (Rj[0][a] Ri[0][b] + Rj[1][a] Ri[1][b]) + Rj[2][a] Ri[2][b]
        const double v = __dadd_rn(__dadd_rn(__dmul_rn(Tj[a], Ti[b]), __dmul_rn(Tj[3 + a], Ti[3 + b])),
                                   __dmul_rn(Tj[6 + a], Ti[6 + b]));
        M[3 * a + b] = (float)v;
      }
      const double tv = __dadd_rn(__dadd_rn(__dmul_rn(Tj[a], d0), __dmul_rn(Tj[3 + a], d1)), __dmul_rn(Tj[6 + a], d2));
      M[9 + a] = (float)tv;
    }
  }
}

void launch_pair_xform(const Tables &t, const double *pose, float *pairM, cudaStream_t st) {
  if (t.n_pairs == 0) return;
  k_pair_xform<<<(t.n_pairs + 127) / 128, 128, 0, st>>>(t.n_pairs, t.pair_a, t.pair_b, pose, pairM);
}

// ------------------------------------------------------------------------------- pair merge
template <typename Acc>
__device__ __forceinline__ void sym_get(const Acc *s, Acc (&m)[3][3]) {
  m[0][0] = s[0]; m[0][1] = s[1]; m[0][2] = s[2];
  m[1][0] = s[1]; m[1][1] = s[3]; m[1][2] = s[4];
  m[2][0] = s[2]; m[2][1] = s[4]; m[2][2] = s[5];
}
template <typename Acc>
__device__ __forceinline__ void full_get(const Acc *s, Acc (&m)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) m[i][j] = s[3 * i + j];
}
// X <- R X R^T
template <typename Acc>
__device__ __forceinline__ void rot33(const Acc (&R)[3][3], Acc (&X)[3][3]) {
  Acc T[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) T[i][j] = R[i][0] * X[0][j] + R[i][1] * X[1][j] + R[i][2] * X[2][j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) X[i][j] = T[i][0] * R[j][0] + T[i][1] * R[j][1] + T[i][2] * R[j][2];
}
template <typename Acc>
__device__ __forceinline__ void rot3(const Acc (&R)[3][3], const Acc *v, Acc (&o)[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) o[i] = R[i][0] * v[0] + R[i][1] * v[1] + R[i][2] * v[2];
}

// Add one direction's sums S (target-frame coordinates, rotated here by R = R_target) into the
// pair's blocks.  src_is_a selects whether the source of the direction is frame a.
template <typename Acc>
__device__ void add_direction(const Acc *S, const Acc (&R)[3][3], bool src_is_a, Acc *blk) {
  Acc Saa[3][3], Sav[3][3], Svv[3][3], Sac[3][3], Svc[3][3], Scc[3][3], ga[3], gv[3], gc[3];
  sym_get(S + P_AA, Saa); full_get(S + P_AV, Sav); sym_get(S + P_VV, Svv);
  full_get(S + P_AC, Sac); full_get(S + P_VC, Svc); sym_get(S + P_CC, Scc);
  rot33(R, Saa); rot33(R, Sav); rot33(R, Svv); rot33(R, Sac); rot33(R, Svc); rot33(R, Scc);
  rot3(R, S + P_GA, ga); rot3(R, S + P_GV, gv); rot3(R, S + P_GC, gc);
  Acc *Ass = blk + (src_is_a ? PB_AA : PB_BB);
  Acc *Att = blk + (src_is_a ? PB_BB : PB_AA);
  Acc *Aab = blk + PB_AB;
  Acc *rs = blk + (src_is_a ? PB_RA : PB_RB);
  Acc *rt = blk + (src_is_a ? PB_RB : PB_RA);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // A_ss = [[Saa, Sav], [Sav^T, Svv]]
      Ass[6 * i + j] += Saa[i][j];
      Ass[6 * i + 3 + j] += Sav[i][j];
      Ass[6 * (3 + i) + j] += Sav[j][i];
      Ass[6 * (3 + i) + 3 + j] += Svv[i][j];
      // A_tt = [[Scc, -Svc^T], [-Svc, Svv]]
      Att[6 * i + j] += Scc[i][j];
      Att[6 * i + 3 + j] += -Svc[j][i];
      Att[6 * (3 + i) + j] += -Svc[i][j];
      Att[6 * (3 + i) + 3 + j] += Svv[i][j];
      // A_st = [[Sac, -Sav], [Svc, -Svv]]  (rows source, cols target)
      const Acc st00 = Sac[i][j], st01 = -Sav[i][j], st10 = Svc[i][j], st11 = -Svv[i][j];
      if (src_is_a) {
        Aab[6 * i + j] += st00;
        Aab[6 * i + 3 + j] += st01;
        Aab[6 * (3 + i) + j] += st10;
        Aab[6 * (3 + i) + 3 + j] += st11;
      } else {  // A_ab = A_st^T
        Aab[6 * j + i] += st00;
        Aab[6 * (3 + j) + i] += st01;
        Aab[6 * j + 3 + i] += st10;
        Aab[6 * (3 + j) + 3 + i] += st11;
      }
    }
    // rhs = -J^T W r : source (ga, gv), target (gc, -gv)
    rs[i] -= ga[i];
    rs[3 + i] -= gv[i];
    rt[i] -= gc[i];
    rt[3 + i] += gv[i];
  }
}

template <typename Acc>
__device__ __forceinline__ void load_R(const double *T, Acc (&R)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R[i][j] = (Acc)T[3 * i + j];
}

template <typename Acc, typename Part>
__global__ void k_pair_merge(Tables t, const double *__restrict__ pose, const Part *__restrict__ dpart,
                             const Part *__restrict__ spart, Acc *__restrict__ pairblk, Acc *__restrict__ pairen,
                             float *__restrict__ pairoff) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= t.n_pairs) return;
  Acc blk[PAIRBLK];
#pragma unroll
  for (int k = 0; k < PAIRBLK; ++k) blk[k] = 0;
  Acc en[PAIREN] = {0, 0, 0, 0};
  const int fa = t.pair_a[p], fb = t.pair_b[p];
  Acc Ra[3][3], Rb[3][3];
  load_R(pose + 12 * fa, Ra);
  load_R(pose + 12 * fb, Rb);
  Acc S[NPART];
  // dense directions
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    const int d = t.pair_dp[2 * p + dir];
    if (d < 0) continue;
#pragma unroll
    for (int k = 0; k < NPART; ++k) S[k] = 0;
    for (int tl = t.dp_tile0[d]; tl < t.dp_tile1[d]; ++tl) {
      const Part *src = dpart + (long long)tl * NPART;
#pragma unroll
      for (int k = 0; k < NPART; ++k) S[k] += (Acc)src[k];
    }
    add_direction<Acc>(S, dir == 0 ? Rb : Ra, dir == 0, blk);
    en[2] += S[P_E0];
    en[1] += S[P_E1];
    en[3] += S[P_CNT];
  }
  // sparse segments (camera-b coordinates, source a)
  if (t.pair_seg1[p] > t.pair_seg0[p]) {
#pragma unroll
    for (int k = 0; k < NPART; ++k) S[k] = 0;
    for (int s = t.pair_seg0[p]; s < t.pair_seg1[p]; ++s) {
      const Part *src = spart + (long long)s * NPART;
#pragma unroll
      for (int k = 0; k < NPART; ++k) S[k] += (Acc)src[k];
    }
    add_direction<Acc>(S, Rb, true, blk);
    en[0] += S[P_E0];
  }
  Acc *out = pairblk + (long long)p * PAIRBLK;
#pragma unroll
  for (int k = 0; k < PAIRBLK; ++k) out[k] = blk[k];
#pragma unroll
  for (int k = 0; k < PAIREN; ++k) pairen[(long long)p * PAIREN + k] = en[k];
#pragma unroll
  for (int k = 0; k < 36; ++k) pairoff[(long long)p * 36 + k] = (float)blk[PB_AB + k];
}

template <typename Acc, typename Part>
void launch_pair_merge(const Tables &t, const double *pose, const Part *dpart, const Part *spart, Acc *pairblk,
                       Acc *pairen, float *pairoff, cudaStream_t st) {
  if (t.n_pairs == 0) return;
  k_pair_merge<Acc, Part><<<(t.n_pairs + 63) / 64, 64, 0, st>>>(t, pose, dpart, spart, pairblk, pairen, pairoff);
}
template void launch_pair_merge<double, double>(const Tables &, const double *, const double *, const double *,
                                                double *, double *, float *, cudaStream_t);
template void launch_pair_merge<float, float>(const Tables &, const double *, const float *, const float *, float *,
                                              float *, float *, cudaStream_t);

// --------------------------------------------------------------------------------- assemble
template <typename Acc>
__global__ void k_assemble(Tables t, const Acc *__restrict__ pairblk, int precond, Acc *__restrict__ Dd,
                           Acc *__restrict__ rhs, float *__restrict__ Df, float *__restrict__ Minv,
                           int *__restrict__ vflags) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= t.n_vars) return;
  Acc D[36], r[6];
#pragma unroll
  for (int k = 0; k < 36; ++k) D[k] = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) r[k] = 0;
  for (int e = t.inc_off[v]; e < t.inc_off[v + 1]; ++e) {
    const int ent = t.inc[e];
    const int p = ent >> 1, side = ent & 1;
    const Acc *b = pairblk + (long long)p * PAIRBLK;
    const Acc *Dsrc = b + (side == 0 ? PB_AA : PB_BB);
    const Acc *rsrc = b + (side == 0 ? PB_RA : PB_RB);
#pragma unroll
    for (int k = 0; k < 36; ++k) D[k] += Dsrc[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) r[k] += rsrc[k];
  }
  int flag = 0;
  bool empty = true;
#pragma unroll
  for (int k = 0; k < 36; ++k) {
    Dd[(long long)v * 36 + k] = D[k];
    Df[(long long)v * 36 + k] = (float)D[k];
    empty = empty && (D[k] == 0);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) rhs[(long long)v * 6 + k] = r[k];
  // preconditioner in FP64 regardless of Acc
  double Mi[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) Mi[k] = 0.0;
  if (empty) {
    flag = 2;  // BF_FLAG_EMPTY_FRAME
  } else {
    bool chol_ok = (precond == 0);
    double L[36];
    if (chol_ok) {
#pragma unroll
      for (int k = 0; k < 36; ++k) L[k] = 0.0;
      for (int j = 0; j < 6 && chol_ok; ++j) {
        double s = (double)D[6 * j + j];
        for (int k = 0; k < j; ++k) s -= L[6 * j + k] * L[6 * j + k];
        if (!(s > 0.0)) {
          chol_ok = false;
          break;
        }
        const double ljj = sqrt(s);
        L[6 * j + j] = ljj;
        for (int i = j + 1; i < 6; ++i) {
          double u = (double)D[6 * i + j];
          for (int k = 0; k < j; ++k) u -= L[6 * i + k] * L[6 * j + k];
          L[6 * i + j] = u / ljj;
        }
      }
      if (chol_ok) {
        // inverse of L (lower), then M^-1 = L^-T L^-1
        double Li[36];
        for (int k = 0; k < 36; ++k) Li[k] = 0.0;
        for (int i = 0; i < 6; ++i) {
          Li[6 * i + i] = 1.0 / L[6 * i + i];
          for (int j = 0; j < i; ++j) {
            double s = 0.0;
            for (int k = j; k < i; ++k) s -= L[6 * i + k] * Li[6 * k + j];
            Li[6 * i + j] = s / L[6 * i + i];
          }
        }
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j < 6; ++j) {
            double s = 0.0;
            for (int k = (i > j ? i : j); k < 6; ++k) s += Li[6 * k + i] * Li[6 * k + j];
            Mi[6 * i + j] = s;
          }
      } else if (precond == 0) {
        flag = 1;  // BF_FLAG_SINGULAR_BLOCK: fall back to the diagonal
      }
    }
    if (!chol_ok) {
      for (int k = 0; k < 6; ++k) {
        const double d = (double)D[7 * k];
        Mi[7 * k] = d > 0.0 ? 1.0 / d : 0.0;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 36; ++k) Minv[(long long)v * 36 + k] = (float)Mi[k];
  vflags[v] = flag;
}

template <typename Acc>
void launch_assemble(const Tables &t, const Acc *pairblk, int precond, Acc *Dd, Acc *rhs, float *Df, float *Minv,
                     int *vflags, cudaStream_t st) {
  if (t.n_vars == 0) return;
  k_assemble<Acc><<<(t.n_vars + 63) / 64, 64, 0, st>>>(t, pairblk, precond, Dd, rhs, Df, Minv, vflags);
}
template void launch_assemble<double>(const Tables &, const double *, int, double *, double *, float *, float *,
                                      int *, cudaStream_t);
template void launch_assemble<float>(const Tables &, const float *, int, float *, float *, float *, float *, int *,
                                     cudaStream_t);

// -------------------------------------------------------------------------------------- PCG
constexpr int PCG_BS = 256;

template <typename Acc>
__device__ __forceinline__ Acc cta_sum(Acc v, Acc *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // protect sh from a previous use
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  Acc s = 0;
#pragma unroll
  for (int w = 0; w < PCG_BS / 32; ++w) s += sh[w];
  return s;
}

// z_v = Minv_v r_v for the row u = 6 v + c
__device__ __forceinline__ float precond_row(const float *__restrict__ Minv, const float *__restrict__ r, int v,
                                             int c) {
  const float *Mr = Minv + (long long)v * 36 + 6 * c;
  const float *rv = r + 6LL * v;
  return Mr[0] * rv[0] + Mr[1] * rv[1] + Mr[2] * rv[2] + Mr[3] * rv[3] + Mr[4] * rv[4] + Mr[5] * rv[5];
}

template <typename Acc>
__global__ void __launch_bounds__(PCG_BS)
    k_pcg(Tables t, const float *__restrict__ Df, const float *__restrict__ pairoff, const float *__restrict__ Minv,
          const Acc *__restrict__ rhs, float *__restrict__ x, float *__restrict__ r, float *__restrict__ z,
          float *__restrict__ p, float *__restrict__ q, int n_pcg, int *__restrict__ pflags) {
  __shared__ Acc sh[PCG_BS / 32];
  const int prob = blockIdx.x;
  const int v0 = t.prob_var0[prob], v1 = t.prob_var1[prob];
  const int u0 = 6 * v0, u1 = 6 * v1;
  for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
    x[u] = 0.f;
    r[u] = (float)rhs[u];
  }
  __syncthreads();
  Acc loc = 0;
  for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
    const float zu = precond_row(Minv, r, u / 6, u % 6);
    z[u] = zu;
    p[u] = zu;
    loc += (Acc)r[u] * (Acc)zu;
  }
  Acc rz = cta_sum(loc, sh);
  int flag = 0;
  for (int it = 0; it < n_pcg; ++it) {
    if (rz == (Acc)0) break;
    // q = A p ; loc = p . q
    loc = 0;
    for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
      const int v = u / 6, c = u % 6;
      const float *Drow = Df + (long long)v * 36 + 6 * c;
      const float *pv = p + 6LL * v;
      float s = Drow[0] * pv[0] + Drow[1] * pv[1] + Drow[2] * pv[2] + Drow[3] * pv[3] + Drow[4] * pv[4] +
                Drow[5] * pv[5];
      for (int e = t.inc_off[v]; e < t.inc_off[v + 1]; ++e) {
        const int ent = t.inc[e];
        const int pr = ent >> 1, side = ent & 1;
        const int other = side == 0 ? t.pair_b[pr] : t.pair_a[pr];
        const int ov = t.frame_var[other];
        if (ov < 0) continue;
        const float *O = pairoff + (long long)pr * 36;
        const float *po = p + 6LL * ov;
        if (side == 0) {  // row of A_ab
          s += O[6 * c] * po[0] + O[6 * c + 1] * po[1] + O[6 * c + 2] * po[2] + O[6 * c + 3] * po[3] +
               O[6 * c + 4] * po[4] + O[6 * c + 5] * po[5];
        } else {  // row of A_ba = A_ab^T
          s += O[c] * po[0] + O[6 + c] * po[1] + O[12 + c] * po[2] + O[18 + c] * po[3] + O[24 + c] * po[4] +
               O[30 + c] * po[5];
        }
      }
      q[u] = s;
      loc += (Acc)p[u] * (Acc)s;
    }
    const Acc pq = cta_sum(loc, sh);
    if (!(pq > (Acc)0)) {
      flag |= 4;  // BF_FLAG_PCG_BREAKDOWN
      break;
    }
    const Acc alpha = rz / pq;
    for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
      x[u] = (float)((Acc)x[u] + alpha * (Acc)p[u]);
      r[u] = (float)((Acc)r[u] - alpha * (Acc)q[u]);
    }
    __syncthreads();
    loc = 0;
    for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) {
      const float zu = precond_row(Minv, r, u / 6, u % 6);
      z[u] = zu;
      loc += (Acc)r[u] * (Acc)zu;
    }
    const Acc rz_new = cta_sum(loc, sh);
    const Acc beta = rz_new / rz;
    rz = rz_new;
    for (int u = u0 + threadIdx.x; u < u1; u += PCG_BS) p[u] = (float)((Acc)z[u] + beta * (Acc)p[u]);
    __syncthreads();
  }
  if (threadIdx.x == 0 && pflags) pflags[prob] |= flag;
}

template <typename Acc>
void launch_pcg(const Tables &t, const float *Df, const float *pairoff, const float *Minv, const Acc *rhs, float *x,
                float *r, float *z, float *p, float *q, int n_pcg, int *pflags, cudaStream_t st) {
  if (t.n_prob == 0) return;
  k_pcg<Acc><<<t.n_prob, PCG_BS, 0, st>>>(t, Df, pairoff, Minv, rhs, x, r, z, p, q, n_pcg, pflags);
}
template void launch_pcg<double>(const Tables &, const float *, const float *, const float *, const double *, float *,
                                 float *, float *, float *, float *, int, int *, cudaStream_t);
template void launch_pcg<float>(const Tables &, const float *, const float *, const float *, const float *, float *,
                                float *, float *, float *, float *, int, int *, cudaStream_t);

// ----------------------------------------------------------------------------- pose update
__global__ void k_update(int n_vars, const int *__restrict__ var_frame, const float *__restrict__ x,
                         double *__restrict__ pose) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_vars) return;
  double *T = pose + 12 * var_frame[v];
  const double w0 = x[6 * v], w1 = x[6 * v + 1], w2 = x[6 * v + 2];
  const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
  const double th = sqrt(th2);
  double A, B;  // Exp(w) = I + A K + B K^2 (Rodrigues)
  if (th < 1e-8) {
    A = 1.0;
    B = 0.5;
  } else {
    A = sin(th) / th;
    B = (1.0 - cos(th)) / th2;
  }
  const double K[3][3] = {{0.0, -w2, w1}, {w2, 0.0, -w0}, {-w1, w0, 0.0}};
  double E[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double K2 = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
      E[i][j] = (i == j ? 1.0 : 0.0) + A * K[i][j] + B * K2;
    }
  double R[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[3 * i + j] = E[i][0] * T[j] + E[i][1] * T[3 + j] + E[i][2] * T[6 + j];
  for (int k = 0; k < 9; ++k) T[k] = R[k];
  T[9] += (double)x[6 * v + 3];
  T[10] += (double)x[6 * v + 4];
  T[11] += (double)x[6 * v + 5];
}

void launch_update(const Tables &t, const float *x, double *pose, cudaStream_t st) {
  if (t.n_vars == 0) return;
  k_update<<<(t.n_vars + 127) / 128, 128, 0, st>>>(t.n_vars, t.var_frame, x, pose);
}

// ------------------------------------------------------------------------- energy reduce
template <typename Acc>
__global__ void k_energy_reduce(Tables t, const Acc *__restrict__ pairen, double *__restrict__ out) {
  const int prob = blockIdx.x;
  if (threadIdx.x >= PAIREN) return;
  Acc s = 0;
  for (int p = t.prob_pair0[prob]; p < t.prob_pair1[prob]; ++p) s += pairen[(long long)p * PAIREN + threadIdx.x];
  out[prob * PAIREN + threadIdx.x] = (double)s;
}

template <typename Acc>
void launch_energy_reduce(const Tables &t, const Acc *pairen, double *out, cudaStream_t st) {
  if (t.n_prob == 0) return;
  k_energy_reduce<Acc><<<t.n_prob, 32, 0, st>>>(t, pairen, out);
}
template void launch_energy_reduce<double>(const Tables &, const double *, double *, cudaStream_t);
template void launch_energy_reduce<float>(const Tables &, const float *, double *, cudaStream_t);

}  // namespace bf
