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
// products are summed in FP32 within a warp (a 32-term tree; in k_pcg_cluster within the CTA)
// and everything above that in FP64, or in k_pcg_cluster as float-float sums (about 48 bits,
// FP32 pipe: the cross-CTA reductions are on its critical path twice per iteration); alpha and
// beta are FP32 quotients of the rounded sums.  B300 issues FP64 at 1/64 of the FP32 rate, so
// per-element FP64 arithmetic would dominate these latency-bound kernels.
#include <cooperative_groups.h>

#include <algorithm>

#include "solve_eval.cuh"

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

// Energy record of every pair alone (the final energy evaluation needs no pair blocks): one
// thread per pair, the same sums in the same order as merge_pair (dense a -> b, sparse segments,
// dense b -> a), so the records equal the full merge's bit for bit.
template <typename Acc>
__global__ void k_pair_energy(Tables t, const Acc *__restrict__ dpart, const Acc *__restrict__ spart,
                              Acc *__restrict__ pairen) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= t.n_pairs) return;
  Acc en[4] = {0, 0, 0, 0};  // e_sparse, e_photo, e_geo, n_dense
  for (int half = 0; half < 2; ++half) {
    const int d = t.pair_dp[2 * p + half];
    if (d >= 0) {
      const int k0 = t.dp_tile0[d], k1 = t.dp_tile1[d];
      Acc e0 = 0, e1 = 0, cn = 0;
      for (int it = k0; it < k1; ++it) e0 += dpart[(long long)it * NPD + D_E0];
      for (int it = k0; it < k1; ++it) e1 += dpart[(long long)it * NPD + D_E1];
      for (int it = k0; it < k1; ++it) cn += dpart[(long long)it * NPD + D_CNT];
      en[2] += e0;
      en[1] += e1;
      en[3] += cn;
    }
    if (spart != nullptr && half == 0 && t.pair_seg1[p] > t.pair_seg0[p]) {
      Acc s = 0;
      for (int it = t.pair_seg0[p]; it < t.pair_seg1[p]; ++it) s += spart[(long long)it * NPART + P_E0];
      en[0] += s;
    }
  }
#pragma unroll
  for (int k = 0; k < PAIREN; ++k) pairen[(long long)p * PAIREN + k] = en[k];
}

template <typename Acc>
int launch_pair_energy(const Tables &t, const Acc *dpart, const Acc *spart, Acc *pairen, cudaStream_t st) {
  if (t.n_pairs == 0) return 0;
  k_pair_energy<Acc><<<(t.n_pairs + 127) / 128, 128, 0, st>>>(t, dpart, spart, pairen);
  return 1;
}
template int launch_pair_energy<double>(const Tables &, const double *, const double *, double *, cudaStream_t);
template int launch_pair_energy<float>(const Tables &, const float *, const float *, float *, cudaStream_t);

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
  static PerDevice max_blocks;
  return (int)max_blocks.get(0, [] {
    int dev = 0, sms = 0, per_sm = 0, per_sm_f = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_coop<double>, COOP_BS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, k_pcg_coop<float>, COOP_BS, 0);
    per_sm = per_sm < per_sm_f ? per_sm : per_sm_f;
    return (long long)sms * (per_sm < 1 ? 1 : per_sm);
  });
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

// Type of the cross-CTA sums: float-float in mixed precision (about 48 bits on the FP32 pipe,
// see FF), FP32 in the plain path.
template <typename Acc>
struct ClusterRed {
  using T = float;
};
template <>
struct ClusterRed<double> {
  using T = FF;
};
__device__ __forceinline__ float red_of(float x, float) { return x; }
__device__ __forceinline__ FF red_of(float x, FF) { return ff_from(x); }
__device__ __forceinline__ float red_add(float a, float b) { return a + b; }
__device__ __forceinline__ FF red_add(FF a, FF b) { return ff_add(a, b); }
__device__ __forceinline__ float red_shfl(float a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
__device__ __forceinline__ FF red_shfl(FF a, int o) { return ff_shfl_xor(a, o); }
__device__ __forceinline__ bool red_zero(float a) { return a == 0.f; }
__device__ __forceinline__ bool red_zero(FF a) { return a.hi == 0.f; }

// Sum of the CL <= 16 per-CTA partials (slot k of each CTA's part array), read lane-parallel from
// the cluster's shared memory and combined by a butterfly over lanes 0-15: lane 0 holds the total.
template <typename R>
__device__ __forceinline__ R cluster_total(cgx::cluster_group &cluster, R *part, int k, int CL) {
  const int lane = threadIdx.x & 31;
  R s = red_of(0.f, R{});
  if (lane < CL) s = cluster.map_shared_rank(part, lane)[k];
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) s = red_add(s, red_shfl(s, o));
  return s;
}

// Fixed-order CTA sum of one FP32 value per warp (lane 0 holds it) into part[k]: a butterfly
// over the CL_WARPS = 16 values in warp 0 (FP32); the wider type starts at the sum over the
// cluster's CTAs.
template <typename R>
__device__ __forceinline__ void cluster_partial(float v, float *wsum, R *part, int k) {
  static_assert(CL_WARPS == 16, "the butterfly below sums 16 warp values");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    float s = lane < CL_WARPS ? wsum[lane] : 0.f;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[k] = red_of(s, R{});
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
  __shared__ Acc eslice[PAIREN];
  cgx::cluster_group cluster = cgx::this_cluster();
  const int rank = (int)cluster.block_rank(), CL = (int)cluster.num_blocks();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (po.energy && warp == CL_WARPS - 1) {
    // this CTA's slice of the energy record, by its last warp while the others fill the block
    // cache: its share of the pairs strided over the lanes, then a reduce-scatter of the four
    // FP64 sums (6 FP64 adds instead of a butterfly per sum); rank 0 adds the slices in rank order
    // after the first barrier
    const int p0 = t.prob_pair0[0], np = t.prob_pair1[0] - p0, chunk = (np + CL - 1) / CL;
    const int pa = p0 + min(np, rank * chunk), pb = p0 + min(np, (rank + 1) * chunk);
    Acc es[PAIREN] = {0, 0, 0, 0};
    for (int q = pa + lane; q < pb; q += 32)
#pragma unroll
      for (int c = 0; c < PAIREN; ++c) es[c] += pairen[(long long)q * PAIREN + c];
    static_assert(PAIREN == 4, "the reduce-scatter below splits four sums");
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    Acc k0 = hi16 ? es[2] : es[0], k1 = hi16 ? es[3] : es[1];
    k0 += __shfl_xor_sync(0xffffffffu, hi16 ? es[0] : es[2], 16);
    k1 += __shfl_xor_sync(0xffffffffu, hi16 ? es[1] : es[3], 16);
    Acc v = hi8 ? k1 : k0;
    v += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((lane & 7) == 0) eslice[lane >> 3] = v;  // lanes 0, 8, 16, 24: sums 0, 1, 2, 3
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
  using R = typename ClusterRed<Acc>::T;
  R *part = (R *)(((uintptr_t)(opn + 6 * per) + 15) & ~(uintptr_t)15);
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
  cluster_partial<R>(loc, wsum, part, 1);
  cluster.sync();  // all CTAs running, owned z / p initialised, energy slices ready
  if (po.energy && rank == 0 && threadIdx.x < PAIREN) {
    Acc v = 0;
    for (int r = 0; r < CL; ++r) v += cluster.map_shared_rank(eslice, r)[threadIdx.x];
    po.energy[threadIdx.x] = (double)v;
  }
  __shared__ PcgScal S;
  R rz = red_of(0.f, R{});  // meaningful in thread 0, which runs the scalar recurrences
  if (warp == 0) {
    const R tot = cluster_total(cluster, part, 1, CL);
    if (lane == 0) {
      rz = tot;
      S.stop = red_zero(rz);
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
    cluster_partial<R>(lpq, wsum, part, 0);
    cluster.sync();  // every CTA has finished reading the old z / p
    if (warp == 0) {
      const R pq = cluster_total(cluster, part, 0, CL);
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
    cluster_partial<R>(lrz, wsum, part, 1);
    cluster.sync();  // the new z / p are visible cluster-wide
    if (warp == 0) {
      const R rz_new = cluster_total(cluster, part, 1, CL);
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

// Largest supported cluster on the current device (16 if it allows non-portable sizes, else 8).
static PerDevice g_cluster_max;
void cluster_size_override(int cl) { g_cluster_max.set(0, cl); }
int cluster_size_max() {
  return (int)g_cluster_max.get(0, [] {
    long long cl = 8;
    if (cudaFuncSetAttribute(k_pcg_cluster<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_pcg_cluster<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess)
      cl = 16;
    cudaGetLastError();
    return cl;
  });
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

bool cluster_cache_fits(int n_vars, int cl, const int *inc_off) {
  size_t b;
  return cluster_layout(n_vars, cl, inc_off, &b).cache;
}

template <typename Acc>
int launch_pcg_cluster(const Tables &t, const float *Df, const float *pairoff, const float *Minv, const Acc *rhs,
                       float *x, int n_pcg, int *pflags, int cl, const int *inc_off_host, const Acc *pairen,
                       PcgOut po, cudaStream_t st) {
  if (t.n_vars == 0) return 0;
  size_t smem = 0;
  const ClusterLayout L = cluster_layout(t.n_vars, cl, inc_off_host, &smem);
  static PerDevice smem_attr;  // one per instantiation: the opt-in above 48 KB, once per device
  if (smem > 48 * 1024 && smem_attr.get(0, [] {
        const bool ok = cudaFuncSetAttribute(k_pcg_cluster<Acc>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)CLUSTER_SMEM_LIMIT) == cudaSuccess;
        cudaGetLastError();
        return ok ? 1LL : 0LL;
      }) == 0)
    return -1;
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
