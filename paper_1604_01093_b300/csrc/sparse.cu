// Sparse feature term (Sec. 4.3, E_sparse = sum ||T_i p_ik - T_j p_jl||^2) and the residual
// maximum of Sec. 4.4.1.
//
// Work item = one segment of correspondences of an unordered pair (a, b) (a pair holds one
// segment per bf_add_correspondences call), evaluated by one warp (4 per CTA, no barrier): at
// 64-256 correspondences per segment the per-segment reduction of 57 sums dominates, so a warp
// reduce-scatter (one shuffle per value kept per step) replaces a CTA tree.  The three residual
// rows of a correspondence are
// evaluated in camera-b coordinates, r' = R_ba p + t_ba - q with M = T_b^-1 T_a; in the
// [a, v, c, -v] form of the partial sums row k has v = e_k, a = (R_ba p) x e_k, c = e_k x q.
// (Rotating all three rows by R_b leaves J^T J and J^T r unchanged, so this equals the
// world-frame Jacobian -[R_a p]_x, I, [R_b q]_x, -I.)  The per-segment sums are reduced in a
// fixed order.
//
// The paper applies the sparse term matrix-free inside PCG (J p, then J^T (J p)); by default
// its 6x6 pair blocks are formed here once per Gauss-Newton iteration, like the dense term,
// because a pair's block costs 72 values while its correspondences are re-read every PCG
// iteration otherwise.  The matrix-free scheme is the BF_SPARSE_MATFREE option (mf_pair in
// solve_eval.cuh); these sums then still give the right-hand side, the preconditioner's diagonal
// blocks and the energy.
#include "sparse_eval.cuh"

namespace bf {

template <int MODE, typename Part>
__global__ void __launch_bounds__(SPARSE_BS)
    k_sparse(Tables t, const float4 *__restrict__ P, const float4 *__restrict__ Q, const float *__restrict__ pairM,
             float w_sparse, Part *__restrict__ part, float *__restrict__ seg_rmax, int *__restrict__ seg_rarg) {
  const int s = blockIdx.x * (SPARSE_BS / 32) + (threadIdx.x >> 5);
  if (s < t.n_segs) sparse_seg<MODE, Part>(s, t, P, Q, pairM, w_sparse, part, seg_rmax, seg_rarg);
}

template <typename Part>
int launch_sparse(int mode, const Tables &t, const float4 *P, const float4 *Q, const float *pairM, float w_sparse,
                   Part *part, float *seg_rmax, int *seg_rarg, cudaStream_t st) {
  if (t.n_segs == 0) return 0;
  const int grid = (t.n_segs + SPARSE_BS / 32 - 1) / (SPARSE_BS / 32);
  if (mode == MODE_ACCUM)
    k_sparse<MODE_ACCUM, Part><<<grid, SPARSE_BS, 0, st>>>(t, P, Q, pairM, w_sparse, part, seg_rmax, seg_rarg);
  else
    k_sparse<MODE_ENERGY, Part><<<grid, SPARSE_BS, 0, st>>>(t, P, Q, pairM, w_sparse, part, seg_rmax, seg_rarg);
  return 1;
}

template int launch_sparse<float>(int, const Tables &, const float4 *, const float4 *, const float *, float, float *,
                                   float *, int *, cudaStream_t);
template int launch_sparse<double>(int, const Tables &, const float4 *, const float4 *, const float *, float,
                                    double *, float *, int *, cudaStream_t);

}  // namespace bf
