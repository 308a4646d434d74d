// Dense photometric + geometric term: association, residuals, Jacobians and the per-tile
// reduction of J^T W J and J^T W r (Sec. 4.3 E_photo / E_geo; Sec. 4.4: the dense system
// matrix is precomputed once per non-linear iteration with local reductions, then only a
// few scattered writes per pair).
//
// Work item = a tile of consecutive source pixels of one directed pair (i -> j).  Every
// thread walks the tile with a block-sized stride (coalesced source reads), evaluates its
// pixel entirely in registers and accumulates the pair's 30 partial sums in FP32 (only v / c
// sums: the source rotation Jacobian a = v x t - c is rebuilt per pair by the merge); the CTA
// then reduces them by a fixed-order tree (warp shuffles, then warps in order) and writes one
// record per tile.  Each run of sequential FP32 additions is at most ceil(tile/blockDim)
// long; everything above a tile is summed in FP64 (mixed precision) by the pair merge.
//
// The association decisions (target pixel, bilinear taps, validity, gates) are computed with
// explicitly rounded FP32 operations in a fixed order (no contraction), so a CPU restatement in
// IEEE FP32 takes the same decisions.  Residuals and Jacobians are free FP32 arithmetic.
//
// Everything is evaluated in the coordinates of the target camera j with the pair transform
// M = T_j^-1 T_i (y = R d + t); the merge rotates the sums to world coordinates with R_j.
#include "bf_internal.cuh"

namespace bf {

#define FM __fmul_rn
#define FA __fadd_rn
#define FS __fsub_rn

struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 cross3(V3 a, V3 b) {
  return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Accumulate one dense residual row (weight w, residual r, Jacobian [v x t - c, v, c, -v]).
__device__ __forceinline__ void accum_vc(float (&acc)[NPD], float w, float r, V3 v, V3 c) {
  const float wv0 = w * v.x, wv1 = w * v.y, wv2 = w * v.z;
  const float wc0 = w * c.x, wc1 = w * c.y, wc2 = w * c.z;
  acc[D_VV + 0] += wv0 * v.x; acc[D_VV + 1] += wv0 * v.y; acc[D_VV + 2] += wv0 * v.z;
  acc[D_VV + 3] += wv1 * v.y; acc[D_VV + 4] += wv1 * v.z; acc[D_VV + 5] += wv2 * v.z;
  acc[D_VC + 0] += wv0 * c.x; acc[D_VC + 1] += wv0 * c.y; acc[D_VC + 2] += wv0 * c.z;
  acc[D_VC + 3] += wv1 * c.x; acc[D_VC + 4] += wv1 * c.y; acc[D_VC + 5] += wv1 * c.z;
  acc[D_VC + 6] += wv2 * c.x; acc[D_VC + 7] += wv2 * c.y; acc[D_VC + 8] += wv2 * c.z;
  acc[D_CC + 0] += wc0 * c.x; acc[D_CC + 1] += wc0 * c.y; acc[D_CC + 2] += wc0 * c.z;
  acc[D_CC + 3] += wc1 * c.y; acc[D_CC + 4] += wc1 * c.z; acc[D_CC + 5] += wc2 * c.z;
  acc[D_GV + 0] += r * wv0; acc[D_GV + 1] += r * wv1; acc[D_GV + 2] += r * wv2;
  acc[D_GC + 0] += r * wc0; acc[D_GC + 1] += r * wc1; acc[D_GC + 2] += r * wc2;
}

// Fixed-order CTA reduction of N values; thread k < N writes out[k].
template <int BS, int N, typename Part>
__device__ __forceinline__ void cta_reduce_store(float (&acc)[N], Part *__restrict__ out) {
  constexpr int NW = BS / 32;
  __shared__ float red[NW][N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float v = acc[k];
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    Part s = (Part)red[0][threadIdx.x];
#pragma unroll
    for (int w = 1; w < NW; ++w) s += (Part)red[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

constexpr int DENSE_BS = 256;

template <int MODE, typename Part>
__global__ void __launch_bounds__(DENSE_BS, 4)
    k_dense(Tables t, FrameStore fs, Intr in, const float *__restrict__ pairM, Gates g, float w_geo, float w_photo,
            Part *__restrict__ part, int *__restrict__ assoc) {
  const int tile = blockIdx.x;
  const int d = t.tile_dp[tile];
  const int px0 = t.tile_px0[tile], px1 = t.tile_px1[tile];
  const int W = in.W, H = in.H;
  const long long HW = (long long)W * H;
  const float4 *__restrict__ As = fs.A + (long long)t.frame_slot[t.dp_src[d]] * HW;
  const float4 *__restrict__ Bs = fs.B + (long long)t.frame_slot[t.dp_src[d]] * HW;
  const float4 *__restrict__ At = fs.A + (long long)t.frame_slot[t.dp_dst[d]] * HW;
  const float4 *__restrict__ Bt = fs.B + (long long)t.frame_slot[t.dp_dst[d]] * HW;
  const float *M = pairM + (t.dp_pair[d] * 2 + t.dp_dir[d]) * 12;
  const float R00 = M[0], R01 = M[1], R02 = M[2], R10 = M[3], R11 = M[4], R12 = M[5];
  const float R20 = M[6], R21 = M[7], R22 = M[8], t0 = M[9], t1 = M[10], t2 = M[11];
  const float fx = in.fx, fy = in.fy, cx = in.cx, cy = in.cy;
  const float Wm1 = (float)(W - 1), Hm1 = (float)(H - 1), Wm3 = (float)(W - 3), Hm3 = (float)(H - 3);

  float acc[NPD];
#pragma unroll
  for (int k = 0; k < NPD; ++k) acc[k] = 0.f;

  float4 a_next = make_float4(0.f, 0.f, 0.f, 0.f);
  if (px0 + (int)threadIdx.x < px1) a_next = As[px0 + threadIdx.x];
  for (int px = px0 + threadIdx.x; px < px1; px += DENSE_BS) {
    int tgt = -1;
    const float4 a = a_next;  // prefetched one iteration ahead
    if (px + DENSE_BS < px1) a_next = As[px + DENSE_BS];
    const bool nvalid = (a.y != 0.f) || (a.z != 0.f) || (a.w != 0.f);
    if (a.x > 0.f && nvalid) {
      const int y = px / W, x = px - y * W;
      const float z = a.x;
      // ---- association decisions, explicitly rounded FP32 in a fixed order ----
      const float dx = FM(fs.kx[x], z), dy = FM(fs.ky[y], z), dz = z;
      const float Y0 = FA(FA(FA(FM(R00, dx), FM(R01, dy)), FM(R02, dz)), t0);
      const float Y1 = FA(FA(FA(FM(R10, dx), FM(R11, dy)), FM(R12, dz)), t1);
      const float Y2 = FA(FA(FA(FM(R20, dx), FM(R21, dy)), FM(R22, dz)), t2);
      if (Y2 > 0.f) {
        const float ux = FA(FM(fx, __fdiv_rn(Y0, Y2)), cx);
        const float uy = FA(FM(fy, __fdiv_rn(Y1, Y2)), cy);
        const float nxf = floorf(FA(ux, 0.5f)), nyf = floorf(FA(uy, 0.5f));
        const float bxf = floorf(ux), byf = floorf(uy);
        if (nxf >= 0.f && nxf <= Wm1 && nyf >= 0.f && nyf <= Hm1 && bxf >= 2.f && FA(bxf, 1.f) <= Wm3 &&
            byf >= 2.f && FA(byf, 1.f) <= Hm3) {
          const int tx = (int)nxf, ty = (int)nyf;
          const int tpx = ty * W + tx;
          const int bx = (int)bxf, by = (int)byf;
          // issue the target loads together: nearest (D, n) and the four (I, Ix, Iy) taps
          const float4 b = At[tpx];
          float4 c00, c01, c10, c11;
          if (MODE != MODE_ASSOC) {
            c00 = Bt[by * W + bx];
            c01 = Bt[by * W + bx + 1];
            c10 = Bt[(by + 1) * W + bx];
            c11 = Bt[(by + 1) * W + bx + 1];
          }
          const bool tnvalid = (b.y != 0.f) || (b.z != 0.f) || (b.w != 0.f);
          if (b.x > 0.f && tnvalid) {
            const float qx = FM(fs.kx[tx], b.x), qy = FM(fs.ky[ty], b.x), qz = b.x;
            const float ex = FS(Y0, qx), ey = FS(Y1, qy), ez = FS(Y2, qz);
            const float dist2 = FA(FA(FM(ex, ex), FM(ey, ey)), FM(ez, ez));
            const float m0 = FA(FA(FM(R00, a.y), FM(R01, a.z)), FM(R02, a.w));
            const float m1 = FA(FA(FM(R10, a.y), FM(R11, a.z)), FM(R12, a.w));
            const float m2 = FA(FA(FM(R20, a.y), FM(R21, a.z)), FM(R22, a.w));
            const float ndot = FA(FA(FM(m0, b.y), FM(m1, b.z)), FM(m2, b.w));
            if (dist2 < g.tau_d2 && ndot > g.tau_n) {
              tgt = tpx;
              if (MODE != MODE_ASSOC) {
                // ---- residuals and Jacobians (free FP32) in camera-j coordinates ----
                const float r_g = m0 * ex + m1 * ey + m2 * ez;
                const float wx = ux - bxf, wy = uy - byf;
                const float w00 = (1.f - wx) * (1.f - wy), w01 = wx * (1.f - wy);
                const float w10 = (1.f - wx) * wy, w11 = wx * wy;
                const float Ij = w00 * c00.x + w01 * c01.x + w10 * c10.x + w11 * c11.x;
                const float gxI = w00 * c00.y + w01 * c01.y + w10 * c10.y + w11 * c11.y;
                const float gyI = w00 * c00.z + w01 * c01.z + w10 * c10.z + w11 * c11.z;
                const float r_p = Bs[px].x - Ij;
                acc[D_E0] += r_g * r_g;
                acc[D_E1] += r_p * r_p;
                acc[D_CNT] += 1.f;
                if (MODE == MODE_ACCUM) {
                  // geometric: v = m, c = m x q
                  const V3 m{m0, m1, m2}, q{qx, qy, qz};
                  accum_vc(acc, w_geo, r_g, m, cross3(m, q));
                  // photometric: v = g = d r_p / d y = -grad I^T Jpi(y), c = g x y
                  const float iz = 1.f / Y2;
                  const float gfx = gxI * fx * iz, gfy = gyI * fy * iz;
                  const V3 gv{-gfx, -gfy, (gfx * Y0 + gfy * Y1) * iz};
                  accum_vc(acc, w_photo, r_p, gv, cross3(gv, V3{Y0, Y1, Y2}));
                }
              }
            }
          }
        }
      }
    }
    if (MODE == MODE_ASSOC) assoc[px] = tgt;
  }
  if (MODE != MODE_ASSOC) cta_reduce_store<DENSE_BS, NPD, Part>(acc, part + (long long)tile * NPD);
}

template <typename Part>
int launch_dense(int mode, const Tables &t, const FrameStore &fs, const Intr &in, const float *pairM, Gates g,
                  float w_geo, float w_photo, Part *part, int *assoc, cudaStream_t st) {
  if (t.n_tiles == 0) return 0;
  if (mode == MODE_ACCUM)
    k_dense<MODE_ACCUM, Part><<<t.n_tiles, DENSE_BS, 0, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  else if (mode == MODE_ENERGY)
    k_dense<MODE_ENERGY, Part><<<t.n_tiles, DENSE_BS, 0, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  else
    k_dense<MODE_ASSOC, Part><<<t.n_tiles, DENSE_BS, 0, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  return 1;
}

template int launch_dense<float>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates, float,
                                  float, float *, int *, cudaStream_t);
template int launch_dense<double>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates, float,
                                   float, double *, int *, cudaStream_t);

}  // namespace bf
