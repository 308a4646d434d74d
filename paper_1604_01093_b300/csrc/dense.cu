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

// Relative pose of a directed pair (FP32): y = R d + t maps source-camera to target-camera points.
struct PairXf {
  float R00, R01, R02, R10, R11, R12, R20, R21, R22, t0, t1, t2;
};

__device__ __forceinline__ PairXf load_xf(const float *M) {
  return PairXf{M[0], M[1], M[2], M[3], M[4], M[5], M[6], M[7], M[8], M[9], M[10], M[11]};
}

// Evaluate source pixel (x, y) of a directed pair: association, gates and (MODE_ACCUM) the
// residual rows' contributions to acc.  a = source (D, n); loadA / loadB read the target's
// (D, n) and (I, Ix, Iy); srcI() gives the source pixel's I.  Returns the associated target
// pixel or -1.
template <int MODE, typename LA, typename LB, typename LI>
__device__ __forceinline__ int eval_pixel(const float4 a, int x, int y, const PairXf &X, const Intr &in,
                                          const float *kx, const float *ky, const Gates &g, LA loadA, LB loadB,
                                          LI srcI, float w_geo, float w_photo, float (&acc)[NPD]) {
  const bool nvalid = (a.y != 0.f) || (a.z != 0.f) || (a.w != 0.f);
  if (!(a.x > 0.f && nvalid)) return -1;
  const int W = in.W, H = in.H;
  const float z = a.x;
  // ---- association decisions, explicitly rounded FP32 in a fixed order ----
  const float dx = FM(kx[x], z), dy = FM(ky[y], z), dz = z;
  const float Y0 = FA(FA(FA(FM(X.R00, dx), FM(X.R01, dy)), FM(X.R02, dz)), X.t0);
  const float Y1 = FA(FA(FA(FM(X.R10, dx), FM(X.R11, dy)), FM(X.R12, dz)), X.t1);
  const float Y2 = FA(FA(FA(FM(X.R20, dx), FM(X.R21, dy)), FM(X.R22, dz)), X.t2);
  if (!(Y2 > 0.f)) return -1;
  const float iz = __frcp_rn(Y2);
  const float ux = FA(FM(in.fx, FM(Y0, iz)), in.cx);
  const float uy = FA(FM(in.fy, FM(Y1, iz)), in.cy);
  const float nxf = floorf(FA(ux, 0.5f)), nyf = floorf(FA(uy, 0.5f));
  const float bxf = floorf(ux), byf = floorf(uy);
  if (!(nxf >= 0.f && nxf <= (float)(W - 1) && nyf >= 0.f && nyf <= (float)(H - 1) && bxf >= 2.f &&
        FA(bxf, 1.f) <= (float)(W - 3) && byf >= 2.f && FA(byf, 1.f) <= (float)(H - 3)))
    return -1;
  const int tx = (int)nxf, ty = (int)nyf;
  const int bx = (int)bxf, by = (int)byf;
  const int tpx = ty * W + tx, b0 = by * W + bx;
  // issue the target reads together: nearest (D, n) and the four (I, Ix, Iy) taps
  const float4 b = loadA(tpx);
  float4 c00, c01, c10, c11;
  if (MODE != MODE_ASSOC) {
    c00 = loadB(b0);
    c01 = loadB(b0 + 1);
    c10 = loadB(b0 + W);
    c11 = loadB(b0 + W + 1);
  }
  const bool tnvalid = (b.y != 0.f) || (b.z != 0.f) || (b.w != 0.f);
  if (!(b.x > 0.f && tnvalid)) return -1;
  const float qx = FM(kx[tx], b.x), qy = FM(ky[ty], b.x), qz = b.x;
  const float ex = FS(Y0, qx), ey = FS(Y1, qy), ez = FS(Y2, qz);
  const float dist2 = FA(FA(FM(ex, ex), FM(ey, ey)), FM(ez, ez));
  const float m0 = FA(FA(FM(X.R00, a.y), FM(X.R01, a.z)), FM(X.R02, a.w));
  const float m1 = FA(FA(FM(X.R10, a.y), FM(X.R11, a.z)), FM(X.R12, a.w));
  const float m2 = FA(FA(FM(X.R20, a.y), FM(X.R21, a.z)), FM(X.R22, a.w));
  const float ndot = FA(FA(FM(m0, b.y), FM(m1, b.z)), FM(m2, b.w));
  if (!(dist2 < g.tau_d2 && ndot > g.tau_n)) return -1;
  if (MODE == MODE_ASSOC) return tpx;
  // ---- residuals and Jacobians (free FP32) in camera-j coordinates ----
  const float r_g = m0 * ex + m1 * ey + m2 * ez;
  const float wx = ux - bxf, wy = uy - byf;
  const float w00 = (1.f - wx) * (1.f - wy), w01 = wx * (1.f - wy);
  const float w10 = (1.f - wx) * wy, w11 = wx * wy;
  const float Ij = w00 * c00.x + w01 * c01.x + w10 * c10.x + w11 * c11.x;
  const float gxI = w00 * c00.y + w01 * c01.y + w10 * c10.y + w11 * c11.y;
  const float gyI = w00 * c00.z + w01 * c01.z + w10 * c10.z + w11 * c11.z;
  const float r_p = srcI() - Ij;
  acc[D_E0] += r_g * r_g;
  acc[D_E1] += r_p * r_p;
  acc[D_CNT] += 1.f;
  if (MODE == MODE_ACCUM) {
    // geometric: v = m, c = m x q
    const V3 m{m0, m1, m2}, q{qx, qy, qz};
    accum_vc(acc, w_geo, r_g, m, cross3(m, q));
    // photometric: v = g = d r_p / d y = -grad I^T Jpi(y), c = g x y
    const float gfx = gxI * in.fx * iz, gfy = gyI * in.fy * iz;
    const V3 gv{-gfx, -gfy, (gfx * Y0 + gfy * Y1) * iz};
    accum_vc(acc, w_photo, r_p, gv, cross3(gv, V3{Y0, Y1, Y2}));
  }
  return tpx;
}

// Pixel walk of one thread: px = start, start + stride, ... with (x, y) advanced incrementally.
struct PixWalk {
  int px, x, y, sx, sy, W;
  __device__ __forceinline__ PixWalk(int start, int stride, int W_) : px(start), W(W_) {
    y = start / W_;
    x = start - y * W_;
    sy = stride / W_;
    sx = stride - sy * W_;
  }
  __device__ __forceinline__ void next(int stride) {
    px += stride;
    x += sx;
    y += sy;
    if (x >= W) {
      x -= W;
      ++y;
    }
  }
};

constexpr int DENSE_BS = 256;

template <int MODE, int KIND, typename Part>
__global__ void __launch_bounds__(DENSE_BS, 4)
    k_dense(Tables t, FrameStore fs, Intr in, const float *__restrict__ pairM, Gates g, float w_geo, float w_photo,
            Part *__restrict__ part, int *__restrict__ assoc) {
  extern __shared__ float ktab[];  // kx[W], ky[H]
  const int tile = blockIdx.x;
  const int d = t.tile_dp[tile];
  const int px0 = t.tile_px0[tile], px1 = t.tile_px1[tile];
  const int W = in.W, H = in.H;
  const long long HW = (long long)W * H;
  const int ss = t.frame_slot[t.dp_src[d]], ts = t.frame_slot[t.dp_dst[d]];
  const PairXf X = load_xf(pairM + (t.dp_pair[d] * 2 + t.dp_dir[d]) * 12);
  float *kx = ktab, *ky = ktab + W;
  for (int k = threadIdx.x; k < W + H; k += DENSE_BS) ktab[k] = k < W ? fs.kx[k] : fs.ky[k - W];
  __syncthreads();
  float acc[NPD];
#pragma unroll
  for (int k = 0; k < NPD; ++k) acc[k] = 0.f;
  if (KIND == BF_STORE_FP32) {
    const float4 *__restrict__ As = fs.A + (long long)ss * HW;
    const float4 *__restrict__ Bs = fs.B + (long long)ss * HW;
    const float4 *__restrict__ At = fs.A + (long long)ts * HW;
    const float4 *__restrict__ Bt = fs.B + (long long)ts * HW;
    auto loadA = [&](int i) { return At[i]; };
    auto loadB = [&](int i) { return Bt[i]; };
    float4 a_next = make_float4(0.f, 0.f, 0.f, 0.f);
    if (px0 + (int)threadIdx.x < px1) a_next = As[px0 + threadIdx.x];
    for (PixWalk w(px0 + threadIdx.x, DENSE_BS, W); w.px < px1; w.next(DENSE_BS)) {
      const float4 a = a_next;  // prefetched one iteration ahead
      if (w.px + DENSE_BS < px1) a_next = As[w.px + DENSE_BS];
      const int px = w.px;
      auto srcI = [&]() { return Bs[px].x; };
      const int tgt = eval_pixel<MODE>(a, w.x, w.y, X, in, kx, ky, g, loadA, loadB, srcI, w_geo, w_photo, acc);
      if (MODE == MODE_ASSOC) assoc[w.px] = tgt;
    }
  } else {
    const uint4 *__restrict__ Ps = fs.P16 + (long long)ss * HW;
    const uint4 *__restrict__ Pt = fs.P16 + (long long)ts * HW;
    auto loadA = [&](int i) { return unpack16_dn<KIND>(Pt[i]); };
    auto loadB = [&](int i) { return unpack16_i<KIND>(Pt[i]); };
    uint4 r_next = make_uint4(0u, 0u, 0u, 0u);
    if (px0 + (int)threadIdx.x < px1) r_next = Ps[px0 + threadIdx.x];
    for (PixWalk w(px0 + threadIdx.x, DENSE_BS, W); w.px < px1; w.next(DENSE_BS)) {
      const uint4 r = r_next;
      if (w.px + DENSE_BS < px1) r_next = Ps[w.px + DENSE_BS];
      auto srcI = [&]() { return unpack16_i<KIND>(r).x; };
      const int tgt = eval_pixel<MODE>(unpack16_dn<KIND>(r), w.x, w.y, X, in, kx, ky, g, loadA, loadB, srcI, w_geo,
                                       w_photo, acc);
      if (MODE == MODE_ASSOC) assoc[w.px] = tgt;
    }
  }
  if (MODE != MODE_ASSOC) cta_reduce_store<DENSE_BS, NPD, Part>(acc, part + (long long)tile * NPD);
}

template <int MODE, typename Part>
static void dense_go(int kind, int n, size_t ks, cudaStream_t st, const Tables &t, const FrameStore &fs,
                     const Intr &in, const float *pairM, Gates g, float w_geo, float w_photo, Part *part, int *assoc) {
  if (kind == BF_STORE_BF16)
    k_dense<MODE, BF_STORE_BF16, Part><<<n, DENSE_BS, ks, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  else if (kind == BF_STORE_FP16)
    k_dense<MODE, BF_STORE_FP16, Part><<<n, DENSE_BS, ks, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  else
    k_dense<MODE, BF_STORE_FP32, Part><<<n, DENSE_BS, ks, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
}

template <typename Part>
int launch_dense(int mode, const Tables &t, const FrameStore &fs, const Intr &in, const float *pairM, Gates g,
                  float w_geo, float w_photo, Part *part, int *assoc, cudaStream_t st) {
  if (t.n_tiles == 0) return 0;
  const size_t ks = (size_t)(in.W + in.H) * sizeof(float);
  if (mode == MODE_ACCUM)
    dense_go<MODE_ACCUM>(fs.storage, t.n_tiles, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  else if (mode == MODE_ENERGY)
    dense_go<MODE_ENERGY>(fs.storage, t.n_tiles, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  else
    dense_go<MODE_ASSOC>(fs.storage, t.n_tiles, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  return 1;
}

// ---------------------------------------------------------------------------------------------
// Target-staged variant.  At the paper's dense resolution (80x60) a frame's two planes take
// 2 x 76.8 KB (FP32; one 76.8 KB record plane with 16-bit storage), so one CTA holds its target
// frame in shared memory: a single thread issues the cp.async.bulk copies completing on an mbarrier, every thread waits (bounded), and all target
// reads of the CTA's source frames then hit shared memory instead of L1/L2.  Work item = one
// target frame with a few of its source frames (the host uses 4, one per quad, so that the
// one-CTA-per-SM grid stays balanced); the CTA's 16 warps form 4 quads and each quad
// evaluates one directed pair at a time (fixed lane-strided pixel order, quad tree reduction,
// one partial per directed pair).
constexpr int STG_BS = 768;
constexpr int STG_QUADS = STG_BS / 128;
constexpr int STG_MAX_SMEM = 200 * 1024;
constexpr long long STG_WAIT_LIMIT = 1LL << 22;

// Dynamic shared memory of the staged kernel: the target frame (32 B/px FP32 planes, 16 B/px
// packed records) plus the ray tables.
int dense_staged_smem(int W, int H, int storage) {
  const long long b = (long long)W * H * (storage == BF_STORE_FP32 ? 32 : 16) + (W + H) * 4;
  return b > (1LL << 30) ? (1 << 30) : (int)b;
}
bool dense_staged_fits(int W, int H, int storage) { return dense_staged_smem(W, H, storage) + 4096 <= STG_MAX_SMEM; }

// Sum of N per-thread values over a quad (4 warps, 128 threads): warp trees, then the 4 warp
// results in order by thread k < N, which writes out[k].
template <int N, typename Part>
__device__ __forceinline__ void quad_reduce_store(float (&acc)[N], float (*red)[N], int quad, Part *__restrict__ out) {
  const int lane = threadIdx.x & 31, wq = (threadIdx.x >> 5) & 3;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float v = acc[k];
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    if (lane == 0) red[wq][k] = v;
  }
  asm volatile("bar.sync %0, 128;" ::"r"(1 + quad) : "memory");
  const int tq = threadIdx.x & 127;
  if (tq < N) {
    Part s = (Part)red[0][tq];
#pragma unroll
    for (int w = 1; w < 4; ++w) s += (Part)red[w][tq];
    out[tq] = s;
  }
  asm volatile("bar.sync %0, 128;" ::"r"(1 + quad) : "memory");  // red reused by the next pair
}

template <int MODE, int KIND, typename Part>
__global__ void __launch_bounds__(STG_BS, 1)
    k_dense_staged(Tables t, FrameStore fs, Intr in, const float *__restrict__ pairM, Gates g, float w_geo,
                   float w_photo, Part *__restrict__ part, int *__restrict__ err) {
  extern __shared__ __align__(128) float4 stg[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ float red[STG_QUADS][4][NPD];
  constexpr bool F32 = KIND == BF_STORE_FP32;
  const int W = in.W, H = in.H, HW = W * H;
  const int k0 = t.wi_off[blockIdx.x], k1 = t.wi_off[blockIdx.x + 1];
  const int tslot = t.frame_slot[t.dp_dst[t.sw_dp[k0]]];
  // FP32: the target's (D, n) and (I, Ix, Iy) planes; 16-bit: its packed records
  float4 *sA = stg, *sB = stg + HW;
  const uint4 *sP = (const uint4 *)stg;
  const unsigned barp = smem_u32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barp) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned bytes = (unsigned)HW * 16u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(barp), "r"((F32 ? 2u : 1u) * bytes)
                 : "memory");
    const void *src0 = F32 ? (const void *)(fs.A + (long long)tslot * HW) : (const void *)(fs.P16 + (long long)tslot * HW);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(sA)),
                 "l"(src0), "r"(bytes), "r"(barp)
                 : "memory");
    if (F32)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(sB)),
                   "l"(fs.B + (long long)tslot * HW), "r"(bytes), "r"(barp)
                   : "memory");
  }
  if (!mbar_wait(barp, 0, STG_WAIT_LIMIT)) {
    // the copies did not land within the limit: report, wait once more for them, then leave
    if (threadIdx.x == 0) atomicExch(err, 1);
    mbar_wait(barp, 0, STG_WAIT_LIMIT);
    return;
  }
  const int quad = threadIdx.x >> 7, tq = threadIdx.x & 127;
  float *kx = (float *)(stg + (F32 ? 2 : 1) * HW), *ky = kx + W;
  for (int k = threadIdx.x; k < W + H; k += STG_BS) kx[k] = k < W ? fs.kx[k] : fs.ky[k - W];
  __syncthreads();
  for (int k = k0 + quad; k < k1; k += STG_QUADS) {
    const int d = t.sw_dp[k];
    const long long so = (long long)t.frame_slot[t.dp_src[d]] * HW;
    const PairXf X = load_xf(pairM + (t.dp_pair[d] * 2 + t.dp_dir[d]) * 12);
    float acc[NPD];
#pragma unroll
    for (int q = 0; q < NPD; ++q) acc[q] = 0.f;
    if (F32) {
      const float4 *__restrict__ As = fs.A + so;
      const float4 *__restrict__ Bs = fs.B + so;
      auto loadA = [&](int i) { return sA[i]; };
      auto loadB = [&](int i) { return sB[i]; };
      float4 a_next = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tq < HW) a_next = As[tq];
      for (PixWalk w(tq, 128, W); w.px < HW; w.next(128)) {
        const float4 a = a_next;
        if (w.px + 128 < HW) a_next = As[w.px + 128];
        const int px = w.px;
        auto srcI = [&]() { return Bs[px].x; };
        eval_pixel<MODE>(a, w.x, w.y, X, in, kx, ky, g, loadA, loadB, srcI, w_geo, w_photo, acc);
      }
    } else {
      const uint4 *__restrict__ Ps = fs.P16 + so;
      auto loadA = [&](int i) { return unpack16_dn<KIND>(sP[i]); };
      auto loadB = [&](int i) { return unpack16_i<KIND>(sP[i]); };
      uint4 r_next = make_uint4(0u, 0u, 0u, 0u);
      if (tq < HW) r_next = Ps[tq];
      for (PixWalk w(tq, 128, W); w.px < HW; w.next(128)) {
        const uint4 r = r_next;
        if (w.px + 128 < HW) r_next = Ps[w.px + 128];
        auto srcI = [&]() { return unpack16_i<KIND>(r).x; };
        eval_pixel<MODE>(unpack16_dn<KIND>(r), w.x, w.y, X, in, kx, ky, g, loadA, loadB, srcI, w_geo, w_photo, acc);
      }
    }
    quad_reduce_store<NPD, Part>(acc, red[quad], quad, part + (long long)d * NPD);
  }
}

template <int MODE, int KIND, typename Part>
static void staged_go(int n, int smem, cudaStream_t st, const Tables &t, const FrameStore &fs, const Intr &in,
                      const float *pairM, Gates g, float w_geo, float w_photo, Part *part, int *err) {
  static bool attr_set = false;  // one flag per instantiation
  if (!attr_set) {
    cudaFuncSetAttribute(k_dense_staged<MODE, KIND, Part>, cudaFuncAttributeMaxDynamicSharedMemorySize, STG_MAX_SMEM);
    attr_set = true;
  }
  k_dense_staged<MODE, KIND, Part><<<n, STG_BS, smem, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, err);
}

template <int MODE, typename Part>
static void staged_kind(int kind, int n, int smem, cudaStream_t st, const Tables &t, const FrameStore &fs,
                        const Intr &in, const float *pairM, Gates g, float w_geo, float w_photo, Part *part, int *err) {
  if (kind == BF_STORE_BF16)
    staged_go<MODE, BF_STORE_BF16, Part>(n, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
  else if (kind == BF_STORE_FP16)
    staged_go<MODE, BF_STORE_FP16, Part>(n, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
  else
    staged_go<MODE, BF_STORE_FP32, Part>(n, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
}

template <typename Part>
int launch_dense_staged(int mode, const Tables &t, const FrameStore &fs, const Intr &in, const float *pairM, Gates g,
                        float w_geo, float w_photo, Part *part, int *err, cudaStream_t st) {
  if (t.n_wi == 0) return 0;
  const int smem = dense_staged_smem(in.W, in.H, fs.storage);
  if (mode == MODE_ACCUM)
    staged_kind<MODE_ACCUM, Part>(fs.storage, t.n_wi, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
  else
    staged_kind<MODE_ENERGY, Part>(fs.storage, t.n_wi, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
  return 1;
}
template int launch_dense_staged<float>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates,
                                        float, float, float *, int *, cudaStream_t);
template int launch_dense_staged<double>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates,
                                         float, float, double *, int *, cudaStream_t);

template int launch_dense<float>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates, float,
                                  float, float *, int *, cudaStream_t);
template int launch_dense<double>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates, float,
                                   float, double *, int *, cudaStream_t);

}  // namespace bf
