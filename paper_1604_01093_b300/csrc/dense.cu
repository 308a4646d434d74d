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
// The association decisions (target pixel, bilinear taps, validity, gates) are computed in FP32
// with explicitly rounded operations in a fixed order (products, sums and fused multiply-adds, no
// other contraction), so that every launch configuration takes the same decisions; they agree with
// the exact (FP64) association except where a value lies within FP32 rounding of its threshold.
// Residuals and Jacobians are free FP32 arithmetic.
//
// Everything is evaluated in the coordinates of the target camera j with the pair transform
// M = T_j^-1 T_i (y = R d + t); the merge rotates the sums to world coordinates with R_j.
#include "dense_eval.cuh"

namespace bf {

// Residency: 4 CTAs per SM (32 warps, 64 registers) for every storage: the accumulating pixel
// loop would like about 80 registers and spills 44-60 bytes at 64, but the extra warps hide more
// of the target gathers' latency (FP32 frames, 256-chunk 320x240 batch: 8.02 ms per launch at 4
// CTAs vs 8.18 ms at 3 without spills; BF16: 7.58 vs 8.18 ms).
template <int MODE, int KIND, bool COMP = false>
struct DenseOcc {
  // compensated sums hold twice the accumulators: 2 CTAs per SM (up to 128 registers, no spills)
  static constexpr int value = COMP ? 2 : 4;
};

// REC (debug): the association of every source pixel is also written to assoc[d * H * W + px].
// COMP: compensated per-thread sums (bf_solve_params.compensated).
template <int MODE, int KIND, typename Part, bool REC, bool COMP>
__global__ void __launch_bounds__(DENSE_BS, DenseOcc<MODE, KIND, COMP>::value)
    k_dense(Tables t, FrameStore fs, Intr in, const float *__restrict__ pairM, Gates g, float w_geo, float w_photo,
            Part *__restrict__ part, int *__restrict__ assoc) {
  extern __shared__ float ktab[];  // kx[W], ky[H]
  __shared__ float red[DENSE_BS / 32][NPD];
  dense_tile<MODE, KIND, Part, false, REC, COMP>(blockIdx.x, t, fs, in, pairM, g, w_geo, w_photo, part, assoc, ktab,
                                                 red);
}

template <int MODE, typename Part, bool REC, bool COMP>
static void dense_go(int kind, int n, size_t ks, cudaStream_t st, const Tables &t, const FrameStore &fs,
                     const Intr &in, const float *pairM, Gates g, float w_geo, float w_photo, Part *part, int *assoc) {
  if (kind == BF_STORE_BF16)
    k_dense<MODE, BF_STORE_BF16, Part, REC, COMP>
        <<<n, DENSE_BS, ks, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  else if (kind == BF_STORE_FP16)
    k_dense<MODE, BF_STORE_FP16, Part, REC, COMP>
        <<<n, DENSE_BS, ks, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  else
    k_dense<MODE, BF_STORE_FP32, Part, REC, COMP>
        <<<n, DENSE_BS, ks, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
}

// assoc: MODE_ASSOC's output; in the other modes nullptr, or (debug) the buffer that records the
// association of every source pixel of every directed pair (H * W ints per directed pair).
// comp: compensated per-thread sums (not combined with recording).
template <typename Part>
int launch_dense(int mode, const Tables &t, const FrameStore &fs, const Intr &in, const float *pairM, Gates g,
                  float w_geo, float w_photo, Part *part, int *assoc, cudaStream_t st, bool comp) {
  if (t.n_tiles == 0) return 0;
  const size_t ks = (size_t)(in.W + in.H) * sizeof(float);
  const int n = t.n_tiles, sg = fs.storage;
  if (mode == MODE_ACCUM) {
    if (assoc)
      dense_go<MODE_ACCUM, Part, true, false>(sg, n, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
    else if (comp)
      dense_go<MODE_ACCUM, Part, false, true>(sg, n, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, nullptr);
    else
      dense_go<MODE_ACCUM, Part, false, false>(sg, n, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, nullptr);
  } else if (mode == MODE_ENERGY) {
    if (assoc)
      dense_go<MODE_ENERGY, Part, true, false>(sg, n, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
    else if (comp)
      dense_go<MODE_ENERGY, Part, false, true>(sg, n, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, nullptr);
    else
      dense_go<MODE_ENERGY, Part, false, false>(sg, n, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, nullptr);
  } else {
    dense_go<MODE_ASSOC, Part, false, false>(sg, n, ks, st, t, fs, in, pairM, g, w_geo, w_photo, part, assoc);
  }
  return 1;
}

// ---------------------------------------------------------------------------------------------
// Target-staged variant.  At the paper's dense resolution (80x60) a frame's two planes take
// 2 x 76.8 KB (FP32; one 76.8 KB record plane with 16-bit storage), so one CTA holds its target
// frame in shared memory: a single thread issues the cp.async.bulk copies completing on an mbarrier, every thread waits (bounded), and all target
// reads of the CTA's source frames then hit shared memory instead of L1/L2.  Work item = one
// target frame with up to 6 of its source frames (a target's pairs split into near-equal items,
// launched largest first, so that the one-CTA-per-SM grid stays balanced); the CTA's 24 warps
// form 6 quads and each quad evaluates one directed pair at a time (fixed lane-strided pixel
// order, quad tree reduction, one partial per directed pair).
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

// Sum of N <= 32 per-thread values over a quad (4 warps, 128 threads): a reduce-scatter per warp
// (lane l ends with value l), then the 4 warp results in order by thread k < N, which writes
// out[k].
template <int N, typename Part>
__device__ __forceinline__ void quad_reduce_store(float (&acc)[N], float (*red)[N], int quad, Part *__restrict__ out) {
  static_assert(N <= 32, "at most 32 values");
  const int lane = threadIdx.x & 31, wq = (threadIdx.x >> 5) & 3;
  float v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = k < N ? acc[k] : 0.f;
  warp_reduce_scatter<32>(v);
  if (lane < N) red[wq][lane] = v[0];
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

template <int MODE, int KIND, typename Part, bool REC>
__global__ void __launch_bounds__(STG_BS, 1)
    k_dense_staged(Tables t, FrameStore fs, Intr in, const float *__restrict__ pairM, Gates g, float w_geo,
                   float w_photo, Part *__restrict__ part, int *__restrict__ err, int *__restrict__ rec) {
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
    // The copies did not land within the limit (at least half a second for 154 KB read from this
    // context's own frame store, in bounds by construction: only a stalled memory system gets here).
    // Report it and skip the evaluation, but keep the CTA, and with it its shared memory, alive
    // until the copies complete, for up to 16 more limits: a CTA that left with a bulk copy in
    // flight could have it land in the shared memory of the next CTA this SM runs.  If even that
    // wait gives up, the CTA leaves; the solve then fails with BF_ERR_TIMEOUT.
    if (threadIdx.x == 0) atomicExch(err, 1);
    for (int r = 0; r < 16 && !mbar_wait(barp, 0, STG_WAIT_LIMIT); ++r) {
    }
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
    DAcc acc;
    acc.zero();
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
        const int tgt = eval_pixel<MODE>(a, w.x, w.y, X, in, kx, ky, g, loadA, loadB, srcI, w_geo, w_photo, acc);
        if (REC) rec[(long long)d * HW + px] = tgt;
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
        const int tgt = eval_pixel<MODE>(unpack16_dn<KIND>(r), w.x, w.y, X, in, kx, ky, g, loadA, loadB, srcI, w_geo,
                                         w_photo, acc);
        if (REC) rec[(long long)d * HW + w.px] = tgt;
      }
    }
    float sums[NPD];
    acc.to_array(sums);
    quad_reduce_store<NPD, Part>(sums, red[quad], quad, part + (long long)d * NPD);
  }
}

template <int MODE, int KIND, typename Part, bool REC>
static void staged_go(int n, int smem, cudaStream_t st, const Tables &t, const FrameStore &fs, const Intr &in,
                      const float *pairM, Gates g, float w_geo, float w_photo, Part *part, int *err, int *rec) {
  static PerDevice attr;  // one per instantiation, set once per device
  attr.get(0, [] {
    cudaFuncSetAttribute(k_dense_staged<MODE, KIND, Part, REC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         STG_MAX_SMEM);
    return 1LL;
  });
  k_dense_staged<MODE, KIND, Part, REC><<<n, STG_BS, smem, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, err, rec);
}

template <int MODE, typename Part, bool REC>
static void staged_kind(int kind, int n, int smem, cudaStream_t st, const Tables &t, const FrameStore &fs,
                        const Intr &in, const float *pairM, Gates g, float w_geo, float w_photo, Part *part, int *err,
                        int *rec) {
  if (kind == BF_STORE_BF16)
    staged_go<MODE, BF_STORE_BF16, Part, REC>(n, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err, rec);
  else if (kind == BF_STORE_FP16)
    staged_go<MODE, BF_STORE_FP16, Part, REC>(n, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err, rec);
  else
    staged_go<MODE, BF_STORE_FP32, Part, REC>(n, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err, rec);
}

// rec: nullptr, or (debug) the buffer that records the association of every source pixel of every
// directed pair (H * W ints per directed pair).
template <typename Part>
int launch_dense_staged(int mode, const Tables &t, const FrameStore &fs, const Intr &in, const float *pairM, Gates g,
                        float w_geo, float w_photo, Part *part, int *err, int *rec, cudaStream_t st) {
  if (t.n_wi == 0) return 0;
  const int smem = dense_staged_smem(in.W, in.H, fs.storage);
  if (mode == MODE_ACCUM) {
    if (rec)
      staged_kind<MODE_ACCUM, Part, true>(fs.storage, t.n_wi, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part,
                                          err, rec);
    else
      staged_kind<MODE_ACCUM, Part, false>(fs.storage, t.n_wi, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part,
                                           err, nullptr);
  } else {
    if (rec)
      staged_kind<MODE_ENERGY, Part, true>(fs.storage, t.n_wi, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part,
                                           err, rec);
    else
      staged_kind<MODE_ENERGY, Part, false>(fs.storage, t.n_wi, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part,
                                            err, nullptr);
  }
  return 1;
}
template int launch_dense_staged<float>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates,
                                        float, float, float *, int *, int *, cudaStream_t);
template int launch_dense_staged<double>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates,
                                         float, float, double *, int *, int *, cudaStream_t);

template int launch_dense<float>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates, float,
                                  float, float *, int *, cudaStream_t, bool);
template int launch_dense<double>(int, const Tables &, const FrameStore &, const Intr &, const float *, Gates, float,
                                   float, double *, int *, cudaStream_t, bool);

}  // namespace bf
