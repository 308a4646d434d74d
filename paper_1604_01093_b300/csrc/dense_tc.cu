// Tensor-core form of the dense term's per-tile sums (an option, bf_solve_params.dense_tc).
//
// The sums the tiled dense kernel forms per thread with FP32 fused multiply-adds (Sec. 4.4: the
// dense J^T W J and J^T W r of a pair, here its 27 v / c sums and the residual terms) are a
// contraction over residual rows: with f = (v, c, r, 0) the 8-wide row of a residual and w its
// weight, the pair's sums are the upper triangle of G = sum_rows (w f) f^T.  Here the rows go to
// shared memory and the 5th-generation tensor cores (tcgen05.mma, kind::tf32, one issuing
// thread, FP32 accumulators in tensor memory) sum them:
//
//   * a CTA of 256 threads evaluates 256 source pixels per iteration with the same device code
//     as the CUDA-core kernels (eval_pixel: association, gates, residuals, Jacobians); each
//     pixel gives a geometric and a photometric row (zero rows where it has no association);
//   * warp s (of 8) stages its 64 rows as "subset" s: rows 8s..8s+7 of a 64 x 8 A tile (w f,
//     K-major: K = residual rows) and of a 64 x 8 B tile (f); one MMA of M = N = 64, K = 8
//     takes 8 rows of every subset, 8 MMAs an iteration; D = A B^T accumulates in a 64 x 64
//     FP32 tensor-memory tile whose 8 diagonal 8 x 8 blocks are the subsets' partial G (the
//     off-diagonal blocks, 7/8 of the MMA work, are products of different pixels and unused:
//     the tensor core's smallest M is 64, eight times the 8-wide rows);
//   * passes = 1: operands rounded to TF32 (10-bit mantissa); passes = 3: each operand split
//     x = hi + lo into two TF32 parts and D += lo_A hi_B + hi_A lo_B + hi_A hi_B, which restores
//     close to FP32 products;
//   * the staging buffer is single: before a warp overwrites it, every thread waits (bounded) on
//     the mbarrier the previous iteration's MMAs complete (tcgen05.commit), so the MMAs of one
//     iteration overlap the next iteration's pixel evaluation;
//   * each iteration's MMAs start a fresh accumulator; after they complete, warps 0-3 read its
//     diagonal blocks (tcgen05.ld) and add them to per-thread FP32 sums: the tensor core's own
//     FP32 accumulation, which does not round every addition to nearest, then only sums runs of
//     64 rows (x passes) instead of a whole tile's (over a 38 400-pixel tile it erred by ~5e-5
//     of the largest sum);
//   * at the end the subsets' blocks are summed in subset order and written as the tile's
//     partial record (the energies and the residual count are summed on the CUDA cores as in
//     k_dense).
//
// The association decisions are those of k_dense (same device functions), so the two options
// differ only in how the sums are rounded.  Every wait is bounded: a wait that gives up sets the
// error word, waits (bounded) for the MMAs in flight, frees the tensor memory and returns.
#include "dense_eval.cuh"

namespace bf {

namespace {

constexpr int TC_BS = 256;    // threads; warp s stages subset s
constexpr int TC_COLS = 64;   // tensor-memory columns of the 64 x 64 FP32 accumulator
constexpr int TC_TILE = 2112; // bytes of one 64 x 8 TF32 operand tile (2048 + 64 of padding)
constexpr int TC_KB = 8;      // MMAs (8 rows of each subset) per iteration
constexpr long long TC_WAIT_LIMIT = 1LL << 22;

template <int PASSES>
struct TcLayout {
  // one MMA's operands: A_hi, B_hi (and A_lo, B_lo), then 16 bytes that move the next MMA's
  // tiles four banks along, so that the eight MMAs' stores of a warp fall in different banks
  static constexpr int tiles = PASSES == 1 ? 2 : 4;
  static constexpr int slot = tiles * TC_TILE + 16;
  static constexpr int bytes = TC_KB * slot;
};

// Byte offset of element (m, k) of a 64 x 8 TF32 tile in the canonical K-major layout without
// swizzle: core matrices of 8 rows x 16 bytes (128 contiguous bytes); neighbours along M 128
// bytes apart (the descriptor's stride offset), the two along K TC_LBO bytes apart (its
// leading-dimension offset).  TC_LBO = 1024 + 64: the half of a warp that stores at once (lanes
// l and l + 1 of 16: four MMA slots x two K core matrices x two 8-byte halves) hits 16 distinct
// 8-byte bank pairs, so the 64-bit stores run without bank conflicts.
constexpr unsigned TC_LBO = 1088, TC_SBO = 128;
__device__ __forceinline__ int tc_off(int m, int k) {
  return (m >> 3) * TC_SBO + (k >> 2) * TC_LBO + (m & 7) * 16 + (k & 3) * 4;
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension byte offset and
// stride byte offset in 16-byte units, descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ unsigned long long tc_sdesc(unsigned saddr) {
  return (unsigned long long)((saddr >> 4) & 0x3FFFu) | ((unsigned long long)(TC_LBO >> 4) << 16) |
         ((unsigned long long)(TC_SBO >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor: dense, D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr unsigned TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((64u >> 4) << 24);

__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor core's (async-proxy) reads
__device__ __forceinline__ void tc_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// whole warp: allocate the accumulator's columns (address written to shared memory)
__device__ __forceinline__ void tc_alloc(unsigned dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(TC_COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(unsigned taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_COLS) : "memory");
}

// whole warp: 8 consecutive columns of the warp's 32 tensor-memory lanes (thread l: lane l),
// complete on return
__device__ __forceinline__ void tc_ld8(unsigned taddr, float (&v)[8]) {
  unsigned r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5); v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

// FP32 -> TF32, round to nearest (ties away), low 13 mantissa bits zero
__device__ __forceinline__ float tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// The accumulator row of D held by tensor-memory lane L (M = 64, one CTA): rows 16w..16w+15 in
// lanes 0-15 of sub-partition w; -1 for the lanes that hold none.
__device__ __forceinline__ int tc_row_of_lane(int L) { return (L & 31) < 16 ? (L >> 5) * 16 + (L & 15) : -1; }

// Stage one thread's two rows (q = 0 at K position kk0, q = 1 at kk0 + 1 of MMA slot kb) as
// feature rows 8s..8s+7 of the A (w f) and B (f) tiles.  rows(a, q) gives (A, B) of feature a of
// row q.
template <int PASSES, typename R>
__device__ __forceinline__ void tc_stage(char *ops, int s, int kb, int kk0, R rows) {
  char *slot = ops + kb * TcLayout<PASSES>::slot;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int off = tc_off(8 * s + a, kk0);  // kk0 even: an 8-byte aligned pair (q = 0, 1)
    const float2 r0 = rows(a, 0), r1 = rows(a, 1);
    const float a0 = tf32_rna(r0.x), a1 = tf32_rna(r1.x);
    const float b0 = tf32_rna(r0.y), b1 = tf32_rna(r1.y);
    *(float2 *)(slot + off) = make_float2(a0, a1);
    *(float2 *)(slot + TC_TILE + off) = make_float2(b0, b1);
    if (PASSES == 3) {
      *(float2 *)(slot + 2 * TC_TILE + off) = make_float2(tf32_rna(__fsub_rn(r0.x, a0)), tf32_rna(__fsub_rn(r1.x, a1)));
      *(float2 *)(slot + 3 * TC_TILE + off) = make_float2(tf32_rna(__fsub_rn(r0.y, b0)), tf32_rna(__fsub_rn(r1.y, b1)));
    }
  }
}

// One iteration's MMAs (issued by one thread), then the commit that arrives on bar when they
// have completed.  fresh: the iteration's first MMA overwrites D instead of adding to it.
template <int PASSES>
__device__ __forceinline__ void tc_issue(unsigned taddr, unsigned ops_s, bool fresh, unsigned bar) {
  tc_fence_after();
#pragma unroll 1
  for (int kb = 0; kb < TC_KB; ++kb) {
    const unsigned s0 = ops_s + kb * TcLayout<PASSES>::slot;
    const unsigned long long ah = tc_sdesc(s0), bh = tc_sdesc(s0 + TC_TILE);
    unsigned acc = fresh && kb == 0 ? 0u : 1u;
    if (PASSES == 3) {
      tc_mma(taddr, tc_sdesc(s0 + 2 * TC_TILE), bh, acc);  // lo_A hi_B
      acc = 1u;
      tc_mma(taddr, ah, tc_sdesc(s0 + 3 * TC_TILE), acc);  // hi_A lo_B
    }
    tc_mma(taddr, ah, bh, acc);  // hi_A hi_B
  }
  tc_commit(bar);
}

// eval_pixel's accumulator for this kernel: the pixel's (at most two) residual rows are kept for
// staging; the energies and the residual count are summed per thread as DAcc does.
struct TcRows {
  float e0, e1, cnt;
  float f[2][7], w[2];
  bool second;
  __device__ __forceinline__ void zero() { e0 = e1 = cnt = 0.f; }
  __device__ __forceinline__ void begin() {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      w[q] = 0.f;
#pragma unroll
      for (int a = 0; a < 7; ++a) f[q][a] = 0.f;
    }
    second = false;
  }
  __device__ __forceinline__ void add_energy(float r_g, float r_p) {
    e0 = __fmaf_rn(r_g, r_g, e0);
    e1 = __fmaf_rn(r_p, r_p, e1);
    cnt += 1.f;
  }
  __device__ __forceinline__ void add_row(float wt, float r, V3 v, V3 c) {
    const float u[7] = {v.x, v.y, v.z, c.x, c.y, c.z, r};
    if (!second) {
#pragma unroll
      for (int a = 0; a < 7; ++a) f[0][a] = u[a];
      w[0] = wt;
      second = true;
    } else {
#pragma unroll
      for (int a = 0; a < 7; ++a) f[1][a] = u[a];
      w[1] = wt;
    }
  }
  // feature a of row q: A = w f_a (the product DAcc forms first, w u_i), B = f_a; feature 7 is 0
  __device__ __forceinline__ float2 operand(int a, int q) const {
    if (a == 7) return make_float2(0.f, 0.f);
    return make_float2(__fmul_rn(w[q], f[q][a]), f[q][a]);
  }
};

// Shared state of a CTA besides the operand tiles.
struct TcSmem {
  unsigned long long bar;
  unsigned taddr;
  int abort;
  float gpart[8][8][8];  // [subset][a][b]: the diagonal blocks
  float ered[TC_BS / 32][3];
};

// Wait until the MMAs committed for iteration `it` have completed (bounded).
__device__ __forceinline__ bool tc_wait_it(unsigned bar, int it) { return mbar_wait(bar, (unsigned)(it & 1), TC_WAIT_LIMIT); }

// Warps 0-3: add this iteration's diagonal blocks of D to the thread's running FP32 sums.  Lane
// l < 16 of warp w holds row r = 16w + l, i.e. row a = r % 8 of subset s = r / 8, whose block
// is columns 8s..8s+7 (one 8-column load for each of the warp's two subsets); other lanes none.
// Each MMA run is one iteration (64 rows of a subset, times the passes), so the tensor core's
// FP32 accumulation only sees short runs and the runs are summed with rounded FP32 additions.
__device__ __forceinline__ void tc_fold(unsigned taddr, int warp, int lane, float (&gacc)[8]) {
  float v0[8], v1[8];
  const unsigned base = taddr + ((unsigned)(32 * warp) << 16) + 16 * warp;
  tc_ld8(base, v0);      // columns of subset 2w
  tc_ld8(base + 8, v1);  // columns of subset 2w + 1
#pragma unroll
  for (int b = 0; b < 8; ++b) gacc[b] = __fadd_rn(gacc[b], lane < 8 ? v0[b] : v1[b]);
}

// After the last commit (it_last, or none when it_last < 0): fold the last run, write the
// threads' sums to sm.gpart, then free the tensor memory.  ok = false: an earlier wait gave up;
// only wait (bounded) for the MMAs in flight and free.
__device__ __forceinline__ void tc_finish(TcSmem &sm, unsigned bar, int it_last, bool ok, int *err,
                                          float (&gacc)[8]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (it_last >= 0 && !tc_wait_it(bar, it_last)) {
    ok = false;
    if (threadIdx.x == 0) atomicExch(err, 1);
  }
  tc_fence_after();
  if (warp < 4) {
    if (ok && it_last >= 0) tc_fold(sm.taddr, warp, lane, gacc);
    if (lane < 16) {
      const int r = tc_row_of_lane(32 * warp + lane);
#pragma unroll
      for (int b = 0; b < 8; ++b) sm.gpart[r >> 3][r & 7][b] = gacc[b];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(sm.taddr);
  }
}

__device__ __forceinline__ void tc_setup(TcSmem &sm) {
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sm.abort = 0;
  }
  if (warp == 0) tc_alloc(smem_u32(&sm.taddr));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

}  // namespace

// One CTA per tile of the tiled decomposition (the tiles of k_dense), MODE_ACCUM.
template <int KIND, typename Part, int PASSES>
__global__ void __launch_bounds__(TC_BS, 3)
    k_dense_tc(Tables t, FrameStore fs, Intr in, const float *__restrict__ pairM, Gates g, float w_geo,
               float w_photo, Part *__restrict__ part, int *err) {
  extern __shared__ __align__(128) char tc_dyn[];
  __shared__ TcSmem sm;
  char *ops = tc_dyn;
  float *ktab = (float *)(tc_dyn + TcLayout<PASSES>::bytes);
  const int tile = blockIdx.x;
  const int d = t.tile_dp[tile];
  const int px0 = t.tile_px0[tile], px1 = t.tile_px1[tile];
  const int W = in.W, H = in.H;
  const long long HW = (long long)W * H;
  const int ss = t.frame_slot[t.dp_src[d]], ts = t.frame_slot[t.dp_dst[d]];
  const PairXf X = load_xf<false>(pairM + (t.dp_pair[d] * 2 + t.dp_dir[d]) * 12);
  float *kx = ktab, *ky = ktab + W;
  for (int k = threadIdx.x; k < W + H; k += TC_BS) ktab[k] = k < W ? fs.kx[k] : fs.ky[k - W];
  tc_setup(sm);
  const unsigned bar = smem_u32(&sm.bar), ops_s = smem_u32(ops);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kb = lane >> 2, kk0 = 2 * (lane & 3);
  TcRows acc;
  acc.zero();
  float gacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int n_it = (px1 - px0 + TC_BS - 1) / TC_BS;
  bool ok = true;
  int it = 0;
  PixWalk w(px0 + threadIdx.x, TC_BS, W);
  for (; it < n_it; ++it, w.next(TC_BS)) {
    acc.begin();
    if (w.px < px1) {
      if (KIND == BF_STORE_FP32) {
        const float4 *__restrict__ At = fs.A + (long long)ts * HW;
        const float4 *__restrict__ Bt = fs.B + (long long)ts * HW;
        const float4 *__restrict__ Bs = fs.B + (long long)ss * HW;
        const int px = w.px;
        eval_pixel<MODE_ACCUM>(fs.A[(long long)ss * HW + px], w.x, w.y, X, in, kx, ky, g,
                               [&](int i) { return At[i]; }, [&](int i) { return Bt[i]; },
                               [&]() { return Bs[px].x; }, w_geo, w_photo, acc);
      } else {
        const uint4 *__restrict__ Pt = fs.P16 + (long long)ts * HW;
        const uint4 r = fs.P16[(long long)ss * HW + w.px];
        eval_pixel<MODE_ACCUM>(unpack16_dn<KIND>(r), w.x, w.y, X, in, kx, ky, g,
                               [&](int i) { return unpack16_dn<KIND>(Pt[i]); },
                               [&](int i) { return unpack16_i<KIND>(Pt[i]); },
                               [&]() { return unpack16_i<KIND>(r).x; }, w_geo, w_photo, acc);
      }
    }
    // the previous iteration's MMAs read the staging buffer and wrote D: wait for them, fold D
    // into the running sums, then overwrite the buffer
    if (it > 0) {
      if (!tc_wait_it(bar, it - 1)) {
        sm.abort = 1;
      } else {
        tc_fence_after();
        if (warp < 4) tc_fold(sm.taddr, warp, lane, gacc);
      }
    }
    tc_stage<PASSES>(ops, warp, kb, kk0, [&](int a, int q) { return acc.operand(a, q); });
    tc_fence_smem();
    tc_fence_before();
    __syncthreads();
    if (sm.abort) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) tc_issue<PASSES>(sm.taddr, ops_s, true, bar);
  }
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  // it iterations issued (when the loop broke, the one that aborted issued nothing)
  tc_finish(sm, bar, it - 1, ok, err, gacc);
  // energies and count: warp sums, then warps in order
  float e[3] = {acc.e0, acc.e1, acc.cnt};
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e[k] += __shfl_down_sync(0xffffffffu, e[k], o);
  if (lane == 0) {
    sm.ered[warp][0] = e[0];
    sm.ered[warp][1] = e[1];
    sm.ered[warp][2] = e[2];
  }
  __syncthreads();
  if (!ok) return;
  // the record: the upper triangle of G = sum over subsets of the diagonal blocks (subset order)
  Part *out = part + (long long)tile * NPD;
  const int k = threadIdx.x;
  auto G = [&](int a, int b) {
    float s = sm.gpart[0][a][b];
#pragma unroll
    for (int q = 1; q < 8; ++q) s += sm.gpart[q][a][b];
    return s;
  };
  if (k < 6) {
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    out[D_VV + k] = (Part)G(ia[k], ib[k]);
    out[D_CC + k] = (Part)G(3 + ia[k], 3 + ib[k]);
  } else if (k < 15) {
    const int j = k - 6;
    out[D_VC + j] = (Part)G(j / 3, 3 + j % 3);
  } else if (k < 18) {
    out[D_GV + (k - 15)] = (Part)G(k - 15, 6);
  } else if (k < 21) {
    out[D_GC + (k - 18)] = (Part)G(3 + k - 18, 6);
  } else if (k < 24) {
    float s = sm.ered[0][k - 21];
#pragma unroll
    for (int q = 1; q < TC_BS / 32; ++q) s += sm.ered[q][k - 21];
    out[(k == 21 ? D_E0 : k == 22 ? D_E1 : D_CNT)] = (Part)s;
  }
}

// Debug probe of the tensor-core path: rows given as inputs instead of evaluated pixels.  fa, fb:
// [8 subsets][n_rows][8] (A = w f and B = f rows), n_rows a multiple of 64; one CTA stages them
// exactly as k_dense_tc does (warp s, lane l: rows 2l and 2l + 1 of each block of 64) and dumps
// the whole accumulator: out[lane][column], 128 lanes x 64 columns (lanes without rows hold
// whatever the tensor memory held).
template <int PASSES>
__global__ void __launch_bounds__(TC_BS, 1)
    k_tc_probe(const float *__restrict__ fa_in, const float *__restrict__ fb_in, int n_rows, float *out, int *err) {
  extern __shared__ __align__(128) char tc_dyn[];
  __shared__ TcSmem sm;
  char *ops = tc_dyn;
  tc_setup(sm);
  const unsigned bar = smem_u32(&sm.bar), ops_s = smem_u32(ops);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kb = lane >> 2, kk0 = 2 * (lane & 3);
  const int n_it = n_rows / 64;
  bool ok = true;
  int it = 0;
  for (; it < n_it; ++it) {
    const long long row0 = ((long long)warp * n_rows + it * 64 + 2 * lane) * 8;
    if (it > 0 && !tc_wait_it(bar, it - 1)) sm.abort = 1;
    tc_stage<PASSES>(ops, warp, kb, kk0, [&](int a, int q) {
      return make_float2(fa_in[row0 + 8 * q + a], fb_in[row0 + 8 * q + a]);
    });
    tc_fence_smem();
    __syncthreads();
    if (sm.abort) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) tc_issue<PASSES>(sm.taddr, ops_s, it == 0, bar);
  }
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  if (it > 0 && !tc_wait_it(bar, it - 1)) {
    ok = false;
    if (threadIdx.x == 0) atomicExch(err, 1);
  }
  tc_fence_after();
  if (ok && warp < 4) {
#pragma unroll
    for (int cb = 0; cb < 8; ++cb) {
      float v[8];
      tc_ld8(sm.taddr + ((unsigned)(32 * warp) << 16) + 8 * cb, v);
#pragma unroll
      for (int b = 0; b < 8; ++b) out[(32 * warp + lane) * 64 + 8 * cb + b] = v[b];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(sm.taddr);
  }
}

template <int KIND, typename Part, int PASSES>
static int tc_go(int n, size_t smem, cudaStream_t st, const Tables &t, const FrameStore &fs, const Intr &in,
                 const float *pairM, Gates g, float w_geo, float w_photo, Part *part, int *err) {
  static PerDevice attr;  // the dynamic shared memory limit, set once per device and size
  const long long ok = attr.get((long long)smem, [smem] {
    return (long long)(cudaFuncSetAttribute(k_dense_tc<KIND, Part, PASSES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem) == cudaSuccess);
  });
  if (!ok) return -1;
  k_dense_tc<KIND, Part, PASSES><<<n, TC_BS, smem, st>>>(t, fs, in, pairM, g, w_geo, w_photo, part, err);
  return 1;
}

template <typename Part, int PASSES>
static int tc_kind(int n, size_t smem, cudaStream_t st, const Tables &t, const FrameStore &fs, const Intr &in,
                   const float *pairM, Gates g, float w_geo, float w_photo, Part *part, int *err) {
  if (fs.storage == BF_STORE_BF16)
    return tc_go<BF_STORE_BF16, Part, PASSES>(n, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
  if (fs.storage == BF_STORE_FP16)
    return tc_go<BF_STORE_FP16, Part, PASSES>(n, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
  return tc_go<BF_STORE_FP32, Part, PASSES>(n, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
}

template <typename Part>
int launch_dense_tc(const Tables &t, const FrameStore &fs, const Intr &in, const float *pairM, Gates g, float w_geo,
                    float w_photo, Part *part, int *err, int passes, cudaStream_t st) {
  if (t.n_tiles == 0) return 0;
  if (passes == 1) {
    const size_t smem = TcLayout<1>::bytes + (size_t)(in.W + in.H) * sizeof(float);
    return tc_kind<Part, 1>(t.n_tiles, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
  }
  const size_t smem = TcLayout<3>::bytes + (size_t)(in.W + in.H) * sizeof(float);
  return tc_kind<Part, 3>(t.n_tiles, smem, st, t, fs, in, pairM, g, w_geo, w_photo, part, err);
}
template int launch_dense_tc<float>(const Tables &, const FrameStore &, const Intr &, const float *, Gates, float,
                                    float, float *, int *, int, cudaStream_t);
template int launch_dense_tc<double>(const Tables &, const FrameStore &, const Intr &, const float *, Gates, float,
                                     float, double *, int *, int, cudaStream_t);

}  // namespace bf

// Runs the probe on the current device; see bf.h.
extern "C" bf_status bf_debug_tc_probe(int n_rows, int passes, const float *fa, const float *fb, float *out) {
  using namespace bf;
  if (n_rows <= 0 || n_rows % 64 != 0 || n_rows > (1 << 16) || (passes != 1 && passes != 3) || !fa || !fb || !out)
    return BF_ERR_INVALID_ARG;
  const size_t in_bytes = (size_t)8 * n_rows * 8 * sizeof(float), out_bytes = (size_t)128 * 64 * sizeof(float);
  float *dA = nullptr, *dB = nullptr, *dO = nullptr;
  int *dE = nullptr;
  bf_status st = BF_OK;
  if (cudaMalloc(&dA, in_bytes) != cudaSuccess || cudaMalloc(&dB, in_bytes) != cudaSuccess ||
      cudaMalloc(&dO, out_bytes) != cudaSuccess || cudaMalloc(&dE, sizeof(int)) != cudaSuccess) {
    st = BF_ERR_OUT_OF_MEMORY;
  } else if (cudaMemcpy(dA, fa, in_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dB, fb, in_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(dO, 0, out_bytes) != cudaSuccess || cudaMemset(dE, 0, sizeof(int)) != cudaSuccess) {
    st = BF_ERR_CUDA;
  } else {
    cudaError_t e;
    if (passes == 1) {
      const int smem = TcLayout<1>::bytes;
      e = cudaFuncSetAttribute(k_tc_probe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) k_tc_probe<1><<<1, TC_BS, smem>>>(dA, dB, n_rows, dO, dE);
    } else {
      const int smem = TcLayout<3>::bytes;
      e = cudaFuncSetAttribute(k_tc_probe<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) k_tc_probe<3><<<1, TC_BS, smem>>>(dA, dB, n_rows, dO, dE);
    }
    int herr = 0;
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(out, dO, out_bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&herr, dE, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = BF_ERR_CUDA;
    else if (herr)
      st = BF_ERR_TIMEOUT;
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dO);
  cudaFree(dE);
  return st;
}
